// CUDA-core kernels of the point-source evaluation (fmm.cu): the
// density gather, the leaf check potentials that feed S~, and the leaf sums
// of L2T and of the near field (S2T).  G = 1 / (4 pi |x - y|) (Sec. 4).
//
// Points live in leaf order in leaf units: s = (x - c) / h with c the
// leaf's centre and h its half-width, stored as two words, hi = s rounded
// to a multiple of 2^-12 (exact in FP32) and lo = s - hi (|lo| <= 2^-13).
// A neighbour leaf sits at 2 (ijk_s - ijk_b) in these units, so the
// difference of two points is (hi_i - 2 delta - hi_j) + (lo_i - lo_j): the
// first term is exact and the sum carries one rounding relative to the
// distance itself, which keeps close pairs (distances far below the box
// size) at FP32 relative accuracy.
#include <cuda_runtime.h>

#include "kernels.h"

namespace kifmm {
namespace {

constexpr float kInv4Pi = 0.0795774715459476679f;
constexpr int kCheckThreads = 256;  // leaf check kernel: up to 2 * 256 surface points
constexpr int kEvalThreads = 128;   // leaf sum kernel: targets and staged sources per pass

__global__ void gather_density_kernel(const float* __restrict__ q, const int* __restrict__ perm,
                                      float4* __restrict__ pts, int n_points) {  // pts: the hi words, w = q
    float* w = reinterpret_cast<float*>(pts);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_points; i += gridDim.x * blockDim.x)
        w[4 * (long)i + 3] = __ldg(q + __ldg(perm + i));
}

// Block b: out[b][i] = scale * sum_{j in leaf b} q_j / |a u_i - s_j| for the
// n upward check points a u_i (leaf units: a = 3 - 2d), columns n..ld-1 zero.
__global__ void __launch_bounds__(kCheckThreads) leaf_check_kernel(const float4* __restrict__ hi,
                                                                   const float4* __restrict__ lo,
                                                                   const int* __restrict__ leaf_start,
                                                                   const float4* __restrict__ usurf, int n, float a,
                                                                   float scale, float* __restrict__ out, int ld) {
    __shared__ float4 src[kCheckThreads];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int beg = __ldg(leaf_start + b), end = __ldg(leaf_start + b + 1);
    float3 x[2];
    float acc[2] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int i = tid + k * kCheckThreads;
        const float4 u = i < n ? __ldg(usurf + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        x[k] = make_float3(a * u.x, a * u.y, a * u.z);
    }
    for (int c0 = beg; c0 < end; c0 += kCheckThreads) {
        __syncthreads();
        const int j = c0 + tid;
        if (j < end) {
            const float4 h4 = __ldg(hi + j), l4 = __ldg(lo + j);
            src[tid] = make_float4(h4.x + l4.x, h4.y + l4.y, h4.z + l4.z, h4.w);
        }
        __syncthreads();
        const int cnt = min(kCheckThreads, end - c0);
#pragma unroll 4
        for (int jj = 0; jj < cnt; ++jj) {
            const float4 y = src[jj];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float dx = x[k].x - y.x, dy = x[k].y - y.y, dz = x[k].z - y.z;
                acc[k] = fmaf(y.w, rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))), acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int i = tid + k * kCheckThreads;
        if (i < n) out[(long)b * ld + i] = scale * acc[k];
    }
    for (int i = n + tid; i < ld; i += kCheckThreads) out[(long)b * ld + i] = 0.f;
}

// Block b, every point i of leaf b (leaf units):
//   out[perm[i]] = scale * ( sum_{j < n} e[b][j] / |s_i - a u_j|                    (L2T, parts & 2)
//                          + sum_{s near b} sum_{j in s, j != i} q_j / |s_i - 2 delta_s - s_j| )
//                                                                                     (S2T, parts & 1)
// with a = 3 - 2d the downward equivalent surface and scale = 1 / (4 pi h).
__global__ void __launch_bounds__(kEvalThreads) leaf_eval_kernel(
    const float4* __restrict__ hi, const float4* __restrict__ lo, const int* __restrict__ leaf_start,
    const int4* __restrict__ leaf_ijk, const int* __restrict__ near_start, const int* __restrict__ near_idx,
    const float4* __restrict__ usurf, int n, float a, float scale, const float* __restrict__ e, int lde,
    const int* __restrict__ perm, float* __restrict__ out, int parts) {
    __shared__ float4 src_hi[kEvalThreads];
    __shared__ float4 src_lo[kEvalThreads];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int beg = __ldg(leaf_start + b), end = __ldg(leaf_start + b + 1);
    const int4 cb = __ldg(leaf_ijk + b);
    for (int t0 = beg; t0 < end; t0 += kEvalThreads) {
        const int i = t0 + tid;
        const float4 xh = i < end ? __ldg(hi + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 xl = i < end ? __ldg(lo + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        float acc = 0.f;
        if (parts & 2) {
            const float sx = xh.x + xl.x, sy = xh.y + xl.y, sz = xh.z + xl.z;
            for (int j0 = 0; j0 < n; j0 += kEvalThreads) {
                __syncthreads();
                const int j = j0 + tid;
                if (j < n) {
                    const float4 u = __ldg(usurf + j);
                    src_hi[tid] = make_float4(a * u.x, a * u.y, a * u.z, __ldg(e + (long)b * lde + j));
                }
                __syncthreads();
                const int cnt = min(kEvalThreads, n - j0);
#pragma unroll 4
                for (int jj = 0; jj < cnt; ++jj) {
                    const float4 y = src_hi[jj];
                    const float dx = sx - y.x, dy = sy - y.y, dz = sz - y.z;
                    acc = fmaf(y.w, rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))), acc);
                }
            }
        }
        if (parts & 1) {
            const int nb = __ldg(near_start + b), ne = __ldg(near_start + b + 1);
            for (int k = nb; k < ne; ++k) {
                const int s = __ldg(near_idx + k);
                const int4 cs = __ldg(leaf_ijk + s);
                // the target's hi word in the source leaf's frame: exact
                const float hx = xh.x - 2.f * (float)(cs.x - cb.x), hy = xh.y - 2.f * (float)(cs.y - cb.y),
                            hz = xh.z - 2.f * (float)(cs.z - cb.z);
                const int sb = __ldg(leaf_start + s), se = __ldg(leaf_start + s + 1);
                for (int j0 = sb; j0 < se; j0 += kEvalThreads) {
                    __syncthreads();
                    const int j = j0 + tid;
                    if (j < se) {
                        src_hi[tid] = __ldg(hi + j);
                        src_lo[tid] = __ldg(lo + j);
                    }
                    __syncthreads();
                    const int cnt = min(kEvalThreads, se - j0);
                    if (s == b) {
                        // the leaf itself: a point does not act on itself
                        for (int jj = 0; jj < cnt; ++jj) {
                            const float4 y = src_hi[jj], yl = src_lo[jj];
                            const float dx = (hx - y.x) + (xl.x - yl.x), dy = (hy - y.y) + (xl.y - yl.y),
                                        dz = (hz - y.z) + (xl.z - yl.z);
                            const bool self = j0 + jj == i;
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            acc = fmaf(self ? 0.f : y.w, rsqrtf(self ? 1.f : r2), acc);
                        }
                    } else {
#pragma unroll 4
                        for (int jj = 0; jj < cnt; ++jj) {
                            const float4 y = src_hi[jj], yl = src_lo[jj];
                            const float dx = (hx - y.x) + (xl.x - yl.x), dy = (hy - y.y) + (xl.y - yl.y),
                                        dz = (hz - y.z) + (xl.z - yl.z);
                            acc = fmaf(y.w, rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))), acc);
                        }
                    }
                }
            }
        }
        if (i < end) out[__ldg(perm + i)] = scale * acc;
    }
}

}  // namespace

cudaError_t launch_gather_density(const float* q, const int* perm, float4* pts, int n_points, cudaStream_t stream) {
    if (n_points <= 0) return cudaSuccess;
    int blocks = (n_points + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    gather_density_kernel<<<blocks, 256, 0, stream>>>(q, perm, pts, n_points);
    return cudaGetLastError();
}

cudaError_t launch_leaf_check(const float4* hi, const float4* lo, const int* leaf_start, int n_leaves,
                              const float4* usurf, int n, float a, float scale, float* out, int ld,
                              cudaStream_t stream) {
    if (n_leaves <= 0) return cudaSuccess;
    if (n > 2 * kCheckThreads || ld < n) return cudaErrorInvalidValue;
    leaf_check_kernel<<<n_leaves, kCheckThreads, 0, stream>>>(hi, lo, leaf_start, usurf, n, a, scale, out, ld);
    return cudaGetLastError();
}

cudaError_t launch_leaf_eval(const float4* hi, const float4* lo, const int* leaf_start, const int4* leaf_ijk,
                             const int* near_start, const int* near_idx, int n_leaves, const float4* usurf, int n,
                             float a, float scale, const float* e, int lde, const int* perm, float* out, int parts,
                             cudaStream_t stream) {
    if (n_leaves <= 0) return cudaSuccess;
    if ((parts & 2) && (!e || lde < n)) return cudaErrorInvalidValue;
    leaf_eval_kernel<<<n_leaves, kEvalThreads, 0, stream>>>(hi, lo, leaf_start, leaf_ijk, near_start, near_idx, usurf,
                                                            n, a, scale, e, lde, perm, out, parts);
    return cudaGetLastError();
}

}  // namespace kifmm
