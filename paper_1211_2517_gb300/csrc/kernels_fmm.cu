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
constexpr int kEvalThreads = 64;    // leaf sum kernel: threads, each with up to two targets
constexpr int kNearCap = 512;       // leaf sum kernel: staged sources per pass (>= n surface points)

__global__ void gather_density_kernel(const float* __restrict__ q, const int* __restrict__ perm,
                                      float4* __restrict__ pts, int n_points) {  // pts: the hi words, w = q
    float* w = reinterpret_cast<float*>(pts);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_points; i += gridDim.x * blockDim.x)
        w[4 * (long)i + 3] = __ldg(q + __ldg(perm + i));
}

// Block b: out[b][i] = scale * sum_{j in leaf b} q_j / |a u_i - s_j| for the
// n upward check points a u_i (leaf units: a = 3 - 2d), columns n..ld-1 zero.
// Thread t takes check points t and t + blockDim.x (blockDim.x >= n / 2).
__global__ void __launch_bounds__(kCheckThreads) leaf_check_kernel(const float4* __restrict__ hi,
                                                                   const float4* __restrict__ lo,
                                                                   const int* __restrict__ leaf_start,
                                                                   const float4* __restrict__ usurf, int n, float a,
                                                                   float scale, float* __restrict__ out, int ld) {
    __shared__ float4 src[kCheckThreads];
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int beg = __ldg(leaf_start + b), end = __ldg(leaf_start + b + 1);
    float3 x[2];
    float acc[2] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int i = tid + k * nt;
        const float4 u = i < n ? __ldg(usurf + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        x[k] = make_float3(a * u.x, a * u.y, a * u.z);
    }
    for (int c0 = beg; c0 < end; c0 += nt) {
        __syncthreads();
        const int j = c0 + tid;
        if (j < end) {
            const float4 h4 = __ldg(hi + j), l4 = __ldg(lo + j);
            src[tid] = make_float4(h4.x + l4.x, h4.y + l4.y, h4.z + l4.z, h4.w);
        }
        __syncthreads();
        const int cnt = min(nt, end - c0);
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
        const int i = tid + k * nt;
        if (i < n) out[(long)b * ld + i] = scale * acc[k];
    }
    for (int i = n + tid; i < ld; i += nt) out[(long)b * ld + i] = 0.f;
}

// Interactions of T targets (leaf units, hi + lo words) with the staged
// sources [j0, j1): acc[t] += q_j / |s_t - y_j|, two sources per step.
template <int T>
__device__ __forceinline__ void near_run(const float4* __restrict__ sh, const float4* __restrict__ sl, int j0, int j1,
                                         const float4 (&xh)[2], const float4 (&xl)[2], float (&acc)[2][2]) {
    int jj = j0;
    for (; jj + 1 < j1; jj += 2) {
        const float4 y0 = sh[jj], l0 = sl[jj], y1 = sh[jj + 1], l1 = sl[jj + 1];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float dx0 = (xh[t].x - y0.x) + (xl[t].x - l0.x), dy0 = (xh[t].y - y0.y) + (xl[t].y - l0.y),
                        dz0 = (xh[t].z - y0.z) + (xl[t].z - l0.z);
            const float dx1 = (xh[t].x - y1.x) + (xl[t].x - l1.x), dy1 = (xh[t].y - y1.y) + (xl[t].y - l1.y),
                        dz1 = (xh[t].z - y1.z) + (xl[t].z - l1.z);
            acc[t][0] = fmaf(y0.w, rsqrtf(fmaf(dx0, dx0, fmaf(dy0, dy0, dz0 * dz0))), acc[t][0]);
            acc[t][1] = fmaf(y1.w, rsqrtf(fmaf(dx1, dx1, fmaf(dy1, dy1, dz1 * dz1))), acc[t][1]);
        }
    }
    if (jj < j1) {
        const float4 y0 = sh[jj], l0 = sl[jj];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float dx0 = (xh[t].x - y0.x) + (xl[t].x - l0.x), dy0 = (xh[t].y - y0.y) + (xl[t].y - l0.y),
                        dz0 = (xh[t].z - y0.z) + (xl[t].z - l0.z);
            acc[t][0] = fmaf(y0.w, rsqrtf(fmaf(dx0, dx0, fmaf(dy0, dy0, dz0 * dz0))), acc[t][0]);
        }
    }
}

// The same over the leaf's own points [j0, j1) (sorted indices i0 + jj - j0),
// skipping the target itself (sorted index it[t]).
template <int T>
__device__ __forceinline__ void self_run(const float4* __restrict__ sh, const float4* __restrict__ sl, int j0, int j1,
                                         int i0, const int (&it)[2], const float4 (&xh)[2], const float4 (&xl)[2],
                                         float (&acc)[2][2]) {
    for (int jj = j0; jj < j1; ++jj) {
        const float4 y = sh[jj], yl = sl[jj];
        const int js = i0 + jj - j0;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float dx = (xh[t].x - y.x) + (xl[t].x - yl.x), dy = (xh[t].y - y.y) + (xl[t].y - yl.y),
                        dz = (xh[t].z - y.z) + (xl[t].z - yl.z);
            const bool self = js == it[t];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            acc[t][1] = fmaf(self ? 0.f : y.w, rsqrtf(self ? 1.f : r2), acc[t][1]);
        }
    }
}

// Block b, every point i of leaf b (leaf units):
//   out[perm[i]] = scale * ( sum_{j < n} e[b][j] / |s_i - a u_j|                    (L2T, parts & 2)
//                          + sum_{s near b} sum_{j in s, j != i} q_j / |s_i - 2 delta_s - s_j| )
//                                                                                     (S2T, parts & 1)
// with a = 3 - 2d the downward equivalent surface and scale = 1 / (4 pi h).
// Each thread takes two targets (i and i + kEvalThreads) when the pass has
// more than kEvalThreads of them, one otherwise.  The near sources are
// staged kNearCap at a time, every neighbour's hi word shifted by its
// 2 delta (exact), the leaf itself first in its near list so that only its
// segment checks for the target itself.
__global__ void __launch_bounds__(kEvalThreads) leaf_eval_kernel(
    const float4* __restrict__ hi, const float4* __restrict__ lo, const int* __restrict__ leaf_start,
    const int4* __restrict__ leaf_ijk, const int* __restrict__ near_start, const int* __restrict__ near_idx,
    const float4* __restrict__ usurf, int n, float a, float scale, const float* __restrict__ e, int lde,
    const int* __restrict__ perm, float* __restrict__ out, int parts) {
    __shared__ float4 src_hi[kNearCap];
    __shared__ float4 src_lo[kNearCap];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int beg = __ldg(leaf_start + b), end = __ldg(leaf_start + b + 1);
    const int4 cb = __ldg(leaf_ijk + b);
    const int nb = __ldg(near_start + b), ne = __ldg(near_start + b + 1);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t0 = beg; t0 < end; t0 += 2 * kEvalThreads) {
        const bool two = t0 + kEvalThreads < end;  // block-uniform
        int it[2] = {t0 + tid, t0 + kEvalThreads + tid};
        float4 xh[2], xl[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            xh[t] = it[t] < end ? __ldg(hi + it[t]) : zero4;
            xl[t] = it[t] < end ? __ldg(lo + it[t]) : zero4;
        }
        float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
        if (parts & 2) {
            // L2T: the surface points as sources with lo = 0 and the targets' own lo
            __syncthreads();
            for (int j = tid; j < n; j += kEvalThreads) {
                const float4 u = __ldg(usurf + j);
                src_hi[j] = make_float4(a * u.x, a * u.y, a * u.z, __ldg(e + (long)b * lde + j));
                src_lo[j] = zero4;
            }
            __syncthreads();
            if (two) near_run<2>(src_hi, src_lo, 0, n, xh, xl, acc);
            else near_run<1>(src_hi, src_lo, 0, n, xh, xl, acc);
        }
        if (parts & 1) {
            int k = nb, seg_off = 0;  // next near leaf and the part of it already staged
            while (k < ne) {
                // stage up to kNearCap sources; [self_a, self_a + self_n) holds the
                // leaf's own points from sorted index self_i0 on
                int fill = 0, self_a = 0, self_n = 0, self_i0 = 0;
                __syncthreads();
                while (k < ne && fill < kNearCap) {
                    const int s = __ldg(near_idx + k);
                    const int sb = __ldg(leaf_start + s) + seg_off, se = __ldg(leaf_start + s + 1);
                    const int take = min(se - sb, kNearCap - fill);
                    const int4 cs = __ldg(leaf_ijk + s);
                    const float ox = 2.f * (float)(cs.x - cb.x), oy = 2.f * (float)(cs.y - cb.y),
                                oz = 2.f * (float)(cs.z - cb.z);
                    for (int j = tid; j < take; j += kEvalThreads) {
                        const float4 h4 = __ldg(hi + sb + j);
                        src_hi[fill + j] = make_float4(h4.x + ox, h4.y + oy, h4.z + oz, h4.w);
                        src_lo[fill + j] = __ldg(lo + sb + j);
                    }
                    if (s == b) {
                        self_a = fill;
                        self_n = take;
                        self_i0 = sb;
                    }
                    fill += take;
                    if (sb + take == se) {
                        ++k;
                        seg_off = 0;
                    } else {
                        seg_off += take;
                    }
                }
                __syncthreads();
                if (two) {
                    self_run<2>(src_hi, src_lo, self_a, self_a + self_n, self_i0, it, xh, xl, acc);
                    near_run<2>(src_hi, src_lo, 0, self_a, xh, xl, acc);
                    near_run<2>(src_hi, src_lo, self_a + self_n, fill, xh, xl, acc);
                } else {
                    self_run<1>(src_hi, src_lo, self_a, self_a + self_n, self_i0, it, xh, xl, acc);
                    near_run<1>(src_hi, src_lo, 0, self_a, xh, xl, acc);
                    near_run<1>(src_hi, src_lo, self_a + self_n, fill, xh, xl, acc);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 2; ++t)
            if (it[t] < end) out[__ldg(perm + it[t])] = scale * (acc[t][0] + acc[t][1]);
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
    const int threads = ((n + 1) / 2 + 31) / 32 * 32;  // two check points per thread
    leaf_check_kernel<<<n_leaves, threads, 0, stream>>>(hi, lo, leaf_start, usurf, n, a, scale, out, ld);
    return cudaGetLastError();
}

cudaError_t launch_leaf_eval(const float4* hi, const float4* lo, const int* leaf_start, const int4* leaf_ijk,
                             const int* near_start, const int* near_idx, int n_leaves, const float4* usurf, int n,
                             float a, float scale, const float* e, int lde, const int* perm, float* out, int parts,
                             cudaStream_t stream) {
    if (n_leaves <= 0) return cudaSuccess;
    if ((parts & 2) && (!e || lde < n || n > kNearCap)) return cudaErrorInvalidValue;
    leaf_eval_kernel<<<n_leaves, kEvalThreads, 0, stream>>>(hi, lo, leaf_start, leaf_ijk, near_start, near_idx, usurf,
                                                            n, a, scale, e, lde, perm, out, parts);
    return cudaGetLastError();
}

}  // namespace kifmm
