// CUDA-core kernels of the point-source evaluation (fmm.cu): the
// density gather, the leaf check potentials that feed S~, and the leaf sums
// of L2T and of the near field (S2T).  G = 1 / (4 pi |x - y|) (Sec. 4);
// for a double layer, dG/dn(y) = n(y) . (x - y) / (4 pi |x - y|^3) in the
// check potentials and the near field (Sec. 4, Eq. (26)), with the
// densities in the hi words' w and the normals n_j as two FP32 words.
//
// Points live in leaf order in leaf units: s = (x - c) / h with c the
// leaf's centre and h its half-width, stored as two words, hi = s rounded
// to a multiple of 2^-20 (exact in FP32 for |s| < 4) and lo = s - hi
// (|lo| <= 2^-21).
// A neighbour leaf sits at 2 (ijk_s - ijk_b) in these units, so the
// difference of two points is (hi_i - 2 delta - hi_j) + (lo_i - lo_j): the
// first term is exact and the sum carries one rounding relative to the
// distance itself, which keeps close pairs (distances far below the box
// size) at FP32 relative accuracy.
//
// Double layer: for sources on a smooth surface n_j . (x_i - x_j) is of
// order |x_i - x_j|^2 / (2 R) (R the radius of curvature), far below the
// terms n_j,k d_k it is summed from, so an FP32 dot product loses the
// close pairs (1.7e-4 relative L2 on the 65,536-point sphere at depth 5 in
// a NumPy emulation).  The near sums therefore form n . d from the exact
// difference of the hi words with the compensated dot product Dot2 of
// Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005) on the normals' hi
// words, plus the small terms n_lo . d_hi + n_hi . d_lo in plain FP32
// (emulated: 3.7e-7).  The check potentials (sources at least 1.8 leaf
// units from the check points) use a plain FP32 dot product.
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
// n upward check points a u_i (leaf units: a = 3 - 2d), columns n..ld-1 zero;
// double layer (DL): scale * sum_j q_j n_j . (a u_i - s_j) / |a u_i - s_j|^3.
// Thread t takes check points t and t + blockDim.x (blockDim.x >= n / 2).
template <bool DL>
__global__ void __launch_bounds__(kCheckThreads) leaf_check_kernel(const float4* __restrict__ hi,
                                                                   const float4* __restrict__ lo,
                                                                   const float4* __restrict__ nhi,
                                                                   const int* __restrict__ leaf_start,
                                                                   const float4* __restrict__ usurf, int n, float a,
                                                                   float scale, float* __restrict__ out, int ld) {
    __shared__ float4 src[kCheckThreads];
    __shared__ float4 srcm[DL ? kCheckThreads : 1];
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
            if (DL) srcm[tid] = __ldg(nhi + j);
        }
        __syncthreads();
        const int cnt = min(nt, end - c0);
#pragma unroll 4
        for (int jj = 0; jj < cnt; ++jj) {
            const float4 y = src[jj];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float dx = x[k].x - y.x, dy = x[k].y - y.y, dz = x[k].z - y.z;
                if (DL) {
                    const float4 m = srcm[jj];
                    const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    acc[k] = fmaf(y.w * fmaf(m.x, dx, fmaf(m.y, dy, m.z * dz)), ri * ri * ri, acc[k]);
                } else {
                    acc[k] = fmaf(y.w, rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))), acc[k]);
                }
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

// n . d for the double layer: d = dh + dl with dh exact; Dot2 (TwoProduct by
// FMA, TwoSum) on n_hi . dh, then the small terms n_lo . dh + n_hi . dl.
// The explicitly rounded operations keep the compiler from contracting
// the error-free transformations.
__device__ __forceinline__ float normal_dot(const float4& nh, const float4& nl, float dhx, float dhy, float dhz,
                                            float dlx, float dly, float dlz) {
    float p = __fmul_rn(nh.x, dhx);
    float s = fmaf(nh.x, dhx, -p);
    {
        const float hh = __fmul_rn(nh.y, dhy), r = fmaf(nh.y, dhy, -hh);
        const float t = __fadd_rn(p, hh), bb = __fsub_rn(t, p);
        s += __fadd_rn(__fsub_rn(p, __fsub_rn(t, bb)), __fsub_rn(hh, bb)) + r;
        p = t;
    }
    {
        const float hh = __fmul_rn(nh.z, dhz), r = fmaf(nh.z, dhz, -hh);
        const float t = __fadd_rn(p, hh), bb = __fsub_rn(t, p);
        s += __fadd_rn(__fsub_rn(p, __fsub_rn(t, bb)), __fsub_rn(hh, bb)) + r;
        p = t;
    }
    const float corr = fmaf(nl.x, dhx, fmaf(nl.y, dhy, fmaf(nl.z, dhz, fmaf(nh.x, dlx, fmaf(nh.y, dly, nh.z * dlz)))));
    return p + (s + corr);
}

// Double layer: acc[t] += q_j n_j . d / |d|^3 with d = s_t - y_j (y_j's hi
// word shifted), the normals' hi and lo words staged in snh, snl.
template <int T>
__device__ __forceinline__ void near_run_dl(const float4* __restrict__ sh, const float4* __restrict__ sl,
                                            const float4* __restrict__ snh, const float4* __restrict__ snl, int j0,
                                            int j1, const float4 (&xh)[2], const float4 (&xl)[2],
                                            float (&acc)[2][2]) {
    for (int jj = j0; jj < j1; ++jj) {
        const float4 y = sh[jj], l = sl[jj], nh = snh[jj], nl = snl[jj];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float dhx = xh[t].x - y.x, dhy = xh[t].y - y.y, dhz = xh[t].z - y.z;
            const float dlx = xl[t].x - l.x, dly = xl[t].y - l.y, dlz = xl[t].z - l.z;
            const float dx = dhx + dlx, dy = dhy + dly, dz = dhz + dlz;
            const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            const float dot = normal_dot(nh, nl, dhx, dhy, dhz, dlx, dly, dlz);
            acc[t][0] = fmaf(y.w * dot, ri * ri * ri, acc[t][0]);
        }
    }
}

// Double layer over the leaf's own points, skipping the target itself.
template <int T>
__device__ __forceinline__ void self_run_dl(const float4* __restrict__ sh, const float4* __restrict__ sl,
                                            const float4* __restrict__ snh, const float4* __restrict__ snl, int j0,
                                            int j1, int i0, const int (&it)[2], const float4 (&xh)[2],
                                            const float4 (&xl)[2], float (&acc)[2][2]) {
    for (int jj = j0; jj < j1; ++jj) {
        const float4 y = sh[jj], l = sl[jj], nh = snh[jj], nl = snl[jj];
        const int js = i0 + jj - j0;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float dhx = xh[t].x - y.x, dhy = xh[t].y - y.y, dhz = xh[t].z - y.z;
            const float dlx = xl[t].x - l.x, dly = xl[t].y - l.y, dlz = xl[t].z - l.z;
            const float dx = dhx + dlx, dy = dhy + dly, dz = dhz + dlz;
            const bool self = js == it[t];
            const float ri = rsqrtf(self ? 1.f : fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            const float dot = self ? 0.f : normal_dot(nh, nl, dhx, dhy, dhz, dlx, dly, dlz);
            acc[t][1] = fmaf(y.w * dot, ri * ri * ri, acc[t][1]);
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
// with a = 3 - 2d the downward equivalent surface and scale = 1 / (4 pi h);
// double layer (DL): the near sum is scale_dl * sum q_j n_j . d / |d|^3 with
// scale_dl = 1 / (4 pi h^2), the L2T part unchanged.
// Each thread takes two targets (i and i + kEvalThreads) when the pass has
// more than kEvalThreads of them, one otherwise.  The near sources are
// staged kNearCap at a time, every neighbour's hi word shifted by its
// 2 delta (exact), the leaf itself first in its near list so that only its
// segment checks for the target itself.
template <bool DL>
__global__ void __launch_bounds__(kEvalThreads) leaf_eval_kernel(
    const float4* __restrict__ hi, const float4* __restrict__ lo, const float4* __restrict__ nhi,
    const float4* __restrict__ nlo, const int* __restrict__ leaf_start, const int4* __restrict__ leaf_ijk, const int* __restrict__ near_start,
    const int* __restrict__ near_idx, const float4* __restrict__ usurf, int n, float a, float scale, float scale_dl,
    const float* __restrict__ e, int lde, const int* __restrict__ perm, float* __restrict__ out, int parts) {
    __shared__ float4 src_hi[kNearCap];
    __shared__ float4 src_lo[kNearCap];
    __shared__ float4 src_nh[DL ? kNearCap : 1];
    __shared__ float4 src_nl[DL ? kNearCap : 1];
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
        float accd[2][2] = {{0.f, 0.f}, {0.f, 0.f}};  // double layer: the near sum
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
                        if (DL) {
                            src_nh[fill + j] = __ldg(nhi + sb + j);
                            src_nl[fill + j] = __ldg(nlo + sb + j);
                        }
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
                if (DL) {
                    if (two) {
                        self_run_dl<2>(src_hi, src_lo, src_nh, src_nl, self_a, self_a + self_n, self_i0, it, xh, xl,
                                       accd);
                        near_run_dl<2>(src_hi, src_lo, src_nh, src_nl, 0, self_a, xh, xl, accd);
                        near_run_dl<2>(src_hi, src_lo, src_nh, src_nl, self_a + self_n, fill, xh, xl, accd);
                    } else {
                        self_run_dl<1>(src_hi, src_lo, src_nh, src_nl, self_a, self_a + self_n, self_i0, it, xh, xl,
                                       accd);
                        near_run_dl<1>(src_hi, src_lo, src_nh, src_nl, 0, self_a, xh, xl, accd);
                        near_run_dl<1>(src_hi, src_lo, src_nh, src_nl, self_a + self_n, fill, xh, xl, accd);
                    }
                } else if (two) {
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
            if (it[t] < end) {
                float v = scale * (acc[t][0] + acc[t][1]);
                if (DL) v = fmaf(scale_dl, accd[t][0] + accd[t][1], v);
                out[__ldg(perm + it[t])] = v;
            }
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

cudaError_t launch_leaf_check(const float4* hi, const float4* lo, const float4* nhi, const int* leaf_start,
                              int n_leaves, const float4* usurf, int n, float a, float scale, float* out, int ld,
                              cudaStream_t stream) {
    if (n_leaves <= 0) return cudaSuccess;
    if (n > 2 * kCheckThreads || ld < n) return cudaErrorInvalidValue;
    const int threads = ((n + 1) / 2 + 31) / 32 * 32;  // two check points per thread
    if (nhi)
        leaf_check_kernel<true><<<n_leaves, threads, 0, stream>>>(hi, lo, nhi, leaf_start, usurf, n, a, scale, out, ld);
    else
        leaf_check_kernel<false><<<n_leaves, threads, 0, stream>>>(hi, lo, nhi, leaf_start, usurf, n, a, scale, out, ld);
    return cudaGetLastError();
}

cudaError_t launch_leaf_eval(const float4* hi, const float4* lo, const float4* nhi, const float4* nlo,
                             const int* leaf_start, const int4* leaf_ijk, const int* near_start, const int* near_idx,
                             int n_leaves, const float4* usurf, int n, float a, float scale, float scale_dl,
                             const float* e, int lde, const int* perm, float* out, int parts, cudaStream_t stream) {
    if (n_leaves <= 0) return cudaSuccess;
    if ((parts & 2) && (!e || lde < n || n > kNearCap)) return cudaErrorInvalidValue;
    if ((nhi == nullptr) != (nlo == nullptr)) return cudaErrorInvalidValue;
    if (nhi)
        leaf_eval_kernel<true><<<n_leaves, kEvalThreads, 0, stream>>>(hi, lo, nhi, nlo, leaf_start, leaf_ijk,
                                                                      near_start, near_idx, usurf, n, a, scale,
                                                                      scale_dl, e, lde, perm, out, parts);
    else
        leaf_eval_kernel<false><<<n_leaves, kEvalThreads, 0, stream>>>(hi, lo, nhi, nlo, leaf_start, leaf_ijk,
                                                                       near_start, near_idx, usurf, n, a, scale,
                                                                       scale_dl, e, lde, perm, out, parts);
    return cudaGetLastError();
}

}  // namespace kifmm
