// CUDA-core kernels of the point-source evaluation (fmm.cu): the
// density gather, the per-point compressed S~ / T~ rows (FP64, once per tree
// and per set of normals), the S~ sums over a leaf's points, and the leaf
// sums of the far field (a row against p~) and of the near field (S2T).  G = 1 / (4 pi |x - y|) (Sec. 4);
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
#include <cuda_bf16.h>

#include "kernels.h"

namespace kifmm {
namespace {

constexpr float kInv4Pi = 0.0795774715459476679f;
constexpr int kEvalThreads = 64;    // leaf sum kernel: threads, each with up to two targets
constexpr int kNearCap = 512;       // leaf sum kernel: staged sources per pass (>= n surface points)

__global__ void gather_density_kernel(const float* __restrict__ q, const int* __restrict__ perm,
                                      float4* __restrict__ pts, int n_points) {  // pts: the hi words, w = q
    float* w = reinterpret_cast<float*>(pts);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_points; i += gridDim.x * blockDim.x)
        w[4 * (long)i + 3] = __ldg(q + __ldg(perm + i));
}

// Per-point compressed rows (Sec. 3.3's S~ = R~^T S and T~ = T U~ applied to
// one point), in FP64: rows[j][a] = scale * sum_i Ws[a][i] g(x_i, s_j) for
// the n check points x_i (leaf units) and the point s_j, with
//   g = 1 / |x_i - s_j|                        (point charges; the same row
//                                               serves S~ and T~ + L2T)
//   g = n_j . (x_i - s_j) / |x_i - s_j|^3      (dipoles: S~ of the double layer)
// Ws is [rp][n] (rows past the rank zero).  Block: 32 points x all rp
// coefficients; the check points go through shared memory 16 at a time with
// the matching columns of Ws (transposed, coefficient-contiguous); thread
// (ty, tx) accumulates points 2 ty, 2 ty + 1 and coefficients tx + 16 k.
constexpr int kRowPts = 32, kRowChunk = 16, kRowMaxK = 18;  // rp <= 288

__global__ void __launch_bounds__(256) point_rows_kernel(const double* __restrict__ pts, const double* __restrict__ nrm,
                                                         int n_points, const double* __restrict__ ws, int rp, int n,
                                                         const double* __restrict__ xsurf, double scale,
                                                         float* __restrict__ rows) {
    __shared__ double g_s[kRowPts][kRowChunk + 1];
    __shared__ double w_s[kRowChunk][kRowMaxK * 16];
    __shared__ double x_s[kRowChunk][3];
    __shared__ double p_s[kRowPts][6];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int j0 = blockIdx.x * kRowPts;
    const int ka = (rp + 15) / 16;
    if (tid < kRowPts) {
        const int j = j0 + tid;
        for (int t = 0; t < 3; ++t) {
            p_s[tid][t] = j < n_points ? pts[3 * (long)j + t] : 0.0;
            p_s[tid][3 + t] = (nrm && j < n_points) ? nrm[3 * (long)j + t] : 0.0;
        }
    }
    double acc[2][kRowMaxK];
#pragma unroll
    for (int k = 0; k < kRowMaxK; ++k) acc[0][k] = acc[1][k] = 0.0;
    for (int i0 = 0; i0 < n; i0 += kRowChunk) {
        __syncthreads();
        if (tid < kRowChunk * 3) {
            const int i = i0 + tid / 3;
            x_s[tid / 3][tid % 3] = i < n ? xsurf[3 * i + tid % 3] : 0.0;
        }
        for (int e = tid; e < kRowChunk * ka * 16; e += blockDim.x) {
            const int ii = e / (ka * 16), a = e % (ka * 16), i = i0 + ii;
            w_s[ii][a] = (i < n && a < rp) ? ws[(long)a * n + i] : 0.0;
        }
        __syncthreads();
        for (int e = tid; e < kRowPts * kRowChunk; e += blockDim.x) {
            const int pt = e / kRowChunk, ii = e % kRowChunk;
            double g = 0.0;
            if (i0 + ii < n && j0 + pt < n_points) {
                const double dx = x_s[ii][0] - p_s[pt][0], dy = x_s[ii][1] - p_s[pt][1], dz = x_s[ii][2] - p_s[pt][2];
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double ri = 1.0 / sqrt(r2);
                g = nrm ? (p_s[pt][3] * dx + p_s[pt][4] * dy + p_s[pt][5] * dz) * ri * ri * ri : ri;
            }
            g_s[pt][ii] = g;
        }
        __syncthreads();
#pragma unroll 4
        for (int ii = 0; ii < kRowChunk; ++ii) {
            const double g0 = g_s[2 * ty][ii], g1 = g_s[2 * ty + 1][ii];
#pragma unroll
            for (int k = 0; k < kRowMaxK; ++k) {
                if (k < ka) {
                    const double w = w_s[ii][tx + 16 * k];
                    acc[0][k] = fma(w, g0, acc[0][k]);
                    acc[1][k] = fma(w, g1, acc[1][k]);
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int j = j0 + 2 * ty + t;
        if (j >= n_points) continue;
#pragma unroll
        for (int k = 0; k < kRowMaxK; ++k) {
            const int a = tx + 16 * k;
            if (k < ka && a < rp) rows[(long)j * rp + a] = (float)(scale * acc[t][k]);
        }
    }
}

// S~ through the rows: q~_b[a] = sum_{j in leaf b} q_j rows[j][a] (q_j in the
// hi words' w), FP32 with Neumaier's compensated summation (TwoSum of
// Knuth / Moller, explicitly rounded so that no contraction breaks it).
// One block per leaf, thread t takes coefficients 4 t .. 4 t + 3.  Writes the
// FP32 row qf[b] and its three BF16 pieces qb[pc][b] (piece stride pstride).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
    const float t = __fadd_rn(s, x);
    const float e = fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
    s = t;
    c = __fadd_rn(c, e);
}

__global__ void leaf_rows_sum_kernel(const float* __restrict__ rows, const float4* __restrict__ hi,
                                     const int* __restrict__ leaf_start, int rp, float* __restrict__ qf,
                                     __nv_bfloat16* __restrict__ qb, long pstride) {
    const int b = blockIdx.x, t = threadIdx.x;
    if (4 * t >= rp) return;
    const int beg = __ldg(leaf_start + b), end = __ldg(leaf_start + b + 1);
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    const float* wq = reinterpret_cast<const float*>(hi) + 3;
    for (int j = beg; j < end; ++j) {
        const float q = __ldg(wq + 4 * (long)j);
        const float4 r = __ldg(reinterpret_cast<const float4*>(rows + (long)j * rp) + t);
        two_sum_acc(s[0], c[0], __fmul_rn(q, r.x));
        two_sum_acc(s[1], c[1], __fmul_rn(q, r.y));
        two_sum_acc(s[2], c[2], __fmul_rn(q, r.z));
        two_sum_acc(s[3], c[3], __fmul_rn(q, r.w));
    }
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __fadd_rn(s[k], c[k]);
    reinterpret_cast<float4*>(qf + (long)b * rp)[t] = make_float4(v[0], v[1], v[2], v[3]);
    // three BF16 pieces, each the rounding of what the earlier ones left
#pragma unroll
    for (int pc = 0; pc < 3; ++pc) {
        __nv_bfloat16 o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[k] = __float2bfloat16_rn(v[k]);
            v[k] = __fsub_rn(v[k], __bfloat162float(o[k]));
        }
        __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(qb + pc * pstride + (long)b * rp + 4 * t);
        dst[0] = __halves2bfloat162(o[0], o[1]);
        dst[1] = __halves2bfloat162(o[2], o[3]);
    }
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
//   out[perm[i]] = trows[i] . p~_b                                                   (far field, parts & 2)
//                + scale * sum_{s near b} sum_{j in s, j != i} q_j / |s_i - 2 delta_s - s_j|
//                                                                                     (S2T, parts & 1)
// with trows[i] the point's T~ row (T~ + L2T of Sec. 3.3 for that point,
// formed in FP64 by point_rows_kernel), p~_b the leaf's compressed downward
// check potentials and scale = 1 / (4 pi h); double layer (DL): the near sum
// is scale_dl * sum q_j n_j . d / |d|^3 with scale_dl = 1 / (4 pi h^2).
// Each thread takes two targets (i and i + kEvalThreads) when the pass has
// more than kEvalThreads of them, one otherwise.  The near sources are
// staged kNearCap at a time, every neighbour's hi word shifted by its
// 2 delta (exact), the leaf itself first in its near list so that only its
// segment checks for the target itself.
template <bool DL>
__global__ void __launch_bounds__(kEvalThreads) leaf_eval_kernel(
    const float4* __restrict__ hi, const float4* __restrict__ lo, const float4* __restrict__ nhi,
    const float4* __restrict__ nlo, const int* __restrict__ leaf_start, const int4* __restrict__ leaf_ijk, const int* __restrict__ near_start,
    const int* __restrict__ near_idx, const float* __restrict__ trows, int rp, const float* __restrict__ pleaf,
    float scale, float scale_dl, const int* __restrict__ perm, float* __restrict__ out, int parts) {
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
        float far[2] = {0.f, 0.f};
        if (parts & 2) {
            // far field: the target's T~ row against the leaf's p~ (staged)
            float* pbuf = reinterpret_cast<float*>(src_lo);
            __syncthreads();
            for (int j = tid; j < rp; j += kEvalThreads) pbuf[j] = __ldg(pleaf + (long)b * rp + j);
            __syncthreads();
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (it[t] >= end) continue;
                const float4* row = reinterpret_cast<const float4*>(trows + (long)it[t] * rp);
                const float4* pv = reinterpret_cast<const float4*>(pbuf);
                float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int k = 0; k < rp / 4; ++k) {
                    const float4 w = __ldg(row + k), pk = pv[k];
                    d.x = fmaf(w.x, pk.x, d.x);
                    d.y = fmaf(w.y, pk.y, d.y);
                    d.z = fmaf(w.z, pk.z, d.z);
                    d.w = fmaf(w.w, pk.w, d.w);
                }
                far[t] = (d.x + d.y) + (d.z + d.w);
            }
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
                float v = fmaf(scale, acc[t][0] + acc[t][1], far[t]);
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

cudaError_t launch_point_rows(const double* pts, const double* nrm, int n_points, const double* ws, int rp, int n,
                              const double* xsurf, double scale, float* rows, cudaStream_t stream) {
    if (n_points <= 0) return cudaSuccess;
    if (rp > kRowMaxK * 16 || rp % 16 != 0 || n < 1) return cudaErrorInvalidValue;
    const int blocks = (n_points + kRowPts - 1) / kRowPts;
    point_rows_kernel<<<blocks, 256, 0, stream>>>(pts, nrm, n_points, ws, rp, n, xsurf, scale, rows);
    return cudaGetLastError();
}

cudaError_t launch_leaf_rows_sum(const float* rows, const float4* hi, const int* leaf_start, int n_leaves, int rp,
                                 float* qf, __nv_bfloat16* qb, long pstride, cudaStream_t stream) {
    if (n_leaves <= 0) return cudaSuccess;
    if (rp % 16 != 0 || rp > 1024) return cudaErrorInvalidValue;
    const int threads = ((rp / 4) + 31) / 32 * 32;
    leaf_rows_sum_kernel<<<n_leaves, threads, 0, stream>>>(rows, hi, leaf_start, rp, qf, qb, pstride);
    return cudaGetLastError();
}

cudaError_t launch_leaf_eval(const float4* hi, const float4* lo, const float4* nhi, const float4* nlo,
                             const int* leaf_start, const int4* leaf_ijk, const int* near_start, const int* near_idx,
                             int n_leaves, const float* trows, int rp, const float* pleaf, float scale, float scale_dl,
                             const int* perm, float* out, int parts, cudaStream_t stream) {
    if (n_leaves <= 0) return cudaSuccess;
    if ((parts & 2) && (!trows || !pleaf || rp % 16 != 0 || rp > 4 * kNearCap)) return cudaErrorInvalidValue;
    if ((nhi == nullptr) != (nlo == nullptr)) return cudaErrorInvalidValue;
    if (nhi)
        leaf_eval_kernel<true><<<n_leaves, kEvalThreads, 0, stream>>>(hi, lo, nhi, nlo, leaf_start, leaf_ijk,
                                                                      near_start, near_idx, trows, rp, pleaf, scale,
                                                                      scale_dl, perm, out, parts);
    else
        leaf_eval_kernel<false><<<n_leaves, kEvalThreads, 0, stream>>>(hi, lo, nhi, nlo, leaf_start, leaf_ijk,
                                                                       near_start, near_idx, trows, rp, pleaf, scale,
                                                                       scale_dl, perm, out, parts);
    return cudaGetLastError();
}

}  // namespace kifmm
