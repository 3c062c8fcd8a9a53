// CUDA-core (SIMT) FP32 kernels of the M2L path.
//
//  * pairs_gemm      D[dst row] += alpha A[src row] W_o^T over offset-grouped
//                    box pairs, a row gather from the sources and an atomic
//                    scatter-add into the targets: the FP32 core
//                    sum_o K~_o q~ and the dense baseline sum_o K_o q
//                    (Eq. (4)).
//  * split_bf16      FP32 -> sum of BF16 pieces for the tensor-core modes.
//
// Tiling: a 256-thread block computes a 128 x 128 output tile in K-steps of
// 8 staged through shared memory (double-buffered); each thread owns an
// 8 x 8 register block (8 contiguous rows, two groups of 4 columns).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace kifmm {

namespace {

constexpr int BM = 128, BN = 128, BK = 8, NT = 256;

struct RowMapPairs {
    const int* src;
    const int* dst;
    int nrhs, pair_begin, row0, nrows;
    __device__ __forceinline__ bool valid(int v) const { return v < nrows; }
    __device__ __forceinline__ long a_row(int v) const {
        const int g = row0 + v;
        const int pr = pair_begin + g / nrhs;
        return (long)src[pr] * nrhs + (g % nrhs);
    }
    __device__ __forceinline__ long d_row(int v) const {
        const int g = row0 + v;
        const int pr = pair_begin + g / nrhs;
        return (long)dst[pr] * nrhs + (g % nrhs);
    }
};

// Accumulate the 128x128 tile into acc.
template <class Map>
__device__ __forceinline__ void tile_product(const float* __restrict__ A, int lda, const float* __restrict__ W, int N,
                                             int K, int n0, const Map& map, float (&acc)[8][8],
                                             float (*As)[BK][BM], float (*Ws)[BK][BN]) {
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    // loader coordinates: row lr, k-offset lk (4 floats)
    const int lr = tid >> 1, lk = (tid & 1) * 4;
    const bool a_ok = map.valid(lr);
    const float* a_ptr = a_ok ? A + map.a_row(lr) * (long)lda : A;
    const bool w_ok = (n0 + lr) < N;
    const float* w_ptr = W + (long)(w_ok ? n0 + lr : 0) * K;

#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    auto load = [&](int k0, float4& av, float4& wv) {
        const int kk = k0 + lk;
        av = make_float4(0.f, 0.f, 0.f, 0.f);
        wv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kk < K) {  // K is a multiple of 4
            if (a_ok) av = *reinterpret_cast<const float4*>(a_ptr + kk);
            if (w_ok) wv = __ldg(reinterpret_cast<const float4*>(w_ptr + kk));
        }
    };
    auto store = [&](int buf, const float4& av, const float4& wv) {
        As[buf][lk + 0][lr] = av.x;
        As[buf][lk + 1][lr] = av.y;
        As[buf][lk + 2][lr] = av.z;
        As[buf][lk + 3][lr] = av.w;
        Ws[buf][lk + 0][lr] = wv.x;
        Ws[buf][lk + 1][lr] = wv.y;
        Ws[buf][lk + 2][lr] = wv.z;
        Ws[buf][lk + 3][lr] = wv.w;
    };

    float4 av, wv;
    load(0, av, wv);
    store(0, av, wv);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) load(k0 + BK, av, wv);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8 + 4]);
            const float4 w0 = *reinterpret_cast<const float4*>(&Ws[buf][k][tx * 4]);
            const float4 w1 = *reinterpret_cast<const float4*>(&Ws[buf][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
        }
        if (more) {
            store(buf ^ 1, av, wv);
            __syncthreads();
            buf ^= 1;
        }
    }
}

__global__ void __launch_bounds__(NT) pairs_gemm_kernel(const float* __restrict__ A, int lda,
                                                        const float* __restrict__ W, int N, int K,
                                                        float* __restrict__ D, int ldd, const Tile* __restrict__ tiles,
                                                        const int* __restrict__ src, const int* __restrict__ dst,
                                                        int nrhs, const ScaleTable scales) {
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Ws[2][BK][BN];
    const Tile t = tiles[blockIdx.x];
    const int n0 = blockIdx.y * BN;
    RowMapPairs map{src, dst, nrhs, t.pair_begin, t.row0, t.nrows};
    float acc[8][8];
    tile_product(A, lda, W + (long)(t.k & 0xFFFF) * N * K, N, K, n0, map, acc, As, Ws);
    const float alpha = scales.s[(t.k >> 16) & 31];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int v = ty * 8 + i;
        if (!map.valid(v)) continue;
        float* drow = D + map.d_row(v) * ldd;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (col < N) atomicAdd(drow + col, alpha * acc[i][j]);
        }
    }
}

__global__ void split_bf16_kernel(const float* __restrict__ x, int rows, int cols, int ld,
                                  __nv_bfloat16* __restrict__ out, long piece_stride, int pieces) {
    const long total = (long)rows * cols;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long r = e / cols, c = e % cols;
        float v = x[r * ld + c];
        for (int p = 0; p < pieces; ++p) {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            out[p * piece_stride + e] = h;
            v -= __bfloat162float(h);  // exact: the residual of a bf16 rounding is representable
        }
    }
}

// Block (t, s) covers rows [16 s, 16 s + 16) of 128-row virtual tile t: the
// rows of one segment (or of the single input) split into BF16 pieces,
// output row t * 128 + r <- input row
// (t - tile_begin) * 128 + r of the tile's segment; columns [cols, ldo) and
// rows past the segment's m_rows are written as zero (skipped when
// pad_rows == 0).  x = x_0 + x_1 + x_2
// with each piece rounded to nearest from the remaining residual.
__global__ void split_rows_kernel(const float* __restrict__ A, int m_rows, int lda, int cols, int ldo,
                                  const RowSeg* __restrict__ segs, int n_segs, __nv_bfloat16* __restrict__ out,
                                  long piece_stride, int pieces, int pad_rows, float* __restrict__ row_inv,
                                  int norm_shift) {
    const int t = blockIdx.x;  // virtual tile; blockIdx.y: 16-row slab of it
    __shared__ int s_seg;
    __shared__ unsigned s_max[16];  // row_inv: bits of the slab rows' largest |x| (ordered as integers)
    const float* src = A;
    int m = m_rows;
    long r0 = (long)t * 128;
    long out0 = r0;  // output row of the tile's first row
    if (row_inv && threadIdx.x < 16) s_max[threadIdx.x] = 0u;
    if (n_segs > 0) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_segs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (segs[mid].tile_begin <= t) lo = mid;
                else hi = mid - 1;
            }
            s_seg = lo;
        }
        __syncthreads();
        const RowSeg sg = segs[s_seg];
        src = sg.Af;
        m = sg.m_rows;
        r0 = (long)(t - sg.tile_begin) * 128;
        out0 = sg.out_row + r0;
    }
    if (row_inv) __syncthreads();
    const int c4n = ldo / 4;
    for (int e = threadIdx.x; e < 16 * c4n; e += blockDim.x) {
        const int r = blockIdx.y * 16 + e / c4n, c = (e % c4n) * 4;
        const long row = r0 + r;
        if (!pad_rows && row >= m) continue;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < m && c < cols) x = __ldg(reinterpret_cast<const float4*>(src + row * lda + c));
        if (row_inv && row < m)
            atomicMax(&s_max[r - blockIdx.y * 16],
                      __float_as_uint(fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w)))));
        __nv_bfloat16* o = out + ((long)t * 128 + r) * ldo + c;
        for (int p = 0; p < pieces; ++p) {
            const __nv_bfloat162 a = __floats2bfloat162_rn(x.x, x.y), b = __floats2bfloat162_rn(x.z, x.w);
            uint2 pk;
            pk.x = *reinterpret_cast<const uint32_t*>(&a);
            pk.y = *reinterpret_cast<const uint32_t*>(&b);
            *reinterpret_cast<uint2*>(o + p * piece_stride) = pk;
            x.x -= __low2float(a);
            x.y -= __high2float(a);
            x.z -= __low2float(b);
            x.w -= __high2float(b);
        }
    }
    if (row_inv) {
        // |q~_i| <= ||q|| <= sqrt(cols) max |x| < 2^(e + 1 + norm_shift) with
        // max |x| in [2^e, 2^(e+1)): the row's power of two 2^(14 - e - norm_shift)
        __syncthreads();
        const long row = r0 + blockIdx.y * 16 + threadIdx.x;
        if (threadIdx.x < 16 && row < m) {
            const unsigned mb = s_max[threadIdx.x];
            int e = mb ? (int)((mb >> 23) & 0xFF) - 127 + norm_shift : 0;
            e = max(-112, min(127, e));  // the power of two and its inverse both normal
            row_inv[out0 + blockIdx.y * 16 + threadIdx.x] = __int_as_float((127 + e - 14) << 23);
        }
    }
}

// One warp per row r < m_rows: with e = floor(log2 max_c |A[r][c]|) read from
// the FP32 exponent field (clamped to [-112, 127]; a zero row takes e = 0),
// sigma = 2^(14 - e) puts the row's largest entry in [2^14, 2^15), inside
// FP16's normal range.  out[0][r][c] = fp16(sigma x), out[1][r][c] =
// fp16(sigma x - out[0][r][c]) (round to nearest), zero for c in
// [cols, ldo); inv[r] = 2^(e - 14).
constexpr int kF16SplitCols = 16;  // columns per lane: ldo <= 512
__global__ void split_rows_f16_scaled_kernel(const float* __restrict__ A, int m_rows, int lda, int cols, int ldo,
                                             __half* __restrict__ out, long piece_stride, float* __restrict__ inv) {
    const int lane = threadIdx.x & 31;
    const long warps = (long)gridDim.x * (blockDim.x >> 5);
    for (long row = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < m_rows; row += warps) {
        float v[kF16SplitCols];
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < kF16SplitCols; ++k) {
            const int c = lane + 32 * k;
            v[k] = c < cols ? __ldg(A + row * lda + c) : 0.f;
            m = fmaxf(m, fabsf(v[k]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        int e = m > 0.f ? ((__float_as_int(m) >> 23) & 0xFF) - 127 : 0;
        e = max(-112, min(127, e));  // sigma and 1 / sigma both normal powers of two
        const float sigma = __int_as_float((127 + 14 - e) << 23);
#pragma unroll
        for (int k = 0; k < kF16SplitCols; ++k) {
            const int c = lane + 32 * k;
            if (c < ldo) {
                const float x = v[k] * sigma;
                const __half h = __float2half_rn(x);
                out[row * ldo + c] = h;
                out[piece_stride + row * ldo + c] = __float2half_rn(x - __half2float(h));
            }
        }
        if (lane == 0) inv[row] = __int_as_float((127 + e - 14) << 23);
    }
}

__global__ void zero_kernel(float4* __restrict__ x, long n4) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n4; e += (long)gridDim.x * blockDim.x)
        x[e] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void scale_kernel(float* __restrict__ x, long n, float beta) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) x[e] *= beta;
}

}  // namespace

cudaError_t launch_scale(float* x, long count, float beta, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    int blocks = (int)((count + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    scale_kernel<<<blocks, 256, 0, stream>>>(x, count, beta);
    return cudaGetLastError();
}

cudaError_t launch_pairs_gemm_fp32(const float* A, int lda, const float* W, int N, int K, float* D, int ldd,
                                   const Tile* tiles, int n_tiles, const int* src, const int* dst, int nrhs,
                                   const ScaleTable& scales, cudaStream_t stream) {
    if (n_tiles <= 0 || N <= 0) return cudaSuccess;
    dim3 grid(n_tiles, (N + BN - 1) / BN);
    pairs_gemm_kernel<<<grid, NT, 0, stream>>>(A, lda, W, N, K, D, ldd, tiles, src, dst, nrhs, scales);
    return cudaGetLastError();
}

cudaError_t launch_pairs_gemm_fp32(const float* A, int lda, const float* W, int N, int K, float* D, int ldd,
                                   const Tile* tiles, int n_tiles, const int* src, const int* dst, int nrhs,
                                   float alpha, cudaStream_t stream) {
    ScaleTable sc{};
    sc.s[0] = alpha;
    return launch_pairs_gemm_fp32(A, lda, W, N, K, D, ldd, tiles, n_tiles, src, dst, nrhs, sc, stream);
}

cudaError_t launch_split_bf16(const float* x, int rows, int cols, int ld, __nv_bfloat16* out, long piece_stride,
                              int pieces, cudaStream_t stream) {
    const long total = (long)rows * cols;
    if (total <= 0) return cudaSuccess;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    split_bf16_kernel<<<blocks, 256, 0, stream>>>(x, rows, cols, ld, out, piece_stride, pieces);
    return cudaGetLastError();
}

cudaError_t launch_split_rows(const float* A, int m_rows, int lda, int cols, int ldo, const RowSeg* segs, int n_segs,
                              int n_tiles, __nv_bfloat16* out, long piece_stride, int pieces, cudaStream_t stream,
                              int pad_rows, float* row_inv) {
    if (n_tiles <= 0) return cudaSuccess;
    if ((lda & 3) || (cols & 3) || (ldo & 3) || cols > ldo || pieces < 1 || pieces > 3) return cudaErrorInvalidValue;
    int shift = 0;  // ceil(log2 sqrt(cols))
    while ((1L << (2 * shift)) < (long)cols) ++shift;
    split_rows_kernel<<<dim3((unsigned)n_tiles, 8), 256, 0, stream>>>(A, m_rows, lda, cols, ldo, segs, n_segs, out,
                                                                      piece_stride, pieces, pad_rows, row_inv, shift);
    return cudaGetLastError();
}

cudaError_t launch_split_rows_f16_scaled(const float* A, int m_rows, int lda, int cols, int ldo, __half* out,
                                         long piece_stride, float* inv, cudaStream_t stream) {
    if (m_rows <= 0) return cudaSuccess;
    if (cols > ldo || ldo > 32 * kF16SplitCols) return cudaErrorInvalidValue;
    long blocks = ((long)m_rows + 7) / 8;  // 8 warps per block, one row per warp
    if (blocks > 152 * 16) blocks = 152 * 16;
    split_rows_f16_scaled_kernel<<<(unsigned)blocks, 256, 0, stream>>>(A, m_rows, lda, cols, ldo, out, piece_stride,
                                                                      inv);
    return cudaGetLastError();
}

// dst[r][c] = src[r][c] + beta * dst[r][c] for c < cols (beta == 0: no read
// of dst), rows of ldd and lds floats.
__global__ void copy_rows_kernel(float* __restrict__ dst, int ldd, const float* __restrict__ src, int lds, long rows,
                                 int cols, float beta) {
    const long total = rows * cols;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long r = e / cols;
        const int c = (int)(e % cols);
        const float v = src[r * lds + c];
        dst[r * ldd + c] = beta == 0.f ? v : fmaf(beta, dst[r * ldd + c], v);
    }
}

cudaError_t launch_copy_rows(float* dst, int ldd, const float* src, int lds, long rows, int cols, float beta,
                             cudaStream_t stream) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    long blocks = (rows * cols + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    copy_rows_kernel<<<(int)blocks, 256, 0, stream>>>(dst, ldd, src, lds, rows, cols, beta);
    return cudaGetLastError();
}

cudaError_t launch_zero(float* x, long count, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    if ((count & 3) != 0 || (reinterpret_cast<uintptr_t>(x) & 15) != 0)
        return cudaMemsetAsync(x, 0, count * sizeof(float), stream);
    long n4 = count / 4;
    int blocks = (int)((n4 + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    zero_kernel<<<blocks, 256, 0, stream>>>(reinterpret_cast<float4*>(x), n4);
    return cudaGetLastError();
}

}  // namespace kifmm
