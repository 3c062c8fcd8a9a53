// Kernel launch wrappers (device code in kernels_simt.cu, kernels_umma.cu,
// kernels_core.cu, kernels_fmm.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstddef>
#include <cstdint>

namespace kifmm {

// One tile of an offset-grouped batch: rows [row0, row0 + nrows) of offset
// (k & 0xFFFF)'s virtual row list; k >> 16 selects a level scale of the
// tensor-core core (0 for single-level batches).  Virtual row v maps to pair = pair_begin + v / nrhs,
// rhs = v % nrhs; the source row is src[pair] * nrhs + rhs and the output
// row dst[pair] * nrhs + rhs.
struct Tile {
    int k;
    int pair_begin;
    int row0;
    int nrows;
};

// Factor applied to a tile's output, selected by tile.k >> 16.
struct ScaleTable {
    float s[32];
};

// Offset-grouped gather-GEMM-scatter, FP32 CUDA cores:
// for every tile, D[dst row] += alpha * A[src row] W_k^T with W_k = W + k * N * K
// (k = tile.k & 0xFFFF; alpha = scales.s[tile.k >> 16], or the scalar).
cudaError_t launch_pairs_gemm_fp32(const float* A, int lda, const float* W, int N, int K, float* D, int ldd,
                                   const Tile* tiles, int n_tiles, const int* src, const int* dst, int nrhs,
                                   const ScaleTable& scales, cudaStream_t stream);
cudaError_t launch_pairs_gemm_fp32(const float* A, int lda, const float* W, int N, int K, float* D, int ldd,
                                   const Tile* tiles, int n_tiles, const int* src, const int* dst, int nrhs,
                                   float alpha, cudaStream_t stream);

// x (FP32 [rows][cols], ld) -> `pieces` BF16 arrays [rows][cols] (piece stride
// `piece_stride` elements) with x ~= sum of pieces (round-to-nearest each).
cudaError_t launch_split_bf16(const float* x, int rows, int cols, int ld, __nv_bfloat16* out, long piece_stride,
                              int pieces, cudaStream_t stream);

// Point-source evaluation (kernels_fmm.cu).  Points in leaf order, leaf b
// holding [leaf_start[b], leaf_start[b+1]), in leaf units s = (x - c_b) / h
// split as hi (a multiple of 2^-20, w = density) + lo; usurf: the n points
// of the [-1,1]^3 cube surface.
// hi[i].w = q[perm[i]].
cudaError_t launch_gather_density(const float* q, const int* perm, float4* hi, int n_points, cudaStream_t stream);
// rows[j][a] = scale * sum_i Ws[a][i] g(x_i, s_j) in FP64, stored as FP32
// ([n_points][rp]; Ws [rp][n] with zero rows past the rank; x_i the n
// check points in leaf units [n][3]; pts the points in leaf units
// [n_points][3]): g = 1 / |x_i - s_j|, or with normals nrm [n_points][3]
// g = n_j . (x_i - s_j) / |x_i - s_j|^3.  rp <= 288, a multiple of 16.
cudaError_t launch_point_rows(const double* pts, const double* nrm, int n_points, const double* ws, int rp, int n,
                              const double* xsurf, double scale, float* rows, cudaStream_t stream);
// qf[b][a] = sum_{j in leaf b} hi[j].w rows[j][a] (compensated FP32 sum) and
// its three BF16 pieces qb[pc][b][a] (piece stride pstride elements).
cudaError_t launch_leaf_rows_sum(const float* rows, const float4* hi, const int* leaf_start, int n_leaves, int rp,
                                 float* qf, __nv_bfloat16* qb, long pstride, cudaStream_t stream);
// out[perm[i]] = trows[i] . pleaf[b] (parts & 2) + near field over
// near_idx[near_start[b]..near_start[b+1]) (parts & 1): scale * sum q_j /
// |d|, or, with the normals' two words nhi + nlo (double layer), scale_dl *
// sum q_j n_j . d / |d|^3.
cudaError_t launch_leaf_eval(const float4* hi, const float4* lo, const float4* nhi, const float4* nlo,
                             const int* leaf_start, const int4* leaf_ijk, const int* near_start, const int* near_idx,
                             int n_leaves, const float* trows, int rp, const float* pleaf, float scale, float scale_dl,
                             const int* perm, float* out, int parts, cudaStream_t stream);

// Rows of A (FP32, m_rows x cols, ld lda) -> two FP16 pieces [2][m_rows][ldo]
// (piece stride piece_stride) of sigma_r x with sigma_r the power of two that
// puts row r's largest |x| in [2^14, 2^15), and inv[r] = 1 / sigma_r.  ldo <= 512.
cudaError_t launch_split_rows_f16_scaled(const float* A, int m_rows, int lda, int cols, int ldo, __half* out,
                                         long piece_stride, float* inv, cudaStream_t stream);

// dst[r][c] = src[r][c] + beta dst[r][c] for r < rows, c < cols.
cudaError_t launch_copy_rows(float* dst, int ldd, const float* src, int lds, long rows, int cols, float beta,
                             cudaStream_t stream);

// Zero `count` floats.
cudaError_t launch_zero(float* x, long count, cudaStream_t stream);

// x *= beta over `count` floats.
cudaError_t launch_scale(float* x, long count, float beta, cudaStream_t stream);

// tcgen05 (UMMA) split-BF16 GEMM with fused gather / scatter, one kernel
// template for the three products of the compressed M2L:
//   core      D[dst row] += A_pieces[src row] K~_o^T          (A_GATHER, E_RED)
//   compress  Dp = pieces(alpha A W^T), Z = 0                 (E_SPLIT)
//   expand    D = alpha A W^T + beta D                        (E_STORE)
// Compress and expand take A either as BF16 pieces pre-split by
// launch_split_rows (A_GATHER with row_identity, drained partials) or as FP32
// rows split inside the kernel (A_ROWS).
// B operands are BF16 pieces [pieces][b_groups][ndim][kdim] read by TMA.
enum UmmaAMode { A_GATHER = 0, A_ROWS = 1 };

// Rows modes over many buffers (batches of many instances): the virtual row
// tiles [tile_begin, tile_begin + ceil(m_rows / 128)) of a launch read rows
// 0..m_rows-1 of Af and write rows of D (E_STORE, with alpha and beta) or
// rows out_row + r of Dp / Df / Z (E_SPLIT).
struct RowSeg {
    const float* Af;
    float* D;
    int m_rows;
    int tile_begin;
    int out_row;
    float alpha, beta;
};
enum UmmaEMode { E_RED = 0, E_STORE = 1, E_SPLIT = 2 };

// FP32 rows -> BF16 pieces [pieces][n_tiles * 128][ldo] (see split_rows_kernel):
// virtual tile t takes rows of the single input A (n_segs = 0: rows
// [128 t, 128 t + 128) of m_rows) or of the segment that owns tile t.
// Output rows past the input's rows are zeroed, or left alone when
// pad_rows == 0.
// With row_inv set, a bound on each input row's 2-norm also gives its power
// of two for an FP16 split after a product with orthonormal columns:
// ||x|| <= sqrt(cols) max |x| < 2^(e + 1) with e the exponent of max |x| plus
// ceil(log2 sqrt(cols)); row_inv[out row] = 2^(e - 14) (e clamped to
// [-112, 127]), the out row being the segment's out_row + its row (or the row).
cudaError_t launch_split_rows(const float* A, int m_rows, int lda, int cols, int ldo, const RowSeg* segs, int n_segs,
                              int n_tiles, __nv_bfloat16* out, long piece_stride, int pieces, cudaStream_t stream,
                              int pad_rows = 1, float* row_inv = nullptr);

struct UmmaArgs {
    // A operand
    const __nv_bfloat16* A;   // A_GATHER: piece 0 base, [rows][kdim]; piece i at A + i * a_piece_stride
    long a_piece_stride;      // elements
    const float* Af;          // A_ROWS: FP32 rows [m_rows][lda]
    int lda;
    int k_valid;              // A_ROWS: valid columns of Af (multiple of 4); beyond: zero
    int m_rows;               // A_ROWS: number of rows
    int kdim;                 // padded K (multiple of 16)
    // B operand (TMA)
    const __nv_bfloat16* B;   // piece 0 base
    int b_groups;             // 316 offsets (core) or 1
    int ndim;                 // N rows per group (multiple of 16)
    int n_chunk;              // N per work item (multiple of 16)
    // work list (A_GATHER): per tile t, 128 A rows row_src[128 t + i] and
    // output rows row_dst[128 t + i] (-1: none), and tile_k[t] = offset |
    // (level index << 16)
    const int* row_src;
    const int* row_dst;
    const int* tile_k;
    int n_tiles;
    int nrhs;
    int zero_row;             // row of the A pieces that is all zero
    float level_scale[32];    // E_RED: factor applied to a tile's output, by tile.k >> 16
    const float* scale_table; // E_RED: when set, replaces level_scale (index tile.k >> 16)
    const RowSeg* segs;       // rows modes: when n_segs > 0, the row segments (device)
    int n_segs;
    int seg_tiles;            // rows modes with segments: total virtual row tiles
    int contiguous;           // core: 1 = each CTA takes a contiguous run of tiles
    int row_identity;         // A_GATHER with E_SPLIT / E_STORE: tile t's A rows are 128 t + i (pre-split pieces),
                              // outputs follow the rows-mode conventions (m_rows or segments)
    int core_resident;        // core, split6 with hilo: 1 = A tile resident in shared memory, K~_o in N blocks
    int core_drain;           // core, split6: K-chunks per partial drained into registers by 8 epilogue warps (0: off)
    int core_bres;            // core, 1 or 2 pieces: the staged-epilogue kernel of kernels_core.cu
    // core, stage 2 (Sec. 3.2): K~_o = Uhat_o Vhat_o with per-offset rank k_o
    int s2_on;
    const __nv_bfloat16* s2_V;  // pieces [pieces][316][96][kdim]: rows of Vhat_o, zero past k_o
    const __nv_bfloat16* s2_U;  // pieces [pieces][316][ndim][96]: rows of Uhat_o, zero past k_o
    const int* s2_k16;          // [316] k_o rounded up to 16 (16..96)
    // epilogue
    float* D;                 // E_RED / E_STORE: FP32 [*][ldd]
    int ldd;
    float alpha, beta;
    int n_valid;              // E_STORE: columns < n_valid are written
    __nv_bfloat16* Dp;        // E_SPLIT: pieces [piece][m_rows][ldd]
    int dp_f16;               // E_SPLIT: Dp holds 2 FP16 pieces of each output row times 1 / dp_row_inv[row]
    const float* dp_row_inv;  // E_SPLIT with dp_f16: per output row, the inverse of its power of two
    long dp_piece_stride;
    int dp_pieces;
    float* Df;                // E_SPLIT: optional FP32 copy [m_rows][ldd]
    float* Z;                 // E_SPLIT: optional buffer [m_rows][ldd] to zero
    // arithmetic
    int n_products;           // 1, 3 or 6 piece products
    int hilo;                 // 1: the (0,0) product accumulates apart from the others
    int f16;                  // A_GATHER: A and B pieces are FP16 (else BF16)
    const float* row_scale;   // E_RED: when set, output row r is scaled by row_scale[row_src[r]]
    int red_bulk;             // E_RED, drained partials: reduce rows into D with TMA bulk reductions
    int mma_pair;             // drained partials: K-chunks of a partial the MMA thread takes per step (<= 1: one)
    int direct_rows;          // E_RED, drained partials: every lane reduces its own row into D (no transpose)
    int* error_flag;          // device int, set when a bounded wait times out
    unsigned long long wait_ns;  // bound of every mbarrier wait in ns (0: the default, 2 s)
};
cudaError_t launch_umma(int amode, int emode, const UmmaArgs& args, int num_sms, cudaStream_t stream);

// The core whose epilogue stages rows in shared memory and reduces them into
// p~ by TMA bulk reductions (kernels_core.cu): 1 or 2 pieces (n_products 1
// or 3); cudaErrorNotSupported when the operands do not fit.
cudaError_t launch_core_stage(const UmmaArgs& args, int num_sms, int max_smem, int dev, cudaStream_t stream);
// The same kernel over up to 8 operators at once (one launch for a batch of
// plans): group i takes its operands, tile list, scale table (required when
// n_groups > 1) and p~ from args[i]; every group has the same piece count
// and FP16 flag, and the launch's error flag and wait bound are args[0]'s.
cudaError_t launch_core_stage_grouped(const UmmaArgs* args, int n_groups, int num_sms, int max_smem, int dev,
                                      cudaStream_t stream);
// Its shared-memory need (0: does not fit max_smem), ring stages in *stages.
size_t core_stage_smem(int pieces, int kdim, int ndim, int max_smem, int* stages);

// A 2-byte-element matrix [rows][cols] as a 2D TMA tensor map with boxes of
// ch (32: 64-byte swizzle, 16: 32-byte swizzle) x box_rows; maps are cached.
cudaError_t tma_map_2d(const void* ptr, uint64_t rows, int cols, int ch, int box_rows, CUtensorMap* out);

}  // namespace kifmm
