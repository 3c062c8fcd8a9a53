// Internal plan object of the C ABI (include/kifmm_m2l.h), shared by the
// translation units that implement its entry points.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.h"
#include "kifmm_internal.h"

namespace kifmm {

constexpr int kTileRows = 128;
// Instances from 2^30 up hold the levels of point-source evaluations.
constexpr int kReservedInstance = 1 << 30;

#define KIFMM_CUDA_TRY(expr)                                                                        \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess) {                                                                    \
            set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                          \
            return _e == cudaErrorMemoryAllocation ? KIFMM_ERR_OOM : KIFMM_ERR_CUDA;               \
        }                                                                                           \
    } while (0)

template <class T>
struct DevBuf {
    T* ptr = nullptr;
    size_t count = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        count = 0;
    }
    cudaError_t ensure(size_t n) {
        if (n <= count && ptr) return cudaSuccess;
        release();
        if (n == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&ptr, n * sizeof(T));
        if (e == cudaSuccess) count = n;
        else ptr = nullptr;
        return e;
    }
    cudaError_t upload(const T* h, size_t n) {
        cudaError_t e = ensure(n);
        if (e != cudaSuccess || n == 0) return e;
        return cudaMemcpy(ptr, h, n * sizeof(T), cudaMemcpyHostToDevice);
    }
};

// Tiles of 128 (pair, rhs) rows for one nrhs: the tile list (CUDA-core
// kernel) and the per-row index tables of the tensor-core kernel.
struct TileSet {
    DevBuf<Tile> tiles;
    DevBuf<int> row_src, row_dst, tile_k;
    int n_tiles = 0;
};

struct PairSet {
    DevBuf<int> src, dst;
    std::vector<int32_t> h_src, h_dst;  // host copies (row tables, multi-level batches)
    std::vector<int64_t> off_begin;  // [317] prefix by offset
    std::map<int, std::unique_ptr<TileSet>> tilesets;  // per nrhs
};

// Pairs of several consecutive levels of one instance, merged for a
// multi-level batch: box indices are offset so that the levels' density
// arrays sit back to back; groups are ordered by offset, then level.
struct MultiState {
    DevBuf<int> src, dst;
    struct Group {
        int k, level_idx;
        int64_t begin, count;
    };
    std::vector<Group> groups;
    std::vector<int32_t> h_src, h_dst;
    int64_t total_boxes = 0;
    std::map<int, std::unique_ptr<TileSet>> tilesets;  // per nrhs
};

// Upload a tile list and build its row tables from host pair arrays.
int make_tileset(const std::vector<Tile>& tiles, const std::vector<int32_t>& src, const std::vector<int32_t>& dst,
                 int nrhs, TileSet& out);

struct LevelState {
    int level = 0, n_boxes = 0;
    double r0 = 1.0;
    int64_t n_pairs = 0;
    PairSet fwd, adj;
};

}  // namespace kifmm

struct kifmm_m2l_plan_s {
    kifmm_m2l_params prm{};
    int device = 0, num_sms = 0;
    int n = 0, r = 0, rp = 0;
    int pieces = 0;   // BF16 pieces of the tensor-core modes
    int products = 0;
    double sym_err = 0;
    std::vector<double> sigma;
    int n_pad = 0;    // n rounded up to 16 (K of the compression, N of the expansion)
    int core_hilo = 0;
    // core launch choices picked by kifmm_m2l_autotune (0: defaults)
    int tune_chunk = 0;
    int tune_contig = 0;
    // core variant (split6, f16x3): 0 classic, 1 A-resident (where it fits),
    // 2 / 3 partials of two / one K-chunks drained into registers, 4 / 5 the
    // same with TMA bulk reductions
    int tune_variant = 2;
    // core launch fields of a variant: 1 A-resident; 2 / 4 / 9 partials of
    // two K-chunks drained into registers, 3 / 5 of one, 6 / 10 of three
    // (f16x3); 4 / 5 reduce the rows into p~ with TMA bulk reductions
    // instead of vector atomics; 9 / 10 issue two K-chunks per MMA step,
    // 11 (f16x3) a whole partial of three; 13 (1 or 2 pieces) the staged
    // epilogue whose rows reach p~ by TMA bulk reductions (kernels_core.cu)
    int variant_drain() const {
        switch (tune_variant) {
            case 2: case 4: return 2;
            case 3: case 5: return 1;
            case 6: case 10: case 11: case 12: case 13: return 3;
            case 9: return 2;
            default: return 0;
        }
    }
    int variant_pair() const {
        return (tune_variant == 11 || tune_variant == 12) ? 3 : (tune_variant == 9 || tune_variant == 10) ? 2 : 1;
    }
    int variant_direct() const { return tune_variant == 12 ? 1 : 0; }
    int variant_bres() const { return tune_variant == 13 ? 1 : 0; }
    int variant_bulk() const { return (tune_variant == 4 || tune_variant == 5) ? 1 : 0; }
    kifmm::DevBuf<float> C, K;
    // tensor-core dense baseline (f16x3 plans): K_o as two FP16 pieces of
    // tau_K K_o [2][316][n_pad][n_pad], 1 / tau_K, and its operand / output buffers
    kifmm::DevBuf<__nv_bfloat16> Kd, dq;
    kifmm::DevBuf<float> dq_inv, dp;
    float dense_inv_scale = 1.0f;
    kifmm::DevBuf<__nv_bfloat16> Cb, Rtb, Ub;  // 3 BF16 pieces each (Cb: 2 FP16 pieces of tau K~ for F16X3)
    float core_inv_scale = 1.0f;               // 1 / tau (F16X3), else 1
    std::vector<double> U64;                   // [n][r] FP64 basis U~ (= R~)
    // compressed pass operators of Sec. 3.3 (point-source evaluation), on first use:
    // Ws in FP64 [rp][n] (rows past the rank zero; the per-point S~ / T~ rows
    // are formed from it), M~ and L~ [8][rp][rp] as 3 BF16 pieces each
    double pass_rcond = 0;
    int pass_kept = 0;
    kifmm::DevBuf<double> Ws64;
    kifmm::DevBuf<__nv_bfloat16> Mb, Lb;
    int next_fmm_instance = 0;
    std::set<kifmm_fmm_s*> fmms;  // live point-source trees on this plan
    // stage 2 (Sec. 3.2): per-offset low-rank cores, off until kifmm_m2l_set_stage2
    int s2_on = 0;
    double s2_c2 = 0;
    std::vector<int> s2_k;                     // [316] ranks k_o
    kifmm::DevBuf<__nv_bfloat16> s2V, s2U;     // 3 BF16 pieces each (F16X3: 2 FP16 pieces of tau_V Vhat, tau_U Uhat, third zero)
    kifmm::DevBuf<int> s2_k16;                 // [316] k_o rounded up to 16
    float s2_inv_scale = 1.0f;                 // 1 / (tau_V tau_U) (F16X3), else 1
    // the factor the core's output rows take besides s_l: undoes the powers
    // of two of the FP16 operands (single stage: the cores'; stage 2: both factors')
    float out_inv_scale() const { return s2_on ? s2_inv_scale : core_inv_scale; }
    kifmm::DevBuf<int> err_flag;
    unsigned long long core_wait_ns = 0;  // bound of the core kernels' waits (0: 2 s)
    std::map<std::pair<int, int>, std::unique_ptr<kifmm::LevelState>> levels;
    // multi-level batches keyed by (instance, level_lo, level_hi, adjoint)
    std::map<std::tuple<int, int, int, int>, std::unique_ptr<kifmm::MultiState>> multi;
    // tracing: (stage, start, stop) event triples recorded by applies
    bool profile = false;
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
    int64_t traced_launches = 0;
    cudaEvent_t get_event() {
        if (!event_pool.empty()) {
            cudaEvent_t e = event_pool.back();
            event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // host-buffer applies: device copies of the densities, a copy stream and
    // events (timing off) that order the chunks' copies and kernels
    kifmm::DevBuf<float> hx, hy;
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> sync_events;
    ~kifmm_m2l_plan_s() {
        for (auto& r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : event_pool) cudaEventDestroy(e);
        for (auto e : sync_events) cudaEventDestroy(e);
        if (copy_stream) cudaStreamDestroy(copy_stream);
    }
    // scratch shared by all levels (apply calls on one plan are serialised)
    kifmm::DevBuf<float> qt, pt;
    kifmm::DevBuf<__nv_bfloat16> qb, sp;  // sp: BF16 pieces of the compression / expansion inputs
    kifmm::DevBuf<float> qs;                // F16X3: 1 / sigma of every q~ row
};


namespace kifmm {

// The registered level, or nullptr.
LevelState* find_level(kifmm_m2l_plan plan, int instance, int level);
// KIFMM_OK when the current device is the plan's device.
int check_device(kifmm_m2l_plan plan);
// N per work item of the compression / expansion GEMMs.
int chunk_for(int ndim);
// N per work item of the core GEMM (the autotuned choice, else the default).
int core_chunk(kifmm_m2l_plan plan);
int core_chunk_default(kifmm_m2l_plan plan);
// Merged pairs of levels lo..hi of one instance (built on first use).
int get_multi_state(kifmm_m2l_plan plan, int instance, int lo, int hi, bool adjoint, MultiState** out);
// Drop cached batches that use `plan` (on destroy).
void forget_batches_of(kifmm_m2l_plan plan);
// Unlink the point-source trees of `plan` (on destroy); their later calls
// fail with KIFMM_ERR_STATE and their destroy only frees them.
void detach_fmms(kifmm_m2l_plan plan);

// Compression (Step 3.1's q~ = R~^T q): the FP32 rows (one buffer of m_rows
// rows, or row segments over n_tiles virtual tiles) are split into BF16
// pieces in `split` (>= 3 * 128 * n_tiles * n_pad elements), then a
// tensor-core GEMM writes q~ as `pieces` BF16 pieces into qb (piece stride
// qb_stride; or FP32 into qt when qt != nullptr) and zeroes p~ rows of pt.
// With f16_inv set (f16x3 core), qb receives two FP16 pieces of every q~ row
// times the power of two of its input row's 2-norm, f16_inv[row] its
// inverse (qt must then be NULL).
int run_compress(kifmm_m2l_plan plan, const float* x, int m_rows, const RowSeg* segs, int n_segs, int n_tiles,
                 __nv_bfloat16* split, __nv_bfloat16* qb, long qb_stride, float* qt, float* pt, cudaStream_t s,
                 float* f16_inv = nullptr);
// Expansion (p = alpha U~ p~ + beta p): the FP32 p~ rows (pt, ld r_pad, or
// segments) are split into BF16 pieces in `split` (>= 3 * 128 * n_tiles *
// r_pad elements), then a tensor-core GEMM writes y (ld n) or, with
// segments, each segment's D with its own alpha and beta.
int run_expand(kifmm_m2l_plan plan, const float* pt, int m_rows, const RowSeg* segs, int n_segs, int n_tiles,
               __nv_bfloat16* split, float* y, float alpha, float beta, cudaStream_t s);
// Elements the split buffer of run_compress / run_expand needs.
size_t split_elems(kifmm_m2l_plan plan, long n_tiles);
// N per work item of the identity-row GEMMs over n_tiles row tiles.
int rows_chunk(int ndim, long n_tiles, int num_sms, int max_n);
// Tile set of a multi-level state for nrhs (built on first use).
int multi_tileset(MultiState& ms, int nrhs, TileSet** out);
// The tensor-core core over a tile set: pt[dst] += scale K~_o qb[src], with
// qb the plan's BF16 pieces (piece stride piece_stride, zero row zero_row);
// stage 2 and the autotuned variant as set on the plan.
int launch_core(kifmm_m2l_plan plan, const __nv_bfloat16* qb, long piece_stride, int zero_row, const TileSet& ts,
                int nrhs, const ScaleTable& scales, float* pt, cudaStream_t s, const float* row_scale = nullptr);
// F16X3 operand of the core: q~ (FP32 rows [rows][rp] in qt) -> two scaled
// FP16 pieces in qb (piece stride piece_stride, row `rows` zero) and the
// row factors 1 / sigma in qs[0..rows] (qs[rows] = 0).
// The zero row (index rows) of the f16x3 core operand and its factor.
int zero_core_operand_row_f16(kifmm_m2l_plan plan, long rows, __nv_bfloat16* qb, long piece_stride, float* qs,
                              cudaStream_t s);
int split_core_operand_f16(kifmm_m2l_plan plan, const float* qt, long rows, __nv_bfloat16* qb, long piece_stride,
                           float* qs, cudaStream_t s);
// Upload value_at(e), e < per, as 3 BF16 pieces [3][per] (piece j = RN of
// the remainder of the earlier pieces).
int upload_pieces(DevBuf<__nv_bfloat16>& dst, size_t per, const std::function<double(size_t)>& value_at);
// Interaction state of one level of one instance (kifmm_m2l_set_level
// without its argument checks).
int register_level(kifmm_m2l_plan plan, int instance, int level, double root_halfwidth, int n_boxes,
                   const int32_t* box_ijk);

}  // namespace kifmm
