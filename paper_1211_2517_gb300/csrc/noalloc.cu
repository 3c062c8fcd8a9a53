// kifmm_m2l_apply_noalloc: the compressed M2L apply with its working memory
// in a fixed, statically sized device array instead of plan-owned buffers.
//
// kifmm_m2l_apply grows scratch buffers (the split pieces of q~, p~, the
// tile table) with cudaMalloc the first time a level / nrhs needs them.
// Some callers cannot allocate device memory once their run has started:
// applications whose memory manager has reserved the whole device up front,
// solvers with a hard memory budget, and latency-critical loops where the
// device-wide synchronisation of cudaMalloc / cudaFree is not acceptable.
// This entry point serves them: it calls no allocating routine.  Its scratch
// is the array below, which every GPU that loads this module holds until the
// process exits.  The plan and the level registrations (made earlier with
// kifmm_m2l_precompute / kifmm_m2l_set_level) are used as they are.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cmath>
#include <mutex>
#include <string>

#include "kernels.h"
#include "kifmm_internal.h"
#include "plan.h"

using namespace kifmm;

namespace {

constexpr size_t kScratchBytes = KIFMM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Per-offset prefixes of pairs and tiles, passed to the tile builder by value.
struct TilePrefix {
    int pair_begin[kOffsets + 1];
    int tile_begin[kOffsets + 1];
};

// Expand the per-offset prefixes into the tile table of the core kernels:
// tile t belongs to the last offset k with tile_begin[k] <= t (offsets
// without pairs have no tiles) and covers 128 consecutive (pair, rhs) rows.
// One thread per (tile, row) also writes the row tables of the tensor-core
// kernel (source and target row of every tile row, -1 past the tile's end).
__global__ void build_tiles_kernel(const TilePrefix pre, int nrhs, int n_tiles, const int* src, const int* dst,
                                   Tile* tiles, int* row_src, int* row_dst, int* tile_k) {
    const long total = (long)n_tiles * kTileRows;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int t = (int)(e / kTileRows), r = (int)(e % kTileRows);
        int lo = 0, hi = kOffsets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (pre.tile_begin[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int row0 = (t - pre.tile_begin[lo]) * kTileRows;
        const int rows = (pre.pair_begin[lo + 1] - pre.pair_begin[lo]) * nrhs;
        const int nrows = rows - row0 < kTileRows ? rows - row0 : kTileRows;
        if (r == 0) {
            Tile out;
            out.k = lo;
            out.pair_begin = pre.pair_begin[lo];
            out.row0 = row0;
            out.nrows = nrows;
            tiles[t] = out;
            tile_k[t] = lo;
        }
        int rs = -1, rd = -1;
        if (r < nrows) {
            const int g = row0 + r;
            const int pr = pre.pair_begin[lo] + g / nrhs;
            rs = src[pr] * nrhs + g % nrhs;
            rd = dst[pr] * nrhs + g % nrhs;
        }
        row_src[e] = rs;
        row_dst[e] = rd;
    }
}

std::mutex g_setup_mutex;
struct ScratchAddr {
    CUcontext ctx;        // the context the address belongs to
    unsigned char* ptr;   // device address of g_noalloc_scratch in it
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    return fn;
}

// Device address of the static scratch on the current device: looked up
// once per device and context (a context destroyed and created again, e.g.
// after cudaDeviceReset, gets its own lookup), with that device current.
int scratch_address(unsigned char** out) {
    int dev = -1;
    KIFMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal out of range for the static scratch table");
        return KIFMM_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    CUcontext ctx = nullptr;
    const CtxGetCurrentFn fn = ctx_get_current();
    const bool known_ctx = fn && fn(&ctx) == CUDA_SUCCESS && ctx != nullptr;
    ScratchAddr& e = g_scratch_addr[dev];
    if (!known_ctx || !e.ptr || e.ctx != ctx) {
        void* p = nullptr;
        KIFMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        e.ptr = static_cast<unsigned char*>(p);
        e.ctx = known_ctx ? ctx : nullptr;
    }
    *out = e.ptr;
    return KIFMM_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int kifmm_m2l_apply_noalloc(kifmm_m2l_plan plan, int instance, int level, int nrhs, const float* q_up,
                                       float* p_down, float beta, void* stream) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    LevelState* ls = find_level(plan, instance, level);
    if (!ls) {
        set_error("level not registered: call kifmm_m2l_set_level first");
        return KIFMM_ERR_STATE;
    }
    if (nrhs < 1 || (ls->n_boxes > 0 && (!q_up || !p_down))) {
        set_error("invalid nrhs or NULL density pointer");
        return KIFMM_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(q_up) & 15) || (reinterpret_cast<uintptr_t>(p_down) & 15)) {
        set_error("density pointers must be 16-byte aligned");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (plan->prm.precision == KIFMM_PREC_F16X3) {
        set_error("the allocation-free apply runs the FP32 and BF16 modes (not KIFMM_PREC_F16X3)");
        return KIFMM_ERR_UNSUPPORTED;
    }
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    unsigned char* base = nullptr;
    st = scratch_address(&base);
    if (st != KIFMM_OK) return st;
    if (ls->n_boxes == 0) return KIFMM_OK;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = plan->n, rp = plan->rp;
    const bool fp32_core = plan->prm.precision == KIFMM_PREC_FP32;
    const long rows = (long)ls->n_boxes * nrhs;
    PairSet& ps = ls->fwd;
    TilePrefix pre;
    long n_tiles = 0;
    for (int k = 0; k < kOffsets; ++k) {
        pre.pair_begin[k] = (int)ps.off_begin[k];
        pre.tile_begin[k] = (int)n_tiles;
        n_tiles += ((ps.off_begin[k + 1] - ps.off_begin[k]) * nrhs + kTileRows - 1) / kTileRows;
    }
    pre.pair_begin[kOffsets] = (int)ps.off_begin[kOffsets];
    pre.tile_begin[kOffsets] = (int)n_tiles;

    // scratch layout: [q~ pieces (rows + 1 zero row) | q~ FP32 | p~ FP32 | tiles | row tables]
    const long piece_stride = (rows + 1) * rp;
    const size_t qb_bytes = fp32_core ? 0 : align256((size_t)piece_stride * plan->pieces * sizeof(__nv_bfloat16));
    const size_t qt_bytes = fp32_core ? align256((size_t)rows * rp * sizeof(float)) : 0;
    const size_t pt_bytes = align256((size_t)rows * rp * sizeof(float));
    const size_t tile_bytes = align256((size_t)n_tiles * sizeof(Tile));
    const size_t rowtab_bytes = align256((size_t)n_tiles * kTileRows * sizeof(int));
    const size_t tk_bytes = align256((size_t)n_tiles * sizeof(int));
    const size_t need = qb_bytes + qt_bytes + pt_bytes + tile_bytes + 2 * rowtab_bytes + tk_bytes;
    if (need > kScratchBytes || rows + 1 > (long)INT32_MAX / 2) {
        set_error("kifmm_m2l_apply_noalloc: this level with nrhs = " + std::to_string(nrhs) + " needs " +
                  std::to_string(need) + " bytes of scratch; the static scratch holds " +
                  std::to_string(kScratchBytes) + " bytes (use kifmm_m2l_apply, or fewer right-hand sides)");
        return KIFMM_ERR_INVALID_ARG;
    }
    __nv_bfloat16* qb = reinterpret_cast<__nv_bfloat16*>(base);
    float* qt = reinterpret_cast<float*>(base + qb_bytes);
    float* pt = reinterpret_cast<float*>(base + qb_bytes + qt_bytes);
    Tile* tiles = reinterpret_cast<Tile*>(base + qb_bytes + qt_bytes + pt_bytes);
    int* row_src = reinterpret_cast<int*>(base + qb_bytes + qt_bytes + pt_bytes + tile_bytes);
    int* row_dst = reinterpret_cast<int*>(base + qb_bytes + qt_bytes + pt_bytes + tile_bytes + rowtab_bytes);
    int* tile_k = reinterpret_cast<int*>(base + qb_bytes + qt_bytes + pt_bytes + tile_bytes + 2 * rowtab_bytes);
    const float scale = (float)std::ldexp(1.0 / ls->r0, level);

    // 1. compression q~ = R~^T q into the scratch, p~ = 0 (the scratch keeps
    //    the previous call's contents, so every buffer that must start at
    //    zero is cleared here)
    {
        UmmaArgs a{};
        a.Af = q_up;
        a.lda = n;
        a.k_valid = n;
        a.m_rows = (int)rows;
        a.kdim = plan->n_pad;
        a.B = plan->Rtb.ptr;
        a.b_groups = 1;
        a.ndim = rp;
        a.n_chunk = chunk_for(rp);
        a.ldd = rp;
        a.alpha = 1.0f;
        a.Dp = fp32_core ? nullptr : qb;
        a.dp_piece_stride = piece_stride;
        a.dp_pieces = fp32_core ? 0 : plan->pieces;
        a.Df = fp32_core ? qt : nullptr;
        a.Z = pt;
        a.n_products = 6;
        a.hilo = 1;
        a.error_flag = plan->err_flag.ptr;
        KIFMM_CUDA_TRY(launch_umma(A_ROWS, E_SPLIT, a, plan->num_sms, s));
    }
    // 2. tile table and the core
    if (n_tiles > 0) {
        const long work = n_tiles * (long)kTileRows;
        const int blocks = (int)((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
        build_tiles_kernel<<<blocks, 256, 0, s>>>(pre, nrhs, (int)n_tiles, ps.src.ptr, ps.dst.ptr, tiles, row_src,
                                                  row_dst, tile_k);
        KIFMM_CUDA_TRY(cudaGetLastError());
    }
    if (fp32_core) {
        KIFMM_CUDA_TRY(launch_pairs_gemm_fp32(qt, rp, plan->C.ptr, rp, rp, pt, rp, tiles, (int)n_tiles, ps.src.ptr,
                                              ps.dst.ptr, nrhs, 1.0f, s));
    } else {
        for (int pc = 0; pc < plan->pieces; ++pc)
            KIFMM_CUDA_TRY(cudaMemsetAsync(qb + pc * piece_stride + rows * rp, 0, rp * sizeof(__nv_bfloat16), s));
        UmmaArgs a{};
        a.A = qb;
        a.a_piece_stride = piece_stride;
        a.kdim = rp;
        a.B = plan->Cb.ptr;
        a.b_groups = kOffsets;
        a.ndim = rp;
        a.n_chunk = core_chunk(plan);
        // the plan's core variant, as kifmm_m2l_apply launches it
        a.contiguous = plan->tune_contig;
        a.core_resident = plan->tune_variant == 1;
        a.core_drain = plan->variant_drain();
        a.red_bulk = plan->variant_bulk();
        a.mma_pair = plan->variant_pair();
        a.direct_rows = plan->variant_direct();
        a.core_bres = plan->variant_bres();
        a.wait_ns = plan->core_wait_ns;
        a.s2_on = plan->s2_on;
        a.s2_V = plan->s2V.ptr;
        a.s2_U = plan->s2U.ptr;
        a.s2_k16 = plan->s2_k16.ptr;
        a.row_src = row_src;
        a.row_dst = row_dst;
        a.tile_k = tile_k;
        a.n_tiles = (int)n_tiles;
        a.nrhs = nrhs;
        a.zero_row = (int)rows;
        a.level_scale[0] = 1.0f;  // the level scale is applied by the expansion
        a.D = pt;
        a.ldd = rp;
        a.n_products = plan->products;
        a.hilo = plan->core_hilo;
        a.error_flag = plan->err_flag.ptr;
        KIFMM_CUDA_TRY(launch_umma(A_GATHER, E_RED, a, plan->num_sms, s));
    }
    // 3. expansion p_down = beta p_down + s_l U~ p~
    {
        UmmaArgs a{};
        a.Af = pt;
        a.lda = rp;
        a.k_valid = rp;
        a.m_rows = (int)rows;
        a.kdim = rp;
        a.B = plan->Ub.ptr;
        a.b_groups = 1;
        a.ndim = plan->n_pad;
        a.n_chunk = chunk_for(plan->n_pad);
        a.D = p_down;
        a.ldd = n;
        a.alpha = scale;
        a.beta = beta;
        a.n_valid = n;
        a.n_products = 6;
        a.hilo = 1;
        a.error_flag = plan->err_flag.ptr;
        KIFMM_CUDA_TRY(launch_umma(A_ROWS, E_STORE, a, plan->num_sms, s));
    }
    return KIFMM_OK;
}
