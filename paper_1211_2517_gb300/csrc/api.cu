// C ABI of the SVD-compressed M2L (include/kifmm_m2l.h): plan object,
// per-level interaction state, scratch management and the apply paths.
//
// Data layout in device memory (n surface points, r rank, rp = r rounded
// up to 16, B boxes of a level, R = nrhs):
//   Rt   [rp][n]   FP32   R~^T, rows r..rp-1 zero            (V^T compression)
//   U    [n][rp]   FP32   U~, columns r..rp-1 zero           (U expansion)
//   C    [316][rp][rp] FP32  K~_o, zero-padded               (FP32 core)
//   Cb   [pieces][316][rp][rp] BF16 split of C              (tensor-core core)
//   K    [316][n][n] FP32 unit-level K_o (dense baseline, on first use)
//   per level: pairs grouped by offset (src, dst int32 [P]) for the forward
//   map and for the adjoint (roles swapped, offset reversed), a tile table
//   per nrhs, and scratch q~ / p~ FP32 [B*R][rp] plus BF16 pieces of q~
//   [pieces][B*R + 1][rp] whose last row is zero.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "kifmm_internal.h"
#include "plan.h"

using namespace kifmm;

namespace {

int pieces_for(int precision) {
    switch (precision) {
        case KIFMM_PREC_BF16: return 1;
        case KIFMM_PREC_SPLIT3: return 2;
        case KIFMM_PREC_SPLIT6: return 3;
        case KIFMM_PREC_F16X3: return 2;
        default: return 0;
    }
}
int products_for(int precision) {
    switch (precision) {
        case KIFMM_PREC_BF16: return 1;
        case KIFMM_PREC_SPLIT3: return 3;
        case KIFMM_PREC_SPLIT6: return 6;
        case KIFMM_PREC_F16X3: return 3;
        default: return 0;
    }
}

// IEEE 754 binary16 of v, round to nearest even (the host side of the FP16
// split of the cores): 10 fraction bits, exponent bias 15, subnormals in
// steps of 2^-24, |v| >= 65520 -> infinity.
uint16_t f16_bits_rn(double v) {
    const uint16_t sign = std::signbit(v) ? 0x8000u : 0u;
    const double a = std::fabs(v);
    if (a == 0.0) return sign;
    if (a >= 65520.0) return sign | 0x7C00u;
    int e2 = 0;
    std::frexp(a, &e2);        // a = f 2^e2, f in [0.5, 1)
    int E = e2 - 1;            // a in [2^E, 2^(E+1))
    if (E < -14) {             // subnormal: multiples of 2^-24 (1024 rounds up to the smallest normal)
        return sign | (uint16_t)std::nearbyint(std::ldexp(a, 24));
    }
    double m = std::nearbyint(std::ldexp(a, 10 - E));  // in [1024, 2048]
    if (m == 2048.0) {
        m = 1024.0;
        ++E;
    }
    if (E > 15) return sign | 0x7C00u;
    return sign | (uint16_t)((E + 15) << 10) | (uint16_t)(m - 1024.0);
}
double f16_bits_to_double(uint16_t b) {
    const int E = (b >> 10) & 0x1F, f = b & 0x3FF;
    const double mag = E == 0 ? std::ldexp((double)f, -24) : std::ldexp(1024.0 + f, E - 25);
    return (b & 0x8000u) ? -mag : mag;
}

// host split of FP64 into BF16 pieces (round to nearest even at each step)
uint16_t bf16_bits_rn(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}
float bf16_to_float(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

int build_pairset(const std::vector<int32_t>& tgt, const std::vector<int32_t>& src,
                  const std::vector<int32_t>& off, PairSet& ps) {
    ps.off_begin.assign(kOffsets + 1, 0);
    for (int32_t k : off) ps.off_begin[k + 1]++;
    for (int k = 0; k < kOffsets; ++k) ps.off_begin[k + 1] += ps.off_begin[k];
    ps.tilesets.clear();
    KIFMM_CUDA_TRY(ps.src.upload(src.data(), src.size()));
    KIFMM_CUDA_TRY(ps.dst.upload(tgt.data(), tgt.size()));
    ps.h_src = src;
    ps.h_dst = tgt;
    return KIFMM_OK;
}

int get_tiles(PairSet& ps, int nrhs, TileSet** out) {
    auto it = ps.tilesets.find(nrhs);
    if (it == ps.tilesets.end()) {
        std::vector<Tile> h;
        for (int k = 0; k < kOffsets; ++k) {
            const int64_t np = ps.off_begin[k + 1] - ps.off_begin[k];
            const int64_t rows = np * nrhs;
            for (int64_t r0 = 0; r0 < rows; r0 += kTileRows) {
                Tile t;
                t.k = k;
                t.pair_begin = (int)ps.off_begin[k];
                t.row0 = (int)r0;
                t.nrows = (int)std::min<int64_t>(kTileRows, rows - r0);
                h.push_back(t);
            }
        }
        auto ts = std::make_unique<TileSet>();
        int st = make_tileset(h, ps.h_src, ps.h_dst, nrhs, *ts);
        if (st != KIFMM_OK) return st;
        it = ps.tilesets.emplace(nrhs, std::move(ts)).first;
    }
    *out = it->second.get();
    return KIFMM_OK;
}

// Records a (start, stop) event pair around one stage when tracing is on.
struct StageTimer {
    kifmm_m2l_plan plan;
    cudaStream_t s;
    int stage;
    int launches;
    cudaEvent_t a = nullptr;
    StageTimer(kifmm_m2l_plan p, cudaStream_t st, int stg, int nl) : plan(p), s(st), stage(stg), launches(nl) {
        if (plan->profile) {
            a = plan->get_event();
            cudaEventRecord(a, s);
        }
    }
    ~StageTimer() {
        if (plan->profile && a) {
            cudaEvent_t b = plan->get_event();
            cudaEventRecord(b, s);
            plan->recs.push_back({stage, a, b});
            plan->traced_launches += launches;
        }
    }
};

// Shared body of apply / apply_adjoint: x_in -> y_out through
//   xt = W_in x ; yt = sum_pairs core xt ; y = beta y + s_l W_out yt
int apply_compressed(kifmm_m2l_plan plan, int instance, int level, int nrhs, const float* x_in, float* y_out,
                     float beta, void* stream, bool adjoint) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    LevelState* ls = find_level(plan, instance, level);
    if (!ls) {
        set_error("level not registered: call kifmm_m2l_set_level first");
        return KIFMM_ERR_STATE;
    }
    if (nrhs < 1 || (ls->n_boxes > 0 && (!x_in || !y_out))) {
        set_error("invalid nrhs or NULL density pointer");
        return KIFMM_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(x_in) & 15) || (reinterpret_cast<uintptr_t>(y_out) & 15)) {
        set_error("density pointers must be 16-byte aligned");
        return KIFMM_ERR_INVALID_ARG;
    }
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    if (ls->n_boxes == 0) return KIFMM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = plan->n, rp = plan->rp;
    const long rows = (long)ls->n_boxes * nrhs;
    if (rows + 1 > (long)INT32_MAX / 2) {
        set_error("too many box rows");
        return KIFMM_ERR_INVALID_ARG;
    }
    const float scale = (float)std::ldexp(1.0 / ls->r0, level);  // (r0 / 2^l)^-1
    const bool fp32_core = plan->prm.precision == KIFMM_PREC_FP32;
    const bool f16_core = plan->prm.precision == KIFMM_PREC_F16X3;
    const long piece_stride = (rows + 1) * rp;
    KIFMM_CUDA_TRY(plan->pt.ensure((size_t)rows * rp));
    if (fp32_core) KIFMM_CUDA_TRY(plan->qt.ensure((size_t)rows * rp));
    if (!fp32_core) KIFMM_CUDA_TRY(plan->qb.ensure((size_t)piece_stride * plan->pieces));
    if (f16_core) KIFMM_CUDA_TRY(plan->qs.ensure((size_t)rows + 1));

    // 1. compression  q~ = R~^T q  (adjoint: U~^T pbar; R~ = U~, so one factor
    //    serves both directions), written as the core's operand; p~ = 0
    const long vtiles = (rows + 127) / 128;
    KIFMM_CUDA_TRY(plan->sp.ensure(split_elems(plan, vtiles)));
    {
        StageTimer timer(plan, s, 0, 2);
        st = run_compress(plan, x_in, (int)rows, nullptr, 0, (int)vtiles, plan->sp.ptr, plan->qb.ptr, piece_stride,
                          fp32_core ? plan->qt.ptr : nullptr, plan->pt.ptr, s, f16_core ? plan->qs.ptr : nullptr);
        if (st != KIFMM_OK) return st;
        if (f16_core) {
            st = zero_core_operand_row_f16(plan, rows, plan->qb.ptr, piece_stride, plan->qs.ptr, s);
            if (st != KIFMM_OK) return st;
        }
    }

    // 2. core over offset-grouped pairs
    PairSet& ps = adjoint ? ls->adj : ls->fwd;
    TileSet* ts = nullptr;
    st = get_tiles(ps, nrhs, &ts);
    if (st != KIFMM_OK) return st;
    if (fp32_core) {
        StageTimer timer(plan, s, 1, 1);
        KIFMM_CUDA_TRY(launch_pairs_gemm_fp32(plan->qt.ptr, rp, plan->C.ptr, rp, rp, plan->pt.ptr, rp,
                                              ts->tiles.ptr, ts->n_tiles, ps.src.ptr, ps.dst.ptr, nrhs, 1.0f, s));
    } else {
        if (!f16_core)
            for (int pc = 0; pc < plan->pieces; ++pc)
                KIFMM_CUDA_TRY(cudaMemsetAsync(plan->qb.ptr + pc * piece_stride + rows * rp, 0,
                                               rp * sizeof(__nv_bfloat16), s));
        ScaleTable unit{};
        unit.s[0] = 1.0f;  // the level scale is applied by the expansion
        StageTimer timer(plan, s, 1, 1);
        st = launch_core(plan, plan->qb.ptr, piece_stride, (int)rows, *ts, nrhs, unit, plan->pt.ptr, s,
                         f16_core ? plan->qs.ptr : nullptr);
        if (st != KIFMM_OK) return st;
    }

    // 3. expansion  y = beta y + s_l U~ p~   (adjoint: R~ q~bar; R~ = U~)
    {
        StageTimer timer(plan, s, 2, 2);
        st = run_expand(plan, plan->pt.ptr, (int)rows, nullptr, 0, (int)vtiles, plan->sp.ptr, y_out, scale, beta, s);
        if (st != KIFMM_OK) return st;
    }
    return KIFMM_OK;
}


int get_multi(kifmm_m2l_plan plan, int instance, int lo, int hi, bool adjoint, MultiState** out) {
    return get_multi_state(plan, instance, lo, hi, adjoint, out);
}

int get_multi_tiles(MultiState& ms, int nrhs, TileSet** out) {
    auto it = ms.tilesets.find(nrhs);
    if (it == ms.tilesets.end()) {
        std::vector<Tile> h;
        for (const auto& g : ms.groups) {
            const int64_t rows = g.count * nrhs;
            for (int64_t r0 = 0; r0 < rows; r0 += kTileRows)
                h.push_back({g.k | (g.level_idx << 16), (int)g.begin, (int)r0,
                             (int)std::min<int64_t>(kTileRows, rows - r0)});
        }
        auto ts = std::make_unique<TileSet>();
        int st = make_tileset(h, ms.h_src, ms.h_dst, nrhs, *ts);
        if (st != KIFMM_OK) return st;
        it = ms.tilesets.emplace(nrhs, std::move(ts)).first;
    }
    *out = it->second.get();
    return KIFMM_OK;
}

// Levels lo..hi of one instance in five launches: split and compression of
// all their rows, one core over the merged offset-ordered tiles (each tile
// scaled by its level's s_l), split and expansion of all rows.
// With x_host / y_host set, the densities are HOST buffers: the rows reach
// the device in chunks on the plan's copy stream, each chunk's split and
// compression starting as soon as it has landed, and the expansion hands
// each chunk of results back the same way, so the copies overlap the
// compression and the expansion.
int apply_levels(kifmm_m2l_plan plan, int instance, int lo, int hi, int nrhs, const float* x_in, float* y_out,
                 float beta, void* stream, bool adjoint, const float* x_host = nullptr, float* y_host = nullptr) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (lo < 0 || hi < lo || hi - lo >= 32) {
        set_error("need 0 <= level_lo <= level_hi < level_lo + 32");
        return KIFMM_ERR_INVALID_ARG;
    }
    for (int l = lo; l <= hi; ++l)
        if (!find_level(plan, instance, l)) {
            set_error("level " + std::to_string(l) + " not registered: call kifmm_m2l_set_level first");
            return KIFMM_ERR_STATE;
        }
    if (nrhs < 1) {
        set_error("nrhs must be >= 1");
        return KIFMM_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(x_in) & 15) || (reinterpret_cast<uintptr_t>(y_out) & 15)) {
        set_error("density pointers must be 16-byte aligned");
        return KIFMM_ERR_INVALID_ARG;
    }
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    MultiState* ms = nullptr;
    st = get_multi(plan, instance, lo, hi, adjoint, &ms);
    if (st != KIFMM_OK) return st;
    if (ms->total_boxes == 0) return KIFMM_OK;
    const bool host = x_host != nullptr;
    if (host ? !y_host : (!x_in || !y_out)) {
        set_error("NULL density pointer");
        return KIFMM_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = plan->n, rp = plan->rp;
    const long rows = (long)ms->total_boxes * nrhs;
    if (rows + 1 > (long)INT32_MAX / 2) {
        set_error("too many box rows");
        return KIFMM_ERR_INVALID_ARG;
    }
    // host mode: device copies of the densities, chunks of whole 128-row tiles
    const int n_chunks = host ? (int)std::min<long>(4, (rows + 127) / 128) : 1;
    const long chunk_rows = ((rows + 127) / 128 + n_chunks - 1) / n_chunks * 128;
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> ev;
    if (host) {
        KIFMM_CUDA_TRY(plan->hx.ensure((size_t)rows * n));
        KIFMM_CUDA_TRY(plan->hy.ensure((size_t)rows * n));
        x_in = plan->hx.ptr;
        y_out = plan->hy.ptr;
        if (!plan->copy_stream) KIFMM_CUDA_TRY(cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking));
        cs = plan->copy_stream;
        while (plan->sync_events.size() < (size_t)(2 * n_chunks + 2)) {
            cudaEvent_t e = nullptr;
            KIFMM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            plan->sync_events.push_back(e);
        }
        // events: 0 start / end, 1 .. n_chunks the inputs, n_chunks + 1 the
        // copied-in p, n_chunks + 2 .. 2 n_chunks + 1 the outputs
        ev = plan->sync_events;
        // the copy stream starts after the work already on the caller's stream
        KIFMM_CUDA_TRY(cudaEventRecord(ev[0], s));
        KIFMM_CUDA_TRY(cudaStreamWaitEvent(cs, ev[0], 0));
        if (beta != 0.f)
            KIFMM_CUDA_TRY(cudaMemcpyAsync(plan->hy.ptr, y_host, (size_t)rows * n * sizeof(float),
                                           cudaMemcpyHostToDevice, cs));
    }
    const bool fp32_core = plan->prm.precision == KIFMM_PREC_FP32;
    const bool f16_core = plan->prm.precision == KIFMM_PREC_F16X3;
    const long piece_stride = (rows + 1) * rp;
    KIFMM_CUDA_TRY(plan->pt.ensure((size_t)rows * rp));
    if (fp32_core) KIFMM_CUDA_TRY(plan->qt.ensure((size_t)rows * rp));
    if (!fp32_core) KIFMM_CUDA_TRY(plan->qb.ensure((size_t)piece_stride * plan->pieces));
    if (f16_core) KIFMM_CUDA_TRY(plan->qs.ensure((size_t)rows + 1));
    TileSet* ts = nullptr;
    st = get_multi_tiles(*ms, nrhs, &ts);
    if (st != KIFMM_OK) return st;
    const long vtiles = (rows + 127) / 128;
    KIFMM_CUDA_TRY(plan->sp.ensure(split_elems(plan, vtiles)));
    {
        StageTimer timer(plan, s, 0, 2 * n_chunks);
        for (int c = 0; c < n_chunks; ++c) {
            const long r0 = c * chunk_rows, mc = std::min(chunk_rows, rows - r0);
            if (mc <= 0) break;
            const long t0 = r0 / 128, tc = (mc + 127) / 128;
            if (host) {
                KIFMM_CUDA_TRY(cudaMemcpyAsync(plan->hx.ptr + r0 * n, x_host + r0 * n, (size_t)mc * n * sizeof(float),
                                               cudaMemcpyHostToDevice, cs));
                KIFMM_CUDA_TRY(cudaEventRecord(ev[1 + c], cs));
                KIFMM_CUDA_TRY(cudaStreamWaitEvent(s, ev[1 + c], 0));
            }
            st = run_compress(plan, x_in + r0 * n, (int)mc, nullptr, 0, (int)tc,
                              plan->sp.ptr + (size_t)3 * 128 * t0 * plan->n_pad, plan->qb.ptr + r0 * rp, piece_stride,
                              fp32_core ? plan->qt.ptr + r0 * rp : nullptr, plan->pt.ptr + r0 * rp, s,
                              f16_core ? plan->qs.ptr + r0 : nullptr);
            if (st != KIFMM_OK) return st;
        }
        if (f16_core) {
            st = zero_core_operand_row_f16(plan, rows, plan->qb.ptr, piece_stride, plan->qs.ptr, s);
            if (st != KIFMM_OK) return st;
        }
    }
    if (host && beta != 0.f) {
        // the expansion accumulates into the copied-in p
        KIFMM_CUDA_TRY(cudaEventRecord(ev[1 + n_chunks], cs));
        KIFMM_CUDA_TRY(cudaStreamWaitEvent(s, ev[1 + n_chunks], 0));
    }
    ScaleTable scales{};
    for (int l = lo; l <= hi; ++l) {
        const LevelState* ls = find_level(plan, instance, l);
        scales.s[l - lo] = (float)std::ldexp(1.0 / ls->r0, l);
    }
    if (fp32_core) {
        StageTimer timer(plan, s, 1, 1);
        KIFMM_CUDA_TRY(launch_pairs_gemm_fp32(plan->qt.ptr, rp, plan->C.ptr, rp, rp, plan->pt.ptr, rp, ts->tiles.ptr,
                                              ts->n_tiles, ms->src.ptr, ms->dst.ptr, nrhs, scales, s));
    } else {
        if (!f16_core)
            for (int pc = 0; pc < plan->pieces; ++pc)
                KIFMM_CUDA_TRY(cudaMemsetAsync(plan->qb.ptr + pc * piece_stride + rows * rp, 0,
                                               rp * sizeof(__nv_bfloat16), s));
        StageTimer timer(plan, s, 1, 1);
        st = launch_core(plan, plan->qb.ptr, piece_stride, (int)rows, *ts, nrhs, scales, plan->pt.ptr, s,
                         f16_core ? plan->qs.ptr : nullptr);
        if (st != KIFMM_OK) return st;
    }
    {
        StageTimer timer(plan, s, 2, 2 * n_chunks);
        for (int c = 0; c < n_chunks; ++c) {
            const long r0 = c * chunk_rows, mc = std::min(chunk_rows, rows - r0);
            if (mc <= 0) break;
            const long t0 = r0 / 128, tc = (mc + 127) / 128;
            st = run_expand(plan, plan->pt.ptr + r0 * rp, (int)mc, nullptr, 0, (int)tc,
                            plan->sp.ptr + (size_t)3 * 128 * t0 * rp, y_out + r0 * n, 1.0f, beta, s);
            if (st != KIFMM_OK) return st;
            if (host) {
                KIFMM_CUDA_TRY(cudaEventRecord(ev[2 + n_chunks + c], s));
                KIFMM_CUDA_TRY(cudaStreamWaitEvent(cs, ev[2 + n_chunks + c], 0));
                KIFMM_CUDA_TRY(cudaMemcpyAsync(y_host + r0 * n, plan->hy.ptr + r0 * n, (size_t)mc * n * sizeof(float),
                                               cudaMemcpyDeviceToHost, cs));
            }
        }
    }
    if (host) {
        // the caller's stream covers every copy
        KIFMM_CUDA_TRY(cudaEventRecord(ev[0], cs));
        KIFMM_CUDA_TRY(cudaStreamWaitEvent(s, ev[0], 0));
    }
    return KIFMM_OK;
}

}  // namespace

namespace kifmm {

int multi_tileset(MultiState& ms, int nrhs, TileSet** out) { return get_multi_tiles(ms, nrhs, out); }

int launch_core(kifmm_m2l_plan plan, const __nv_bfloat16* qb, long piece_stride, int zero_row, const TileSet& ts,
                int nrhs, const ScaleTable& scales, float* pt, cudaStream_t s, const float* row_scale) {
    UmmaArgs a{};
    if (plan->prm.precision == KIFMM_PREC_F16X3) {
        if (!row_scale) {
            set_error("the FP16 core needs the per-row factors of its operand");
            return KIFMM_ERR_INVALID_ARG;
        }
        a.f16 = 1;
        a.row_scale = row_scale;
    }
    a.A = qb;
    a.a_piece_stride = piece_stride;
    a.kdim = plan->rp;
    a.B = plan->Cb.ptr;
    a.b_groups = kOffsets;
    a.ndim = plan->rp;
    a.n_chunk = core_chunk(plan);
    a.contiguous = plan->tune_contig;
    a.core_resident = plan->tune_variant == 1;
    a.core_drain = plan->variant_drain();
    a.red_bulk = plan->variant_bulk();
    a.mma_pair = plan->variant_pair();
    a.direct_rows = plan->variant_direct();
    a.core_bres = plan->variant_bres();
    a.s2_on = plan->s2_on;
    a.s2_V = plan->s2V.ptr;
    a.s2_U = plan->s2U.ptr;
    a.s2_k16 = plan->s2_k16.ptr;
    a.row_src = ts.row_src.ptr;
    a.row_dst = ts.row_dst.ptr;
    a.tile_k = ts.tile_k.ptr;
    a.n_tiles = ts.n_tiles;
    a.nrhs = nrhs;
    a.zero_row = zero_row;
    for (int i = 0; i < 32; ++i) a.level_scale[i] = scales.s[i] * plan->out_inv_scale();
    a.D = pt;
    a.ldd = plan->rp;
    a.n_products = plan->products;
    a.hilo = plan->core_hilo;
    a.error_flag = plan->err_flag.ptr;
    a.wait_ns = plan->core_wait_ns;
    KIFMM_CUDA_TRY(launch_umma(A_GATHER, E_RED, a, plan->num_sms, s));
    return KIFMM_OK;
}

int zero_core_operand_row_f16(kifmm_m2l_plan plan, long rows, __nv_bfloat16* qb, long piece_stride, float* qs,
                              cudaStream_t s) {
    const int rp = plan->rp;
    for (int pc = 0; pc < 2; ++pc)
        KIFMM_CUDA_TRY(cudaMemsetAsync(qb + pc * piece_stride + rows * rp, 0, rp * sizeof(__nv_bfloat16), s));
    KIFMM_CUDA_TRY(cudaMemsetAsync(qs + rows, 0, sizeof(float), s));
    return KIFMM_OK;
}

int split_core_operand_f16(kifmm_m2l_plan plan, const float* qt, long rows, __nv_bfloat16* qb, long piece_stride,
                           float* qs, cudaStream_t s) {
    const int rp = plan->rp;
    KIFMM_CUDA_TRY(launch_split_rows_f16_scaled(qt, (int)rows, rp, rp, rp, reinterpret_cast<__half*>(qb), piece_stride,
                                                qs, s));
    for (int pc = 0; pc < 2; ++pc)
        KIFMM_CUDA_TRY(cudaMemsetAsync(qb + pc * piece_stride + rows * rp, 0, rp * sizeof(__nv_bfloat16), s));
    KIFMM_CUDA_TRY(cudaMemsetAsync(qs + rows, 0, sizeof(float), s));
    return KIFMM_OK;
}

int upload_pieces(DevBuf<__nv_bfloat16>& dst, size_t per, const std::function<double(size_t)>& value_at) {
    std::vector<uint16_t> h(per * 3, 0);
    for (size_t e = 0; e < per; ++e) {
        double v = value_at(e);
        if (v == 0.0) continue;
        for (int pc = 0; pc < 3; ++pc) {
            const uint16_t b = bf16_bits_rn((float)v);
            h[pc * per + e] = b;
            v -= (double)bf16_to_float(b);
        }
    }
    KIFMM_CUDA_TRY(dst.ensure(h.size()));
    KIFMM_CUDA_TRY(cudaMemcpy(dst.ptr, h.data(), h.size() * 2, cudaMemcpyHostToDevice));
    return KIFMM_OK;
}

// N per work item of the compression / expansion GEMMs: <= 64, so that the
// partial sums of a row fit in registers next to a loaded TMEM chunk, and
// four accumulator slots (two partials, two lo) fit in the TMEM columns.
int chunk_for(int ndim) {
    const int parts = (ndim + 63) / 64;
    return ((ndim + parts - 1) / parts + 15) / 16 * 16;
}

int core_chunk(kifmm_m2l_plan plan) { return plan->tune_chunk ? plan->tune_chunk : core_chunk_default(plan); }

int core_chunk_default(kifmm_m2l_plan plan) {
    const int rp = plan->rp;
    // hi and lo side by side must fit the 512 TMEM columns (one slot); a
    // split of N would gather every A row once per part, which costs more
    // than the lost overlap of epilogue and MMA
    if (plan->core_hilo && plan->products > 1 && 2 * rp > 512) return (rp / 2 + 15) / 16 * 16;
    return rp;
}

// N per work item of the identity-row GEMMs: <= max_n (at most 192: 96
// running sums per thread in the drained epilogue), split further while the
// tiles would not fill two waves of CTAs.
int rows_chunk(int ndim, long n_tiles, int num_sms, int max_n) {
    int c = (ndim + max_n - 1) / max_n;
    while (n_tiles * c < 2L * num_sms && ndim / (c + 1) >= 64) ++c;
    return ((ndim + c - 1) / c + 15) / 16 * 16;
}

size_t split_elems(kifmm_m2l_plan plan, long n_tiles) {
    return (size_t)3 * 128 * (size_t)std::max<long>(n_tiles, 1) * (size_t)std::max(plan->n_pad, plan->rp);
}

int run_compress(kifmm_m2l_plan plan, const float* x, int m_rows, const RowSeg* segs, int n_segs, int n_tiles,
                 __nv_bfloat16* split, __nv_bfloat16* qb, long qb_stride, float* qt, float* pt, cudaStream_t s,
                 float* f16_inv) {
    if (n_tiles <= 0) return KIFMM_OK;
    const int n = plan->n, np = plan->n_pad, rp = plan->rp;
    const long sp_stride = (long)n_tiles * 128 * np;
    KIFMM_CUDA_TRY(launch_split_rows(x, m_rows, n, n, np, segs, n_segs, n_tiles, split, sp_stride, 3, s, 1, f16_inv));
    UmmaArgs a{};
    a.A = split;
    a.a_piece_stride = sp_stride;
    a.kdim = np;
    a.B = plan->Rtb.ptr;
    a.b_groups = 1;
    a.ndim = rp;
    a.n_chunk = rows_chunk(rp, n_tiles, plan->num_sms, 128);
    a.row_identity = 1;
    a.n_tiles = n_tiles;
    a.m_rows = m_rows;
    a.segs = segs;
    a.n_segs = n_segs;
    a.seg_tiles = n_tiles;
    a.ldd = rp;
    a.alpha = 1.0f;
    a.Dp = qt ? nullptr : qb;
    a.dp_piece_stride = qb_stride;
    a.dp_pieces = qt ? 0 : (f16_inv ? 2 : plan->pieces);
    // f16x3: q~ rows as two FP16 pieces after the power of two of the input
    // row's 2-norm (|q~_i| <= ||q~|| <= ||q|| with orthonormal R~ columns, so
    // the pieces stay below 2^15), written by the GEMM itself
    a.dp_f16 = f16_inv ? 1 : 0;
    a.dp_row_inv = f16_inv;
    a.Df = qt;
    a.Z = pt;
    a.n_products = 6;
    a.hilo = 1;
    // three K-chunks per drained partial, the (0,0) product in its own half of
    // the slot (N <= 128 so that two slots of 2 N columns fit): 6
    // full-magnitude MMAs per accumulator chain
    a.core_drain = 3;
    a.error_flag = plan->err_flag.ptr;
    KIFMM_CUDA_TRY(launch_umma(A_GATHER, E_SPLIT, a, plan->num_sms, s));
    return KIFMM_OK;
}

int run_expand(kifmm_m2l_plan plan, const float* pt, int m_rows, const RowSeg* segs, int n_segs, int n_tiles,
               __nv_bfloat16* split, float* y, float alpha, float beta, cudaStream_t s) {
    if (n_tiles <= 0) return KIFMM_OK;
    const int n = plan->n, np = plan->n_pad, rp = plan->rp;
    const long sp_stride = (long)n_tiles * 128 * rp;
    KIFMM_CUDA_TRY(launch_split_rows(pt, m_rows, rp, rp, rp, segs, n_segs, n_tiles, split, sp_stride, 3, s));
    UmmaArgs a{};
    a.A = split;
    a.a_piece_stride = sp_stride;
    a.kdim = rp;
    a.B = plan->Ub.ptr;
    a.b_groups = 1;
    a.ndim = np;
    a.n_chunk = rows_chunk(np, n_tiles, plan->num_sms, 192);
    a.row_identity = 1;
    a.n_tiles = n_tiles;
    a.m_rows = m_rows;
    a.segs = segs;
    a.n_segs = n_segs;
    a.seg_tiles = n_tiles;
    a.D = y;
    a.ldd = n;
    a.alpha = alpha;
    a.beta = beta;
    a.n_valid = n;
    a.n_products = 6;
    a.hilo = 1;
    // three K-chunks per drained partial with the (0,0) product apart where
    // two slots of 2 N columns fit (N <= 128); wider N parts (n_pad / 2 at
    // p = 8) fall back to one K-chunk per partial in the launcher
    a.core_drain = 3;
    a.error_flag = plan->err_flag.ptr;
    KIFMM_CUDA_TRY(launch_umma(A_GATHER, E_STORE, a, plan->num_sms, s));
    return KIFMM_OK;
}

int check_device(kifmm_m2l_plan plan) {
    int dev = -1;
    KIFMM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != plan->device) {
        set_error("the current CUDA device differs from the plan's device");
        return KIFMM_ERR_INVALID_ARG;
    }
    return KIFMM_OK;
}

int make_tileset(const std::vector<Tile>& tiles, const std::vector<int32_t>& src, const std::vector<int32_t>& dst,
                 int nrhs, TileSet& out) {
    const size_t nt = tiles.size();
    std::vector<int> rs(nt * kTileRows, -1), rd(nt * kTileRows, -1), tk(nt);
    for (size_t t = 0; t < nt; ++t) {
        const Tile& tl = tiles[t];
        tk[t] = tl.k;
        for (int r = 0; r < tl.nrows; ++r) {
            const int64_t g = (int64_t)tl.row0 + r;
            const int64_t pr = tl.pair_begin + g / nrhs;
            const int64_t rhs = g % nrhs;
            rs[t * kTileRows + r] = (int)(src[pr] * (int64_t)nrhs + rhs);
            rd[t * kTileRows + r] = (int)(dst[pr] * (int64_t)nrhs + rhs);
        }
    }
    KIFMM_CUDA_TRY(out.tiles.upload(tiles.data(), nt));
    KIFMM_CUDA_TRY(out.row_src.upload(rs.data(), rs.size()));
    KIFMM_CUDA_TRY(out.row_dst.upload(rd.data(), rd.size()));
    KIFMM_CUDA_TRY(out.tile_k.upload(tk.data(), tk.size()));
    out.n_tiles = (int)nt;
    return KIFMM_OK;
}

// Merged pairs of levels lo..hi of one instance (forward or adjoint), built
// on first use and cached in the plan.
int get_multi_state(kifmm_m2l_plan plan, int instance, int lo, int hi, bool adjoint, MultiState** out) {
    const auto key = std::make_tuple(instance, lo, hi, adjoint ? 1 : 0);
    auto it = plan->multi.find(key);
    if (it != plan->multi.end()) {
        *out = it->second.get();
        return KIFMM_OK;
    }
    auto ms = std::make_unique<MultiState>();
    std::vector<int64_t> box_off(hi - lo + 1);
    std::vector<PairSet*> sets(hi - lo + 1);
    for (int l = lo; l <= hi; ++l) {
        LevelState* ls = find_level(plan, instance, l);
        box_off[l - lo] = ms->total_boxes;
        ms->total_boxes += ls->n_boxes;
        sets[l - lo] = adjoint ? &ls->adj : &ls->fwd;
    }
    std::vector<int32_t> src, dst;
    for (int k = 0; k < kOffsets; ++k)
        for (int li = 0; li <= hi - lo; ++li) {
            PairSet& ps = *sets[li];
            const int64_t b = ps.off_begin[k], e = ps.off_begin[k + 1];
            if (e == b) continue;
            ms->groups.push_back({k, li, (int64_t)src.size(), e - b});
            for (int64_t i = b; i < e; ++i) {
                src.push_back((int32_t)(ps.h_src[i] + box_off[li]));
                dst.push_back((int32_t)(ps.h_dst[i] + box_off[li]));
            }
        }
    KIFMM_CUDA_TRY(ms->src.upload(src.data(), src.size()));
    KIFMM_CUDA_TRY(ms->dst.upload(dst.data(), dst.size()));
    ms->h_src.swap(src);
    ms->h_dst.swap(dst);
    *out = ms.get();
    plan->multi[key] = std::move(ms);
    return KIFMM_OK;
}

LevelState* find_level(kifmm_m2l_plan plan, int instance, int level) {
    auto it = plan->levels.find({instance, level});
    return it == plan->levels.end() ? nullptr : it->second.get();
}

}  // namespace kifmm

namespace kifmm {

int register_level(kifmm_m2l_plan plan, int instance, int level, double root_halfwidth, int n_boxes,
                   const int32_t* box_ijk) {
    int st = KIFMM_OK;
    if (plan->prm.kernel_id == KIFMM_KERNEL_YUKAWA) {
        // the operators were formed for boxes of one half-width (Sec. 3.1, O(L) case)
        const double h = std::ldexp(root_halfwidth, -level), hp = plan->prm.box_halfwidth;
        if (!(std::fabs(h - hp) <= 1e-12 * hp)) {
            set_error("this Yukawa plan serves boxes of half-width " + std::to_string(hp) + ", level " +
                      std::to_string(level) + " has " + std::to_string(h) + ": one plan per level");
            return KIFMM_ERR_INVALID_ARG;
        }
    }
    try {
        std::vector<int32_t> tg, sr, of;
        st = build_pairs(level, n_boxes, box_ijk, tg, sr, of);
        if (st != KIFMM_OK) return st;
        auto ls = std::make_unique<LevelState>();
        ls->level = level;
        ls->n_boxes = n_boxes;
        ls->r0 = root_halfwidth;
        ls->n_pairs = (int64_t)tg.size();
        st = build_pairset(tg, sr, of, ls->fwd);
        if (st != KIFMM_OK) return st;
        // adjoint: target' = s, source' = t, offset' = -o; regroup by offset'
        int offs[kOffsets][3];
        offsets316(offs);
        std::vector<int> neg(kOffsets);
        for (int k = 0; k < kOffsets; ++k) neg[k] = offset_index(-offs[k][0], -offs[k][1], -offs[k][2]);
        std::vector<int32_t> atg(tg.size()), asr(tg.size()), aof(tg.size());
        // regroup by reversed offset, each group sorted by its new target
        std::vector<std::vector<std::pair<int32_t, int32_t>>> grp(kOffsets);
        for (size_t i = 0; i < tg.size(); ++i) grp[neg[of[i]]].push_back({sr[i], tg[i]});
        size_t w = 0;
        for (int k = 0; k < kOffsets; ++k) {
            std::sort(grp[k].begin(), grp[k].end());
            for (auto& ts : grp[k]) {
                atg[w] = ts.first;
                asr[w] = ts.second;
                aof[w] = k;
                ++w;
            }
        }
        st = build_pairset(atg, asr, aof, ls->adj);
        if (st != KIFMM_OK) return st;
        forget_batches_of(plan);
        plan->levels[{instance, level}] = std::move(ls);
        for (auto it = plan->multi.begin(); it != plan->multi.end();) {
            const auto& key = it->first;
            if (std::get<0>(key) == instance && std::get<1>(key) <= level && level <= std::get<2>(key))
                it = plan->multi.erase(it);
            else
                ++it;
        }
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    return KIFMM_OK;
}

}  // namespace kifmm

extern "C" {

const char* kifmm_m2l_last_error(void) { return kifmm::last_error(); }

const char* kifmm_m2l_version(void) { return "kifmm_m2l 0.1 (sm_103a)"; }

int kifmm_m2l_factors_host(const kifmm_m2l_params* params, int* n, int* r, double* sigma, double* U, double* C) {
    int st = check_params(params);
    if (st != KIFMM_OK) return st;
    Factors f;
    st = compute_factors(*params, f);
    if (st != KIFMM_OK) return st;
    if (n) *n = f.n;
    if (r) *r = f.r;
    if (sigma) std::memcpy(sigma, f.sigma.data(), sizeof(double) * f.n);
    if (U) std::memcpy(U, f.U.data(), sizeof(double) * f.U.size());
    if (C) std::memcpy(C, f.C.data(), sizeof(double) * f.C.size());
    return KIFMM_OK;
}

int kifmm_m2l_pairs_host(int level, int n_boxes, const int32_t* box_ijk, int64_t* n_pairs, int32_t* targets,
                         int32_t* sources, int32_t* offsets) {
    if (!n_pairs) {
        set_error("n_pairs is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    std::vector<int32_t> tg, sr, of;
    int st;
    try {
        st = build_pairs(level, n_boxes, box_ijk, tg, sr, of);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    if (st != KIFMM_OK) return st;
    if (targets) {
        if (!sources || !offsets) {
            set_error("targets, sources and offsets must all be given");
            return KIFMM_ERR_INVALID_ARG;
        }
        std::memcpy(targets, tg.data(), tg.size() * 4);
        std::memcpy(sources, sr.data(), sr.size() * 4);
        std::memcpy(offsets, of.data(), of.size() * 4);
    }
    *n_pairs = (int64_t)tg.size();
    return KIFMM_OK;
}

int kifmm_m2l_precompute(const kifmm_m2l_params* params, kifmm_m2l_plan* out) {
    if (!out) {
        set_error("out is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int st = check_params(params);
    if (st != KIFMM_OK) return st;
    std::unique_ptr<kifmm_m2l_plan_s> plan;
    try {
        plan.reset(new kifmm_m2l_plan_s());
        plan->prm = *params;
        Factors f;
        st = compute_factors(*params, f);
        if (st != KIFMM_OK) return st;
        if (f.sym_err > 1e-10) {
            set_error("K~_o^T = K~_{-o} does not hold (relative error " + std::to_string(f.sym_err) + ")");
            return KIFMM_ERR_UNSUPPORTED;
        }
        KIFMM_CUDA_TRY(cudaGetDevice(&plan->device));
        KIFMM_CUDA_TRY(cudaDeviceGetAttribute(&plan->num_sms, cudaDevAttrMultiProcessorCount, plan->device));
        const int n = f.n, r = f.r, rp = (r + 15) / 16 * 16;
        plan->n = n;
        plan->r = r;
        plan->rp = rp;
        plan->sym_err = f.sym_err;
        plan->sigma = f.sigma;
        plan->pieces = pieces_for(params->precision);
        plan->products = products_for(params->precision);
        {
            int major = 0, minor = 0;
            KIFMM_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, plan->device));
            KIFMM_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, plan->device));
            if (major != 10 || minor != 3) {
                set_error("this library's tcgen05 kernels need an sm_103 (GB300) device");
                return KIFMM_ERR_UNSUPPORTED;
            }
        }
        const int np = (n + 15) / 16 * 16;
        plan->n_pad = np;
        std::vector<float> h_c((size_t)kOffsets * rp * rp, 0.f);
        for (int k = 0; k < kOffsets; ++k)
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b)
                    h_c[((size_t)k * rp + a) * rp + b] = (float)f.C[((size_t)k * r + a) * r + b];
        KIFMM_CUDA_TRY(plan->C.upload(h_c.data(), h_c.size()));
        // 3-piece BF16 splits of the FP64 factors: piece j = RN(x - earlier pieces)
        auto split_upload = [&](DevBuf<__nv_bfloat16>& dst, size_t per, auto value_at) -> int {
            return upload_pieces(dst, per, value_at);
        };
        plan->U64 = f.U;
        // K~_o as [316][rp][rp]
        st = split_upload(plan->Cb, (size_t)kOffsets * rp * rp, [&](size_t e) -> double {
            const size_t k = e / ((size_t)rp * rp), a = (e / rp) % rp, b = e % rp;
            return (a < (size_t)r && b < (size_t)r) ? f.C[(k * r + a) * r + b] : 0.0;
        });
        if (st != KIFMM_OK) return st;
        // R~^T as [rp][np]: row a = column a of R~ (= U~)
        st = split_upload(plan->Rtb, (size_t)rp * np, [&](size_t e) -> double {
            const size_t a = e / np, i = e % np;
            return (a < (size_t)r && i < (size_t)n) ? f.U[i * r + a] : 0.0;
        });
        if (st != KIFMM_OK) return st;
        // U~ as [np][rp]
        st = split_upload(plan->Ub, (size_t)np * rp, [&](size_t e) -> double {
            const size_t i = e / rp, a = e % rp;
            return (a < (size_t)r && i < (size_t)n) ? f.U[i * r + a] : 0.0;
        });
        if (st != KIFMM_OK) return st;
        if (params->precision == KIFMM_PREC_F16X3) {
            // K~_o as two FP16 pieces of tau K~_o, tau the power of two that puts
            // max |K~| in [2^13, 2^14); the core divides by tau in its output scale
            double cmax = 0;
            for (double v : f.C) cmax = std::max(cmax, std::fabs(v));
            int e2 = 0;
            std::frexp(cmax > 0 ? cmax : 1.0, &e2);  // cmax in [2^(e2-1), 2^e2)
            const double tau = std::ldexp(1.0, 14 - e2);
            plan->core_inv_scale = (float)(1.0 / tau);
            const size_t per = (size_t)kOffsets * rp * rp;
            std::vector<uint16_t> h(per * 2, 0);
            for (size_t e = 0; e < per; ++e) {
                const size_t k = e / ((size_t)rp * rp), a = (e / rp) % rp, b = e % rp;
                if (a >= (size_t)r || b >= (size_t)r) continue;
                const double v = tau * f.C[(k * r + a) * r + b];
                h[e] = f16_bits_rn(v);
                h[per + e] = f16_bits_rn(v - f16_bits_to_double(h[e]));
            }
            KIFMM_CUDA_TRY(plan->Cb.ensure(h.size()));
            KIFMM_CUDA_TRY(cudaMemcpy(plan->Cb.ptr, h.data(), h.size() * 2, cudaMemcpyHostToDevice));
        }
        // SPLIT6 keeps the (0,0) product in its own accumulator: the tensor
        // core's accumulation error grows with the number of MMA steps that
        // round at the full magnitude, and the 5 small products would
        // otherwise add 5 such steps per K step.  F16X3 likewise.
        plan->core_hilo = (params->precision == KIFMM_PREC_SPLIT6 || params->precision == KIFMM_PREC_F16X3) ? 1 : 0;
        KIFMM_CUDA_TRY(plan->err_flag.ensure(1));
        KIFMM_CUDA_TRY(cudaMemset(plan->err_flag.ptr, 0, sizeof(int)));
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    *out = plan.release();
    return KIFMM_OK;
}

int kifmm_m2l_destroy(kifmm_m2l_plan plan) {
    if (plan) {
        forget_batches_of(plan);
        detach_fmms(plan);
    }
    delete plan;
    return KIFMM_OK;
}

int kifmm_m2l_plan_rank(kifmm_m2l_plan plan, int* r, int* r_pad, int* n) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (r) *r = plan->r;
    if (r_pad) *r_pad = plan->rp;
    if (n) *n = plan->n;
    return KIFMM_OK;
}

int kifmm_m2l_set_stage2(kifmm_m2l_plan plan, double c2) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    // cached batches hold scale tables made for the previous operator
    forget_batches_of(plan);
    if (!(c2 > 0)) {
        plan->s2_on = 0;
        plan->s2_c2 = 0;
        plan->s2_k.clear();
        plan->s2_inv_scale = 1.0f;
        return KIFMM_OK;
    }
    if (plan->prm.precision == KIFMM_PREC_FP32) {
        set_error("stage 2 runs on the tensor-core precisions only (FP32 plans use the SIMT core)");
        return KIFMM_ERR_UNSUPPORTED;
    }
    if (plan->rp > 512 - 2 * 96) {
        set_error("stage 2 needs r_pad <= 320");
        return KIFMM_ERR_UNSUPPORTED;
    }
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    try {
        Factors f;
        st = compute_factors(plan->prm, f);
        if (st != KIFMM_OK) return st;
        Stage2 s2;
        st = compute_stage2(f, c2, s2);
        if (st != KIFMM_OK) return st;
        int kmax = 0;
        for (int k : s2.k) kmax = std::max(kmax, k);
        if (kmax > 96) {
            set_error("stage 2: a per-offset rank exceeds 96 (largest " + std::to_string(kmax) +
                      "); use a larger c2");
            return KIFMM_ERR_UNSUPPORTED;
        }
        const int r = plan->r, rp = plan->rp;
        std::vector<int> k16(kOffsets);
        for (int o = 0; o < kOffsets; ++o) k16[o] = std::max(16, (s2.k[o] + 15) / 16 * 16);
        // Vhat_o rows, [3][316][96][rp]; Uhat_o rows, [3][316][rp][96]; zero
        // padding.  BF16 modes: three BF16 pieces.  F16X3: two FP16 pieces of
        // tau x (tau the power of two that puts the factor's largest entry in
        // [2^13, 2^14)), the third piece zero; the core divides by both taus.
        const bool f16 = plan->prm.precision == KIFMM_PREC_F16X3;
        auto split_upload = [&](kifmm::DevBuf<__nv_bfloat16>& dst, size_t per, auto value_at, double* inv) -> int {
            double tau = 1.0;
            if (f16) {
                double vmax = 0;
                for (size_t e = 0; e < per; ++e) vmax = std::max(vmax, std::fabs(value_at(e)));
                int e2 = 0;
                std::frexp(vmax > 0 ? vmax : 1.0, &e2);  // vmax in [2^(e2-1), 2^e2)
                tau = std::ldexp(1.0, 14 - e2);
            }
            *inv = 1.0 / tau;
            std::vector<uint16_t> h(per * 3, 0);
            for (size_t e = 0; e < per; ++e) {
                double v = value_at(e);
                if (v == 0.0) continue;
                if (f16) {
                    v *= tau;
                    h[e] = f16_bits_rn(v);
                    h[per + e] = f16_bits_rn(v - f16_bits_to_double(h[e]));
                    continue;
                }
                for (int pc = 0; pc < 3; ++pc) {
                    const uint16_t b = bf16_bits_rn((float)v);
                    h[pc * per + e] = b;
                    v -= (double)bf16_to_float(b);
                }
            }
            KIFMM_CUDA_TRY(dst.ensure(h.size()));
            KIFMM_CUDA_TRY(cudaMemcpy(dst.ptr, h.data(), h.size() * 2, cudaMemcpyHostToDevice));
            return KIFMM_OK;
        };
        double inv_v = 1.0, inv_u = 1.0;
        st = split_upload(plan->s2V, (size_t)kOffsets * 96 * rp, [&](size_t e) -> double {
            const size_t o = e / ((size_t)96 * rp), j = (e / rp) % 96, b = e % rp;
            return (j < (size_t)s2.k[o] && b < (size_t)r) ? s2.Vh[o][j * r + b] : 0.0;
        }, &inv_v);
        if (st != KIFMM_OK) return st;
        st = split_upload(plan->s2U, (size_t)kOffsets * rp * 96, [&](size_t e) -> double {
            const size_t o = e / ((size_t)rp * 96), a = (e / 96) % rp, j = e % 96;
            return (a < (size_t)r && j < (size_t)s2.k[o]) ? s2.Uh[o][a * s2.k[o] + j] : 0.0;
        }, &inv_u);
        if (st != KIFMM_OK) return st;
        plan->s2_inv_scale = (float)(inv_v * inv_u);
        KIFMM_CUDA_TRY(plan->s2_k16.upload(k16.data(), k16.size()));
        plan->s2_k = s2.k;
        plan->s2_c2 = c2;
        plan->s2_on = 1;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed in kifmm_m2l_set_stage2");
        return KIFMM_ERR_OOM;
    }
    return KIFMM_OK;
}

int kifmm_m2l_stage2_host(const kifmm_m2l_params* params, double c2, int* k, double* core) {
    int st = check_params(params);
    if (st != KIFMM_OK) return st;
    if (!k) {
        set_error("k is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    try {
        Factors f;
        st = compute_factors(*params, f);
        if (st != KIFMM_OK) return st;
        Stage2 s2;
        st = compute_stage2(f, c2, s2);
        if (st != KIFMM_OK) return st;
        const int r = f.r;
        for (int o = 0; o < kOffsets; ++o) {
            k[o] = s2.k[o];
            if (!core) continue;
            double* c = core + (size_t)o * r * r;
            const int ko = s2.k[o];
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b) {
                    double acc = 0;
                    for (int j = 0; j < ko; ++j) acc += s2.Uh[o][(size_t)a * ko + j] * s2.Vh[o][(size_t)j * r + b];
                    c[(size_t)a * r + b] = acc;
                }
        }
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed in kifmm_m2l_stage2_host");
        return KIFMM_ERR_OOM;
    }
    return KIFMM_OK;
}

int kifmm_m2l_stage2_ranks(kifmm_m2l_plan plan, int* k) {
    if (!plan || !k) {
        set_error("plan or k is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (!plan->s2_on) {
        set_error("stage 2 is off: call kifmm_m2l_set_stage2 first");
        return KIFMM_ERR_STATE;
    }
    for (int o = 0; o < kOffsets; ++o) k[o] = plan->s2_k[o];
    return KIFMM_OK;
}

int kifmm_m2l_set_level(kifmm_m2l_plan plan, int instance, int level, double root_halfwidth, int n_boxes,
                        const int32_t* box_ijk) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (instance < 0 || !(root_halfwidth > 0) || !std::isfinite(root_halfwidth)) {
        set_error("instance must be >= 0 and root_halfwidth > 0");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (instance >= kReservedInstance) {
        set_error("instances >= 2^30 are reserved for point-source evaluations");
        return KIFMM_ERR_INVALID_ARG;
    }
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    return register_level(plan, instance, level, root_halfwidth, n_boxes, box_ijk);
}

int kifmm_m2l_sync(kifmm_m2l_plan plan, void* stream) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    KIFMM_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int flag = 0;
    KIFMM_CUDA_TRY(cudaMemcpy(&flag, plan->err_flag.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        KIFMM_CUDA_TRY(cudaMemset(plan->err_flag.ptr, 0, sizeof(int)));
        set_error("a bounded wait inside the tensor-core kernel timed out; results are invalid");
        return KIFMM_ERR_TIMEOUT;
    }
    return KIFMM_OK;
}

int kifmm_m2l_set_wait_limit(kifmm_m2l_plan plan, unsigned long long ns) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    plan->core_wait_ns = ns;
    return KIFMM_OK;
}

int kifmm_m2l_profile_enable(kifmm_m2l_plan plan, int enable) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    plan->profile = enable != 0;
    return KIFMM_OK;
}

int kifmm_m2l_profile_read(kifmm_m2l_plan plan, double* ms, int64_t* launches) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    double acc[3] = {0, 0, 0};
    int status = KIFMM_OK;
    for (auto& r : plan->recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess && status == KIFMM_OK) {
            set_error(std::string("cudaEventElapsedTime: ") + cudaGetErrorString(e));
            status = KIFMM_ERR_CUDA;
        }
        acc[r.stage] += t;
        plan->event_pool.push_back(r.a);
        plan->event_pool.push_back(r.b);
    }
    plan->recs.clear();
    if (ms)
        for (int i = 0; i < 3; ++i) ms[i] = acc[i];
    if (launches) *launches = plan->traced_launches;
    plan->traced_launches = 0;
    return status;
}

int kifmm_m2l_level_pairs(kifmm_m2l_plan plan, int instance, int level, int64_t* n_pairs) {
    if (!plan || !n_pairs) {
        set_error("plan or n_pairs is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    LevelState* ls = find_level(plan, instance, level);
    if (!ls) {
        set_error("level not registered");
        return KIFMM_ERR_STATE;
    }
    *n_pairs = ls->n_pairs;
    return KIFMM_OK;
}

int kifmm_m2l_apply(kifmm_m2l_plan plan, int instance, int level, int nrhs, const float* q_up, float* p_down,
                    float beta, void* stream) {
    return apply_compressed(plan, instance, level, nrhs, q_up, p_down, beta, stream, false);
}

int kifmm_m2l_apply_adjoint(kifmm_m2l_plan plan, int instance, int level, int nrhs, const float* pbar_down,
                            float* qbar_up, float beta, void* stream) {
    return apply_compressed(plan, instance, level, nrhs, pbar_down, qbar_up, beta, stream, true);
}

int kifmm_m2l_apply_levels(kifmm_m2l_plan plan, int instance, int level_lo, int level_hi, int nrhs,
                           const float* q_up, float* p_down, float beta, void* stream) {
    return apply_levels(plan, instance, level_lo, level_hi, nrhs, q_up, p_down, beta, stream, false);
}

int kifmm_m2l_apply_levels_adjoint(kifmm_m2l_plan plan, int instance, int level_lo, int level_hi, int nrhs,
                                   const float* pbar_down, float* qbar_up, float beta, void* stream) {
    return apply_levels(plan, instance, level_lo, level_hi, nrhs, pbar_down, qbar_up, beta, stream, true);
}

int kifmm_m2l_apply_levels_host(kifmm_m2l_plan plan, int instance, int level_lo, int level_hi, int nrhs,
                                const float* q_up_host, float* p_down_host, float beta, void* stream) {
    if (!q_up_host || !p_down_host) {
        set_error("NULL host density pointer");
        return KIFMM_ERR_INVALID_ARG;
    }
    return apply_levels(plan, instance, level_lo, level_hi, nrhs, nullptr, nullptr, beta, stream, false, q_up_host,
                        p_down_host);
}

int kifmm_m2l_apply_dense(kifmm_m2l_plan plan, int instance, int level, int nrhs, const float* q_up, float* p_down,
                          float beta, void* stream) {
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
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    const int n = plan->n;
    if (!plan->K.ptr) {
        std::vector<float> hk((size_t)kOffsets * n * n);
        std::vector<double> kd((size_t)n * n);
        int offs[kOffsets][3];
        offsets316(offs);
        const std::vector<double> u = unit_surface(plan->prm.p);
        for (int k = 0; k < kOffsets; ++k) {
            unit_m2l_matrix(plan->prm.p, plan->prm.d, offs[k], u, kd.data(), kernel_kh(plan->prm));
            for (size_t i = 0; i < kd.size(); ++i) hk[(size_t)k * n * n + i] = (float)kd[i];
        }
        KIFMM_CUDA_TRY(plan->K.upload(hk.data(), hk.size()));
    }
    if (ls->n_boxes == 0) return KIFMM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long rows = (long)ls->n_boxes * nrhs;
    const float scale = (float)std::ldexp(1.0 / ls->r0, level);
    // p_down = beta p_down + s_l sum K q : scale the old values, then scatter-add
    if (beta == 0.f) {
        KIFMM_CUDA_TRY(launch_zero(p_down, rows * n, s));
    } else if (beta != 1.f) {
        KIFMM_CUDA_TRY(launch_scale(p_down, rows * n, beta, s));
    }
    TileSet* ts = nullptr;
    st = get_tiles(ls->fwd, nrhs, &ts);
    if (st != KIFMM_OK) return st;
    KIFMM_CUDA_TRY(launch_pairs_gemm_fp32(q_up, n, plan->K.ptr, n, n, p_down, n, ts->tiles.ptr, ts->n_tiles,
                                          ls->fwd.src.ptr, ls->fwd.dst.ptr, nrhs, scale, s));
    return KIFMM_OK;
}

int kifmm_m2l_apply_dense_tc(kifmm_m2l_plan plan, int instance, int level, int nrhs, const float* q_up,
                             float* p_down, float beta, void* stream) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (plan->prm.precision != KIFMM_PREC_F16X3 || plan->prm.kernel_id != KIFMM_KERNEL_LAPLACE) {
        set_error("the tensor-core dense M2L runs the f16x3 arithmetic of Laplace plans (KIFMM_PREC_F16X3)");
        return KIFMM_ERR_UNSUPPORTED;
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
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    const int n = plan->n, np = plan->n_pad;
    if (!plan->Kd.ptr) {
        // K_o as two FP16 pieces of tau K_o, tau the power of two that puts
        // max |K_o| in [2^13, 2^14); the core divides by tau in its output scale
        int offs[kOffsets][3];
        offsets316(offs);
        const std::vector<double> u = unit_surface(plan->prm.p);
        std::vector<double> kd((size_t)kOffsets * n * n);
        for (int k = 0; k < kOffsets; ++k)
            unit_m2l_matrix(plan->prm.p, plan->prm.d, offs[k], u, kd.data() + (size_t)k * n * n, 0.0);
        double kmax = 0;
        for (double v : kd) kmax = std::max(kmax, std::fabs(v));
        int e2 = 0;
        std::frexp(kmax > 0 ? kmax : 1.0, &e2);
        const double tau = std::ldexp(1.0, 14 - e2);
        const size_t per = (size_t)kOffsets * np * np;
        std::vector<uint16_t> h(per * 2, 0);
        for (int k = 0; k < kOffsets; ++k)
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) {
                    const double v = tau * kd[((size_t)k * n + a) * n + b];
                    const size_t e = ((size_t)k * np + a) * np + b;
                    h[e] = f16_bits_rn(v);
                    h[per + e] = f16_bits_rn(v - f16_bits_to_double(h[e]));
                }
        KIFMM_CUDA_TRY(plan->Kd.ensure(h.size()));
        KIFMM_CUDA_TRY(cudaMemcpy(plan->Kd.ptr, h.data(), h.size() * 2, cudaMemcpyHostToDevice));
        plan->dense_inv_scale = (float)(1.0 / tau);
    }
    if (ls->n_boxes == 0) return KIFMM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long rows = (long)ls->n_boxes * nrhs;
    if (rows + 1 > (long)INT32_MAX / 2) {
        set_error("too many box rows");
        return KIFMM_ERR_INVALID_ARG;
    }
    const long pstride = (rows + 1) * np;
    KIFMM_CUDA_TRY(plan->dq.ensure((size_t)2 * pstride));
    KIFMM_CUDA_TRY(plan->dq_inv.ensure((size_t)rows + 1));
    KIFMM_CUDA_TRY(plan->dp.ensure((size_t)rows * np));
    // operand: the q_up rows as scaled FP16 pieces (zero row last), output zeroed
    KIFMM_CUDA_TRY(launch_split_rows_f16_scaled(q_up, (int)rows, n, n, np, reinterpret_cast<__half*>(plan->dq.ptr),
                                                pstride, plan->dq_inv.ptr, s));
    for (int pc = 0; pc < 2; ++pc)
        KIFMM_CUDA_TRY(cudaMemsetAsync(plan->dq.ptr + pc * pstride + rows * np, 0, np * sizeof(__nv_bfloat16), s));
    KIFMM_CUDA_TRY(cudaMemsetAsync(plan->dq_inv.ptr + rows, 0, sizeof(float), s));
    KIFMM_CUDA_TRY(launch_zero(plan->dp.ptr, rows * np, s));
    TileSet* ts = nullptr;
    st = get_tiles(ls->fwd, nrhs, &ts);
    if (st != KIFMM_OK) return st;
    UmmaArgs a{};
    a.A = plan->dq.ptr;
    a.a_piece_stride = pstride;
    a.kdim = np;
    a.B = plan->Kd.ptr;
    a.b_groups = kOffsets;
    a.ndim = np;
    a.n_chunk = ((np / 2 + 15) / 16) * 16;
    a.core_bres = 1;
    a.core_drain = 3;
    a.contiguous = 1;
    a.row_src = ts->row_src.ptr;
    a.row_dst = ts->row_dst.ptr;
    a.tile_k = ts->tile_k.ptr;
    a.n_tiles = ts->n_tiles;
    a.nrhs = nrhs;
    a.zero_row = (int)rows;
    a.level_scale[0] = (float)std::ldexp(1.0 / ls->r0, level) * plan->dense_inv_scale;
    a.D = plan->dp.ptr;
    a.ldd = np;
    a.n_products = 3;
    a.hilo = 1;
    a.f16 = 1;
    a.row_scale = plan->dq_inv.ptr;
    a.error_flag = plan->err_flag.ptr;
    a.wait_ns = plan->core_wait_ns;
    KIFMM_CUDA_TRY(launch_umma(A_GATHER, E_RED, a, plan->num_sms, s));
    // p_down = beta p_down + the first n columns
    KIFMM_CUDA_TRY(launch_copy_rows(p_down, n, plan->dp.ptr, np, rows, n, beta, s));
    return KIFMM_OK;
}

}  // extern "C"
