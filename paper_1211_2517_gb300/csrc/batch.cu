// kifmm_m2l_apply_batch: the compressed M2L of many FMM instances (uneven
// sizes, several operators p, several right-hand-side counts) as one
// grouped batch.
//
// Items are grouped by plan (one operator each).  Per plan, persistent
// launches cover every item of the group:
//   compression  one rows-mode launch over the items' rows (a segment table
//                maps row tiles to each item's input buffer),
//   core         one offset-ordered tile list merged over all items and
//                levels (row tables in a batch-wide row space, a scale table
//                with s_l of every (item, level)),
//   expansion    one rows-mode launch writing each item's output buffer.
// When every plan's core runs on the staged-epilogue kernel (1 or 2 pieces,
// the same arithmetic, no stage 2, at most 8 plans), the cores of all plans
// are one launch: each plan is a group with its own K~_o, rank and tile
// list, and the launch's CTAs share the summed work.
// With use_graph the whole batch is captured once into a CUDA graph, cached
// by the batch's signature, and replayed by later calls.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "kifmm_internal.h"
#include "plan.h"

using namespace kifmm;

namespace {

struct PlanGroup {
    kifmm_m2l_plan plan = nullptr;
    std::vector<int> items;       // indices into the batch
    std::vector<long> row_base;   // per item: first row in the group's row space
    long rows_total = 0;
    int in_tiles = 0;             // virtual row tiles of the compression / expansion
    DevBuf<RowSeg> seg_in, seg_out;
    DevBuf<float> scales;
    TileSet tiles;
    DevBuf<__nv_bfloat16> qb;     // pieces of q~ [pieces][rows_total + 1][r_pad]
    DevBuf<__nv_bfloat16> sp;     // BF16 pieces of the compression / expansion inputs
    DevBuf<float> pt;             // p~ [rows_total][r_pad]
    DevBuf<float> qs;             // f16x3: inverse row factors of the q~ pieces [rows_total + 1]
};

struct BatchEntry {
    std::vector<std::unique_ptr<PlanGroup>> groups;
    bool one_core = false;  // the cores of all groups in one grouped launch
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    // the groups' launch chains run side by side on these streams, forked
    // from and joined back into the caller's (or the capture) stream
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    ~BatchEntry() {
        if (exec) cudaGraphExecDestroy(exec);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        for (auto x : side) cudaStreamDestroy(x);
        for (auto x : ev) cudaEventDestroy(x);
    }
};

std::mutex g_batch_mutex;
std::map<std::string, std::unique_ptr<BatchEntry>> g_batches;

std::string signature(int n, const kifmm_m2l_batch_item* it) {
    std::string sig;
    for (int i = 0; i < n; ++i) {
        const kifmm_m2l_batch_item& x = it[i];
        char buf[256];
        uint32_t b;
        std::memcpy(&b, &x.beta, 4);
        std::snprintf(buf, sizeof(buf), "%p/%d/%d/%d/%d/%p/%p/%08x;", (void*)x.plan, x.instance, x.level_lo,
                      x.level_hi, x.nrhs, (const void*)x.q_up, (void*)x.p_down, b);
        sig += buf;
    }
    return sig;
}

// Merged tiles and row tables of all items of one plan.
int build_group(PlanGroup& g, const kifmm_m2l_batch_item* items) {
    kifmm_m2l_plan plan = g.plan;
    struct ItemPairs {
        MultiState* ms;
        int nrhs;
        long base;
        int scale_base;
    };
    std::vector<ItemPairs> ip;
    std::vector<float> scales;
    std::vector<RowSeg> seg_in, seg_out;
    long rows = 0;
    int tiles_so_far = 0;
    for (int idx : g.items) {
        const kifmm_m2l_batch_item& x = items[idx];
        MultiState* ms = nullptr;
        int st = get_multi_state(plan, x.instance, x.level_lo, x.level_hi, false, &ms);
        if (st != KIFMM_OK) return st;
        ItemPairs p{ms, x.nrhs, rows, (int)scales.size()};
        for (int l = x.level_lo; l <= x.level_hi; ++l)
            scales.push_back((float)(std::ldexp(1.0 / find_level(plan, x.instance, l)->r0, l) * plan->out_inv_scale()));
        const long item_rows = ms->total_boxes * x.nrhs;
        g.row_base.push_back(rows);
        RowSeg si{x.q_up, nullptr, (int)item_rows, tiles_so_far, (int)rows, 1.0f, 0.0f};
        seg_in.push_back(si);
        seg_out.push_back({nullptr, x.p_down, (int)item_rows, tiles_so_far, 0, 1.0f, x.beta});
        tiles_so_far += (int)((item_rows + kTileRows - 1) / kTileRows);
        rows += item_rows;
        ip.push_back(p);
    }
    if (scales.size() >= 65536 || rows + 1 > (long)INT32_MAX / 2) {
        set_error("batch too large (levels or rows)");
        return KIFMM_ERR_INVALID_ARG;
    }
    g.rows_total = rows;
    g.in_tiles = tiles_so_far;
    // expansion reads p~ rows [base, base + rows) of the group's scratch
    KIFMM_CUDA_TRY(g.pt.ensure((size_t)std::max<long>(rows, 1) * plan->rp));
    KIFMM_CUDA_TRY(g.qb.ensure((size_t)(rows + 1) * plan->rp * std::max(plan->pieces, 1)));
    KIFMM_CUDA_TRY(g.sp.ensure(split_elems(plan, tiles_so_far)));
    if (plan->prm.precision == KIFMM_PREC_F16X3) {
        KIFMM_CUDA_TRY(g.qs.ensure((size_t)rows + 1));
    }
    for (size_t i = 0; i < seg_out.size(); ++i) seg_out[i].Af = g.pt.ptr + ip[i].base * plan->rp;
    KIFMM_CUDA_TRY(g.seg_in.upload(seg_in.data(), seg_in.size()));
    KIFMM_CUDA_TRY(g.seg_out.upload(seg_out.data(), seg_out.size()));
    KIFMM_CUDA_TRY(g.scales.upload(scales.data(), scales.size()));
    // merged tile list: offset-major over all items and levels
    std::vector<Tile> tl;
    std::vector<int> rs, rd, tk;
    for (int k = 0; k < kOffsets; ++k)
        for (const ItemPairs& p : ip)
            for (const auto& grp : p.ms->groups) {
                if (grp.k != k) continue;
                const int64_t nrow = grp.count * p.nrhs;
                for (int64_t r0 = 0; r0 < nrow; r0 += kTileRows) {
                    const int nr = (int)std::min<int64_t>(kTileRows, nrow - r0);
                    const int code = k | ((p.scale_base + grp.level_idx) << 16);
                    tl.push_back({code, (int)grp.begin, (int)r0, nr});
                    tk.push_back(code);
                    for (int r = 0; r < kTileRows; ++r) {
                        int s = -1, d = -1;
                        if (r < nr) {
                            const int64_t gr = r0 + r;
                            const int64_t pr = grp.begin + gr / p.nrhs;
                            const int64_t rhs = gr % p.nrhs;
                            s = (int)(p.base + p.ms->h_src[pr] * (int64_t)p.nrhs + rhs);
                            d = (int)(p.base + p.ms->h_dst[pr] * (int64_t)p.nrhs + rhs);
                        }
                        rs.push_back(s);
                        rd.push_back(d);
                    }
                }
            }
    KIFMM_CUDA_TRY(g.tiles.tiles.upload(tl.data(), tl.size()));
    KIFMM_CUDA_TRY(g.tiles.row_src.upload(rs.data(), rs.size()));
    KIFMM_CUDA_TRY(g.tiles.row_dst.upload(rd.data(), rd.size()));
    KIFMM_CUDA_TRY(g.tiles.tile_k.upload(tk.data(), tk.size()));
    g.tiles.n_tiles = (int)tl.size();
    return KIFMM_OK;
}

// Split and compression of one plan group (for f16x3 the GEMM writes the
// scaled FP16 pieces itself): the core's q~ pieces, p~ cleared.
int enqueue_compress(PlanGroup& g, cudaStream_t s) {
    kifmm_m2l_plan plan = g.plan;
    const int rp = plan->rp;
    const bool f16 = plan->prm.precision == KIFMM_PREC_F16X3;
    const long piece_stride = (g.rows_total + 1) * rp;
    {
        const int st = run_compress(plan, nullptr, 0, g.seg_in.ptr, (int)g.items.size(), g.in_tiles, g.sp.ptr,
                                    g.qb.ptr, piece_stride, nullptr, g.pt.ptr, s, f16 ? g.qs.ptr : nullptr);
        if (st != KIFMM_OK) return st;
    }
    if (f16) {
        const int st = zero_core_operand_row_f16(plan, g.rows_total, g.qb.ptr, piece_stride, g.qs.ptr, s);
        if (st != KIFMM_OK) return st;
    } else {
        for (int pc = 0; pc < plan->pieces; ++pc)
            KIFMM_CUDA_TRY(cudaMemsetAsync(g.qb.ptr + pc * piece_stride + g.rows_total * rp, 0,
                                           rp * sizeof(__nv_bfloat16), s));
    }
    return KIFMM_OK;
}

// The core operands of one plan group.
UmmaArgs core_args(PlanGroup& g) {
    kifmm_m2l_plan plan = g.plan;
    const int rp = plan->rp;
    const bool f16 = plan->prm.precision == KIFMM_PREC_F16X3;
    const long piece_stride = (g.rows_total + 1) * rp;
    UmmaArgs a{};
    {
        a.A = g.qb.ptr;
        a.a_piece_stride = piece_stride;
        a.kdim = rp;
        a.B = plan->Cb.ptr;
        a.b_groups = kOffsets;
        a.ndim = rp;
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
        a.row_src = g.tiles.row_src.ptr;
        a.row_dst = g.tiles.row_dst.ptr;
        a.tile_k = g.tiles.tile_k.ptr;
        a.n_tiles = g.tiles.n_tiles;
        a.nrhs = 1;
        a.zero_row = (int)g.rows_total;
        a.scale_table = g.scales.ptr;
        a.D = g.pt.ptr;
        a.ldd = rp;
        a.n_products = plan->products;
        a.hilo = plan->core_hilo;
        a.f16 = f16 ? 1 : 0;
        a.row_scale = f16 ? g.qs.ptr : nullptr;
        a.error_flag = plan->err_flag.ptr;
        a.wait_ns = plan->core_wait_ns;
    }
    return a;
}

int enqueue_expand(PlanGroup& g, cudaStream_t s) {
    return run_expand(g.plan, nullptr, 0, g.seg_out.ptr, (int)g.items.size(), g.in_tiles, g.sp.ptr, nullptr, 1.0f,
                      0.0f, s);
}

// Whether the cores of all groups can be one grouped launch.
bool one_core_launch(const BatchEntry& e) {
    if (e.groups.empty() || e.groups.size() > 8) return false;
    const kifmm_m2l_plan p0 = e.groups[0]->plan;
    for (const auto& g : e.groups) {
        const kifmm_m2l_plan p = g->plan;
        if (p->s2_on || (p->products != 1 && p->products != 3) || p->products != p0->products ||
            p->prm.precision != p0->prm.precision || p->num_sms != p0->num_sms || p->rp % 16 != 0)
            return false;
    }
    return true;
}

// Fork: every side stream waits for the work already on s (event k).
int fork_sides(BatchEntry& e, cudaStream_t s, int k) {
    KIFMM_CUDA_TRY(cudaEventRecord(e.ev[k], s));
    for (auto x : e.side) KIFMM_CUDA_TRY(cudaStreamWaitEvent(x, e.ev[k], 0));
    return KIFMM_OK;
}

// Join: s waits for everything on the side streams (events k, k + 1, ...).
int join_sides(BatchEntry& e, cudaStream_t s, int k) {
    for (size_t i = 0; i < e.side.size(); ++i) {
        KIFMM_CUDA_TRY(cudaEventRecord(e.ev[k + i], e.side[i]));
        KIFMM_CUDA_TRY(cudaStreamWaitEvent(s, e.ev[k + i], 0));
    }
    return KIFMM_OK;
}

int enqueue_all(BatchEntry& e, cudaStream_t s) {
    // group g's launches go to side stream g % k: the groups' small
    // compressions and expansions (and, without a grouped core, their whole
    // chains) overlap instead of queueing behind one another
    const size_t k = std::min<size_t>(e.groups.size(), 4);
    while (e.side.size() < k) {
        cudaStream_t x = nullptr;
        KIFMM_CUDA_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        e.side.push_back(x);
    }
    while (e.ev.size() < 3 * k + 2) {
        cudaEvent_t x = nullptr;
        KIFMM_CUDA_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        e.ev.push_back(x);
    }
    int st = fork_sides(e, s, 0);
    if (st != KIFMM_OK) return st;
    if (!e.one_core) {
        for (size_t i = 0; i < e.groups.size(); ++i) {
            PlanGroup& g = *e.groups[i];
            cudaStream_t x = e.side[i % k];
            if (g.rows_total == 0) continue;
            st = enqueue_compress(g, x);
            if (st != KIFMM_OK) return st;
            const UmmaArgs a = core_args(g);
            KIFMM_CUDA_TRY(launch_umma(A_GATHER, E_RED, a, g.plan->num_sms, x));
            st = enqueue_expand(g, x);
            if (st != KIFMM_OK) return st;
        }
        return join_sides(e, s, 1);
    }
    std::vector<UmmaArgs> args;
    for (size_t i = 0; i < e.groups.size(); ++i) {
        PlanGroup& g = *e.groups[i];
        if (g.rows_total == 0) continue;
        st = enqueue_compress(g, e.side[i % k]);
        if (st != KIFMM_OK) return st;
        args.push_back(core_args(g));
    }
    st = join_sides(e, s, 1);
    if (st != KIFMM_OK) return st;
    if (args.empty()) return KIFMM_OK;
    int dev = 0, max_smem = 0;
    KIFMM_CUDA_TRY(cudaGetDevice(&dev));
    KIFMM_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    KIFMM_CUDA_TRY(launch_core_stage_grouped(args.data(), (int)args.size(), e.groups[0]->plan->num_sms, max_smem,
                                             dev, s));
    st = fork_sides(e, s, 1 + k);
    if (st != KIFMM_OK) return st;
    for (size_t i = 0; i < e.groups.size(); ++i) {
        PlanGroup& g = *e.groups[i];
        if (g.rows_total == 0) continue;
        st = enqueue_expand(g, e.side[i % k]);
        if (st != KIFMM_OK) return st;
    }
    return join_sides(e, s, 2 + k);
}

}  // namespace

namespace kifmm {

// Drop cached batches that use `plan` (called when the plan is destroyed).
void forget_batches_of(kifmm_m2l_plan plan) {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        bool uses = false;
        for (auto& g : it->second->groups) uses = uses || g->plan == plan;
        if (uses) it = g_batches.erase(it);
        else ++it;
    }
}

}  // namespace kifmm

extern "C" int kifmm_m2l_apply_batch(int n_items, const kifmm_m2l_batch_item* items, int use_graph, void* stream) {
    if (n_items < 0 || (n_items > 0 && !items)) {
        set_error("invalid batch");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (n_items == 0) return KIFMM_OK;
    // validate every item
    for (int i = 0; i < n_items; ++i) {
        const kifmm_m2l_batch_item& x = items[i];
        if (!x.plan) {
            set_error("batch item " + std::to_string(i) + ": plan is NULL");
            return KIFMM_ERR_INVALID_ARG;
        }
        if (x.plan->prm.precision == KIFMM_PREC_FP32) {
            set_error("batch item " + std::to_string(i) + ": batches run the tensor-core modes (not KIFMM_PREC_FP32)");
            return KIFMM_ERR_UNSUPPORTED;
        }
        if (x.nrhs < 1 || x.level_lo < 0 || x.level_hi < x.level_lo || x.level_hi - x.level_lo >= 32) {
            set_error("batch item " + std::to_string(i) + ": invalid nrhs or level range");
            return KIFMM_ERR_INVALID_ARG;
        }
        for (int l = x.level_lo; l <= x.level_hi; ++l)
            if (!find_level(x.plan, x.instance, l)) {
                set_error("batch item " + std::to_string(i) + ": level " + std::to_string(l) + " not registered");
                return KIFMM_ERR_STATE;
            }
        if ((reinterpret_cast<uintptr_t>(x.q_up) & 15) || (reinterpret_cast<uintptr_t>(x.p_down) & 15) ||
            !x.q_up || !x.p_down) {
            set_error("batch item " + std::to_string(i) + ": density pointers must be non-NULL and 16-byte aligned");
            return KIFMM_ERR_INVALID_ARG;
        }
        int st = check_device(x.plan);
        if (st != KIFMM_OK) return st;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    const std::string sig = signature(n_items, items);
    auto it = g_batches.find(sig);
    BatchEntry* e = nullptr;
    if (it == g_batches.end()) {
        auto ne = std::make_unique<BatchEntry>();
        std::map<kifmm_m2l_plan, PlanGroup*> by_plan;
        for (int i = 0; i < n_items; ++i) {
            auto f = by_plan.find(items[i].plan);
            if (f == by_plan.end()) {
                ne->groups.push_back(std::make_unique<PlanGroup>());
                ne->groups.back()->plan = items[i].plan;
                f = by_plan.emplace(items[i].plan, ne->groups.back().get()).first;
            }
            f->second->items.push_back(i);
        }
        for (auto& g : ne->groups) {
            int st = build_group(*g, items);
            if (st != KIFMM_OK) return st;
        }
        ne->one_core = one_core_launch(*ne);
        if (g_batches.size() >= 16) g_batches.clear();
        e = ne.get();
        g_batches[sig] = std::move(ne);
    } else {
        e = it->second.get();
    }
    if (!use_graph) return enqueue_all(*e, s);
    if (!e->exec) {
        // one eager pass first: every lazy host-side setup (tensor maps, kernel
        // attributes) is done before capture
        int st = enqueue_all(*e, s);
        if (st != KIFMM_OK) return st;
        KIFMM_CUDA_TRY(cudaStreamCreateWithFlags(&e->capture_stream, cudaStreamNonBlocking));
        KIFMM_CUDA_TRY(cudaStreamBeginCapture(e->capture_stream, cudaStreamCaptureModeThreadLocal));
        st = enqueue_all(*e, e->capture_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(e->capture_stream, &graph);
        if (st != KIFMM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        KIFMM_CUDA_TRY(ce);
        ce = cudaGraphInstantiate(&e->exec, graph, 0);
        cudaGraphDestroy(graph);
        KIFMM_CUDA_TRY(ce);
        return KIFMM_OK;  // the eager pass produced this call's result
    }
    KIFMM_CUDA_TRY(cudaGraphLaunch(e->exec, s));
    return KIFMM_OK;
}
