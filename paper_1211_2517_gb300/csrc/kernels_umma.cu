// tcgen05 (5th-generation tensor core) kernels of the compressed M2L.
//
// One kernel template computes the three products of Eq. (14) restricted
// to M2L, each as a split-BF16 GEMM with FP32 accumulation in tensor memory:
//
//   compress  q~ = R~^T q        A = FP32 rows of q, split to BF16 pieces
//                                in shared memory; output written as the
//                                BF16 pieces the core consumes (E_SPLIT)
//   core      p~^t += K~_o q~^s  one dense GEMM per offset o over every box
//                                pair sharing it: A gathers source rows of
//                                q~, B = K~_o, each output row is reduced
//                                into its target's p~ row (E_RED)
//   expand    p = s_l U~ p~ (+ beta p)                            (E_STORE)
//
// Split precision: x = x_0 + x_1 + x_2 with BF16 pieces; a product keeps
// the piece products (i, j) of order <= 2^-16 (6 of them for 3 pieces, 3
// for 2, 1 for 1).  With `hilo`, the (0,0) product accumulates in its own
// TMEM accumulator and the small ones in another, so the large terms are
// rounded once per 16-element MMA step instead of once per product.
//
// Warp roles of a persistent CTA (one per SM, 384 threads):
//   warps 0-3  epilogue: TMEM -> registers -> per-warp shared-memory
//              transpose -> coalesced 16-byte global reductions / stores
//   warps 4-10 producers: A tiles into 64B-swizzled shared memory (cp.async
//              gather of BF16 rows, one ring slot per warp; or, in the rows
//              modes, warps 4-7 load FP32 rows and split them in registers);
//              a producer thread also TMA-loads the B tiles
//   warp 11    TMEM allocation and the single MMA-issuing thread
// Stages cycle through full/empty mbarriers; two TMEM accumulator slots
// (when they fit in 512 columns) overlap the epilogue of one work item
// with the MMAs of the next.
//
// Every mbarrier wait is bounded (about two seconds of %globaltimer); on
// timeout the kernel raises a device error flag, every role stops, copies in
// flight are waited for (bounded), and TMEM is freed before exit.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cuda_bf16.h>

#include <cstdint>
#include <map>
#include <type_traits>
#include <mutex>

#include "kernels.h"
#include "kifmm_m2l.h"
#include "umma_ptx.h"

namespace kifmm {

namespace {

using namespace ptx;

constexpr int kEpiWarps = 4, kProdWarps = 7;
constexpr int kRowsProdWarps = 4;  // producer warps of the rows modes (128 threads, one per tile row)
constexpr int kThreads = (kEpiWarps + kProdWarps + 1) * 32;  // 384
// K elements per pipeline stage (64-byte rows, 64-byte swizzle).  The
// templates also support 16 (32-byte rows, 32-byte swizzle); measured on the
// core, twice the stages of half the size cost more than they hide.
__host__ __device__ constexpr int chunk_of(int) { return 32; }
constexpr int kCBoxRows = 64;           // rows per TMA box of K~_o

struct Smem {
    // barriers live at the start of dynamic shared memory
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t tmem_full[2];   // whole-item accumulator slots (core), lo slots (rows modes)
    uint64_t tmem_empty[2];
    uint64_t part_full[2];   // rows modes: per K-chunk partial of the (0,0) product
    uint64_t part_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    volatile int abort_flag;
    unsigned long long wait_ns;  // bound of every mbarrier wait of this launch
};

struct Layout {
    int stages, na, nc, c_rows_alloc, n_acc, acc_cols, n_items, n_chunks, kc_count;
    int prod_warps;  // A_GATHER: producer warps in use; divides `stages`
    int drain;       // A_GATHER: K-chunks per partial drained by 8 epilogue warps (0: no drain; see the epilogue)
    int dhilo;       // drained partials keep the (0,0) product in its own half of the slot (2 N columns per slot)
    int a_tma;       // identity-row gathers: the A pieces by TMA (amap) instead of per-lane cp.async
    int a_rows;      // rows of one A piece in amap
    uint32_t a_bytes, c_bytes, stage_bytes, trans_off;
};


constexpr int kTransStride = 36;  // floats per row of the epilogue transpose buffer (16-byte rows, no bank conflicts)
constexpr int kMaxRowsChunk = 64; // N per work item of the rows modes (partial sums live in registers)
constexpr int kPartChunks = 2;    // rows modes: K-chunks per drained partial of the (0,0) product

// x (low half) and y (high half) rounded to nearest-even BF16 and packed
__device__ __forceinline__ uint32_t cvt_bf16x2(float x, float y) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(y), "f"(x));
    return d;
}

// Split x and y into `np` BF16 pieces each (round to nearest at each step,
// x_i + x_(i+1) + ... reproduces x to 8 np bits); piece i of both is h[i]
// (x low half, y high half); pieces past np are zero.  The BF16 values
// convert back to FP32 exactly by placing their bits in the high half.
__device__ __forceinline__ void split3x2(float x, float y, uint32_t (&h)[3], int np) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i < np) {
            h[i] = cvt_bf16x2(x, y);
            x -= __uint_as_float(h[i] << 16);
            y -= __uint_as_float(h[i] & 0xFFFF0000u);
        } else {
            h[i] = 0u;
        }
    }
}

template <int AMODE, int EMODE>
__global__ void __launch_bounds__(kThreads, 1)
    umma_kernel(const __grid_constant__ CUtensorMap bmap, const __grid_constant__ CUtensorMap amap, const UmmaArgs args,
                const Layout L) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    uint8_t* smem_raw = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    Smem* sm = reinterpret_cast<Smem*>(smem_raw);
    uint8_t* stage_base = smem_raw + 1024;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int S = L.stages;
    constexpr int CH = chunk_of(AMODE);  // K elements per stage
    constexpr int RB = CH * 2;           // bytes per shared-memory row
    const int KC = L.kc_count;
    const int n_chunks = L.n_chunks;
    // Work items of this CTA: every gridDim.x-th item (consecutive CTAs take
    // consecutive offset-ordered tiles, which share K~_o in L2), or, for the
    // core when `contiguous` is set, a contiguous run of the tile list
    const bool contig = AMODE == A_GATHER && args.contiguous;
    const int i_beg = contig ? (int)((long)L.n_items * blockIdx.x / gridDim.x) : (int)blockIdx.x;
    const int i_end = contig ? (int)((long)L.n_items * (blockIdx.x + 1) / gridDim.x) : L.n_items;
    const int i_step = contig ? 1 : (int)gridDim.x;
    // rows modes: segment of a virtual row tile (binary search)
    auto find_seg = [&](int tt) -> int {
        int lo = 0, hi = args.n_segs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (args.segs[mid].tile_begin <= tt) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&sm->full[s], (AMODE == A_GATHER ? 32 : kRowsProdWarps * 32) + 1);
            mbar_init(&sm->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sm->tmem_full[a], 1);
            mbar_init(&sm->tmem_empty[a], kEpiWarps * 32);
            mbar_init(&sm->part_full[a], 1);
            mbar_init(&sm->part_empty[a], (AMODE == A_GATHER && L.drain ? 2 : 1) * kEpiWarps * 32);
        }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        sm->wait_ns = args.wait_ns ? args.wait_ns : kWaitNs;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kEpiWarps + kProdWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&sm->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;

    auto a_smem = [&](int s, int piece) -> uint32_t {
        return smem_u32(stage_base + (size_t)s * L.stage_bytes + (size_t)piece * L.a_bytes);
    };
    auto c_smem = [&](int s, int piece) -> uint32_t {
        return smem_u32(stage_base + (size_t)s * L.stage_bytes + (size_t)L.na * L.a_bytes +
                        (size_t)piece * L.c_bytes);
    };
    // work item -> (tile or row tile, N chunk)
    auto item_tile = [&](int item) { return item / n_chunks; };
    auto item_n0 = [&](int item) { return (item % n_chunks) * args.n_chunk; };
    auto item_nthis = [&](int item) { return min(args.n_chunk, args.ndim - item_n0(item)); };

    // drain mode: warps 7-10 (idle producers when at most 3 stages) are a
    // second epilogue group
    const bool epi2 = AMODE == A_GATHER && L.drain && warp >= kEpiWarps + 3 && warp < kEpiWarps + kProdWarps;
    if (warp >= kEpiWarps && warp < kEpiWarps + kProdWarps && !epi2) {
        // ================= producers =================
        const int v = threadIdx.x - kEpiWarps * 32;  // 0..127
        const bool tma_thread = AMODE == A_GATHER ? (lane == 0) : (v == 0);
        int it = 0;
        bool ok = true;
        int group = 0;  // B group (offset) of the current item, A_GATHER only
        auto issue_b = [&](int s, int item, int kc) {
            mbar_arrive_expect_tx(&sm->full[s], (uint32_t)L.nc * L.c_rows_alloc * RB);
            for (int pc = 0; pc < L.nc; ++pc) {
                const int row_base = (pc * args.b_groups + group) * args.ndim + item_n0(item);
                for (int rb = 0; rb < L.c_rows_alloc; rb += kCBoxRows)
                    tma_load_2d(c_smem(s, pc) + rb * RB, &bmap, kc * CH, row_base + rb, &sm->full[s]);
            }
        };
        if (AMODE == A_GATHER) {
            // Stage it belongs to producer warp it % P (P = L.prod_warps <= S
            // ring slots).  That warp gathers all 128 rows of the stage (lane
            // l copies 16-byte chunk l % CPR of rows l / CPR + RPI i: one
            // instruction covers RPI rows of CH * 2 contiguous bytes); every
            // lane's copies arrive on the stage's full barrier when they land,
            // so a warp has as many stages in flight as the ring allows.  A
            // warp waiting on a slot's empty barrier is at most one phase
            // ahead of it: its previous stage (it - P) already waited for the
            // consumption of it - P - S, which is at or after it - 2 S when
            // P <= S.
            const int P = L.prod_warps;
            constexpr int CPR = CH / 8;          // 16-byte chunks per row and stage
            constexpr int RPI = 32 / CPR;        // rows per warp instruction
            constexpr int NR = kTileM / RPI;     // rows per lane
            const int pw = warp - kEpiWarps, cch = lane % CPR, rl = lane / CPR;
            // row indices of this and of the next item (prefetched while the
            // current one streams: no dependent load at an item's start)
            int srow[NR], nrow[NR], ngroup = 0;
            auto load_rows = [&](int item) {
                const int t = item_tile(item);
                if (args.row_identity) {
#pragma unroll
                    for (int i = 0; i < NR; ++i) nrow[i] = t * kTileM + rl + RPI * i;
                    ngroup = 0;
                } else {
#pragma unroll
                    for (int i = 0; i < NR; ++i) nrow[i] = __ldg(args.row_src + (long)t * kTileM + rl + RPI * i);
                    ngroup = __ldg(args.tile_k + t) & 0xFFFF;
                }
            };
            if (pw < P && i_beg < i_end) load_rows(i_beg);
            for (int item = i_beg; item < i_end && ok; item += i_step) {
                if (pw < P) {
#pragma unroll
                    for (int i = 0; i < NR; ++i) srow[i] = nrow[i] < 0 ? args.zero_row : nrow[i];
                    group = ngroup;
                    if (item + i_step < i_end) load_rows(item + i_step);
                }
                for (int kc = 0; kc < KC; ++kc, ++it) {
                    if (it % P != pw) continue;
                    const int s = it % S;
                    const uint32_t ph = (uint32_t)(it / S) & 1u;
                    if (!mbar_wait(&sm->empty[s], ph ^ 1u, sm, args.error_flag)) {
                        ok = false;
                        break;
                    }
                    if (L.a_tma) {
                        // identity rows: the tile's 128 rows of every piece as
                        // one TMA box each (columns past kdim read as zero); lane
                        // 0 arrives twice (A and B bytes), the other lanes once
                        if (lane == 0) {
                            mbar_arrive_expect_tx(&sm->full[s], (uint32_t)L.na * L.a_bytes);
                            const int t = item_tile(item);
                            for (int pc = 0; pc < L.na; ++pc)
                                tma_load_2d(a_smem(s, pc), &amap, kc * CH, pc * L.a_rows + t * kTileM, &sm->full[s]);
                            issue_b(s, item, kc);
                        } else {
                            mbar_arrive(&sm->full[s]);
                        }
                        continue;
                    }
                    const int col = kc * CH + cch * 8;
                    const uint32_t bytes = col < args.kdim ? 16u : 0u;
                    const int colc = col < args.kdim ? col : 0;
                    for (int pc = 0; pc < L.na; ++pc) {
                        const __nv_bfloat16* base = args.A + pc * args.a_piece_stride + colc;
                        const uint32_t sbase = a_smem(s, pc);
#pragma unroll
                        for (int i = 0; i < NR; ++i)
                            cp_async16(sbase + swz<CH>(rl + RPI * i, cch), base + (long)srow[i] * args.kdim, bytes);
                    }
                    if (lane == 0) issue_b(s, item, kc);
                    // the stage is full once every lane's copies land; the warp
                    // moves on without waiting (the MMA thread fences the
                    // generic-proxy writes before its tensor-core reads)
                    cp_async_mbar_arrive(&sm->full[s]);
                }
            }
            cp_async_wait_0();
        } else if (v < kRowsProdWarps * 32) {
            // FP32 rows: thread v loads float4 f = v + 128 i (i = 0..7) of the
            // 128 x 32 tile, row f / 8, columns 4 (f % 8) .. +3 (a warp reads
            // 4 rows x 128 contiguous bytes), splits them into BF16 pieces and
            // stores them swizzled.
            float4 buf[8];
            auto load = [&](int item, int kc) {
                const int tt = item_tile(item);
                const float* Af = args.Af;
                long m0 = (long)tt * kTileM, mrows = args.m_rows;
                if (args.n_segs > 0) {
                    const RowSeg sg = args.segs[find_seg(tt)];
                    Af = sg.Af;
                    m0 = (long)(tt - sg.tile_begin) * kTileM;
                    mrows = sg.m_rows;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int f = v + 128 * i;
                    const long row = m0 + f / 8;
                    const int col = kc * CH + 4 * (f % 8);
                    buf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (row < mrows && col < args.k_valid)
                        buf[i] = __ldg(reinterpret_cast<const float4*>(Af + row * args.lda + col));
                }
            };
            int item = blockIdx.x, kc = 0;
            if (item < L.n_items) load(item, 0);
            while (item < L.n_items && ok) {
                const int s = it % S;
                const uint32_t ph = (uint32_t)(it / S) & 1u;
                if (!mbar_wait(&sm->empty[s], ph ^ 1u, sm, args.error_flag)) {
                    ok = false;
                    break;
                }
                if (tma_thread) issue_b(s, item, kc);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int f = v + 128 * i;
                    const int row = f / 8, c4 = f % 8;
                    uint32_t lo[3], hi[3];
                    split3x2(buf[i].x, buf[i].y, lo, L.na);
                    split3x2(buf[i].z, buf[i].w, hi, L.na);
                    const uint32_t off = swz<CH>(row, c4 >> 1) + (c4 & 1) * 8;
#pragma unroll
                    for (int pc = 0; pc < 3; ++pc) {
                        if (pc >= L.na) break;
                        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a_smem(s, pc) + off), "r"(lo[pc]),
                                     "r"(hi[pc])
                                     : "memory");
                    }
                }
                fence_proxy_async();
                mbar_arrive(&sm->full[s]);
                ++it;
                if (++kc == KC) {
                    kc = 0;
                    item += gridDim.x;
                }
                if (item < L.n_items) load(item, kc);  // in flight while waiting for the next slot
            }
        }
        if (!ok && tma_thread) {
            const unsigned long long t0 = global_ns();
            while (global_ns() - t0 < 1000000ull) {
            }
        }
    } else if (warp == kEpiWarps + kProdWarps) {
        // ================= MMA issuer =================
        // Core (A_GATHER): one accumulator slot per work item (hi and, with
        // hilo, lo side by side), double-buffered when two fit.
        // Rows modes: the (0,0) product of every kPartChunks K-chunks goes to
        // one of two ping-pong partial slots that the epilogue drains into
        // FP32 registers (no accumulator chain is longer than 4 MMA steps);
        // the small products accumulate over the item in a lo slot.
        // One thread issues at the tensor pipe's own rate only if its
        // instruction stream between MMAs is a few integer adds: the product
        // table is a compile-time constant (NP = n_products), descriptors are
        // advanced by adding 16-byte offsets to one base descriptor, and the
        // ring position is kept incrementally.
        if (lane == 0) {
            auto run = [&](auto np_tag) {
                constexpr int NP = decltype(np_tag)::value;
                constexpr int P0 = 6 - NP;
                const uint64_t desc0 = umma_desc<CH>(smem_u32(stage_base));
                const uint32_t stage_u = L.stage_bytes >> 4, a_u = L.a_bytes >> 4, c_u = L.c_bytes >> 4;
                const uint32_t c0_u = (uint32_t)L.na * a_u;
                // drain (core): every product into one per-K-chunk partial
                const bool drain = AMODE == A_GATHER && L.drain;
                const int group_max = drain && args.mma_pair > 1 ? (args.mma_pair < S - 1 ? args.mma_pair : S - 1) : 1;
                const bool split_lo = AMODE == A_ROWS || (args.hilo && !drain) || (drain && L.dhilo);
                const uint32_t slot_cols = (uint32_t)((L.dhilo ? 2 : 1) * args.n_chunk);
                int s = 0, tcount = 0, pcount = 0;
                uint32_t ph = 0;
                bool ok = true;
                for (int item = i_beg; item < i_end && ok; item += i_step, ++tcount) {
                    const int acc = L.n_acc == 2 ? (tcount & 1) : 0;
                    const uint32_t aph = (uint32_t)(L.n_acc == 2 ? (tcount >> 1) : tcount) & 1u;
                    if (!drain && !mbar_wait(&sm->tmem_empty[acc], aph ^ 1u, sm, args.error_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int nthis = item_nthis(item);
                    const int nA = nthis <= 256 ? nthis : ((nthis / 2 + 15) / 16) * 16;
                    const int nB = nthis - nA;
                    const uint32_t idA = umma_idesc(nA, args.f16), idB = nB > 0 ? umma_idesc(nB, args.f16) : 0u;
                    const uint32_t nB_off = (uint32_t)(nA * RB) >> 4;
                    uint32_t d_hi, d_lo;
                    if (AMODE == A_ROWS) {
                        // columns: part[0], part[1], lo[0], lo[1], each n_chunk wide
                        d_lo = tmem + (uint32_t)((2 + acc) * args.n_chunk);
                        d_hi = d_lo;  // set per K-chunk
                    } else {
                        d_hi = tmem + (uint32_t)(acc * L.acc_cols);
                        d_lo = args.hilo ? d_hi + (uint32_t)args.n_chunk : d_hi;
                    }
                    bool hi_on = false, lo_on = false;  // accumulate into the slot (false: overwrite)
                    int ps = 0;
                    for (int kc = 0; kc < KC; ++kc) {
                        if ((AMODE == A_ROWS && kc % kPartChunks == 0) || (drain && kc % L.drain == 0)) {
                            ps = pcount & 1;
                            const uint32_t pph = (uint32_t)(pcount >> 1) & 1u;
                            if (!mbar_wait(&sm->part_empty[ps], pph ^ 1u, sm, args.error_flag)) {
                                ok = false;
                                break;
                            }
                            d_hi = tmem + (uint32_t)ps * slot_cols;
                            if (drain) d_lo = L.dhilo ? d_hi + (uint32_t)args.n_chunk : d_hi;
                            hi_on = false;
                            if (drain && L.dhilo) lo_on = false;  // rows modes: lo spans the item
                        }
                        // with mma_pair > 1 the next chunks of the same partial (up to
                        // mma_pair in all, leaving a ring slot to the producers) are
                        // issued in the same step, their stages waited for here as well
                        int grp = 1;
                        while (grp < group_max && kc + grp < KC && (kc + grp) % L.drain != 0) ++grp;
                        bool got_all = true;
                        {
                            int ss = s;
                            uint32_t pp = ph;
                            for (int gi = 0; gi < grp && got_all; ++gi) {
                                got_all = mbar_wait(&sm->full[ss], pp, sm, args.error_flag);
                                if (++ss == S) {
                                    ss = 0;
                                    pp ^= 1u;
                                }
                            }
                        }
                        if (!got_all) {
                            ok = false;
                            break;
                        }
                        if (AMODE == A_GATHER) fence_proxy_async();  // cp.async data -> tensor-core reads
                        tc_fence_after();
                        constexpr int8_t kA[6] = {2, 1, 0, 1, 0, 0}, kB[6] = {0, 1, 2, 0, 1, 0};
                        auto issue_chunk = [&](int ss, int kk) {
                            const bool two = args.kdim - kk * CH >= 32;  // K steps of 16 in this chunk: 2 or 1
                            const uint64_t sd = desc0 + (uint64_t)((uint32_t)ss * stage_u);
                            if (two && nB == 0) {
                                // common case, kept free of branches between the MMAs
#pragma unroll
                                for (int pi = P0; pi < 6; ++pi) {
                                    const bool to_hi = (kA[pi] == 0 && kB[pi] == 0) || !split_lo;
                                    const uint32_t d = to_hi ? d_hi : d_lo;
                                    const uint64_t ad = sd + (uint64_t)(kA[pi] * a_u);
                                    const uint64_t bd = sd + (uint64_t)(c0_u + kB[pi] * c_u);
                                    umma_bf16(d, ad, bd, idA, (to_hi ? hi_on : lo_on) ? 1u : 0u);
                                    umma_bf16(d, ad + 2, bd + 2, idA, 1u);
                                    hi_on = hi_on || to_hi;
                                    lo_on = lo_on || !to_hi;
                                }
                            } else {
#pragma unroll
                                for (int pi = P0; pi < 6; ++pi) {
                                    const bool to_hi = (kA[pi] == 0 && kB[pi] == 0) || !split_lo;
                                    const uint32_t d = to_hi ? d_hi : d_lo;
                                    const uint64_t ad = sd + (uint64_t)(kA[pi] * a_u);
                                    const uint64_t bd = sd + (uint64_t)(c0_u + kB[pi] * c_u);
                                    const uint32_t en0 = (to_hi ? hi_on : lo_on) ? 1u : 0u;
                                    umma_bf16(d, ad, bd, idA, en0);
                                    if (nB > 0) umma_bf16(d + (uint32_t)nA, ad, bd + nB_off, idB, en0);
                                    if (two) {
                                        umma_bf16(d, ad + 2, bd + 2, idA, 1u);
                                        if (nB > 0) umma_bf16(d + (uint32_t)nA, ad + 2, bd + nB_off + 2, idB, 1u);
                                    }
                                    hi_on = hi_on || to_hi;
                                    lo_on = lo_on || !to_hi;
                                }
                            }
                            umma_commit(&sm->empty[ss]);
                        };
                        issue_chunk(s, kc);
                        for (int gi = 1; gi < grp; ++gi) {
                            if (++s == S) {
                                s = 0;
                                ph ^= 1u;
                            }
                            ++kc;
                            issue_chunk(s, kc);
                        }
                        if ((AMODE == A_ROWS && (kc % kPartChunks == kPartChunks - 1 || kc == KC - 1)) ||
                            (drain && (kc % L.drain == L.drain - 1 || kc == KC - 1))) {
                            umma_commit(&sm->part_full[ps]);
                            ++pcount;
                        }
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    if (!drain) umma_commit(&sm->tmem_full[acc]);
                }
            };
            if (args.n_products == 1) run(std::integral_constant<int, 1>{});
            else if (args.n_products == 3) run(std::integral_constant<int, 3>{});
            else run(std::integral_constant<int, 6>{});
            umma_commit(&sm->drain);
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&sm->drain, 0u) && global_ns() - t0 < kWaitNs) {
            }
        }
        __syncwarp();
    } else if (AMODE == A_GATHER && L.drain) {
        // ================= epilogue, drain mode (core) =================
        // Eight warps: warp w reads TMEM lane quarter w mod 4 and the 32-wide
        // column chunks of its half of the item's N columns (warps 0-3 the
        // first half, warps 7-10 the second).  Each partial (L.drain K-chunks
        // of every product) is added to per-row FP32 running sums in
        // registers (round to nearest), so no accumulator chain in TMEM is
        // longer than L.drain K-chunks, and the MMAs run up to two partials
        // ahead of the drains.  After the tile's last partial the sums are
        // scaled by s_l and reduced into p~ as in the classic epilogue; the
        // MMAs of the next tile fill the two partial slots meanwhile.
        const int q = warp & 3;
        const int half = warp < kEpiWarps ? 0 : 1;
        const int ew = warp < kEpiWarps ? warp : warp - 3;
        float* trans = reinterpret_cast<float*>(smem_raw + L.trans_off) + ew * 32 * kTransStride;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int pcount = 0;
        int e_nxt_row = -1, e_nxt_k = 0;
        float e_nxt_rs = 1.f;  // per-row factor of the A row (row_scale), this lane's row
        auto row_factor = [&](int t) -> float {
            if (!args.row_scale) return 1.f;
            const int sr = __ldg(args.row_src + (long)t * kTileM + q * 32 + lane);
            return sr >= 0 ? __ldg(args.row_scale + sr) : 0.f;
        };
        if (EMODE == E_RED && i_beg < i_end) {
            const int t0 = item_tile(i_beg);
            e_nxt_row = __ldg(args.row_dst + (long)t0 * kTileM + q * 32 + lane);
            e_nxt_k = __ldg(args.tile_k + t0);
            e_nxt_rs = row_factor(t0);
        }
        bool ok = true;
        for (int item = i_beg; item < i_end && ok; item += i_step) {
            long orow = e_nxt_row;
            float oscale = 1.0f, rsc = 1.0f;
            float* e_dbase = args.D;
            float e_alpha = args.alpha, e_beta = args.beta;
            if (EMODE == E_RED) {
                oscale = args.scale_table ? __ldg(args.scale_table + (e_nxt_k >> 16))
                                          : args.level_scale[(e_nxt_k >> 16) & 31];
                rsc = e_nxt_rs;
                if (item + i_step < i_end) {
                    const int tn = item_tile(item + i_step);
                    e_nxt_row = __ldg(args.row_dst + (long)tn * kTileM + q * 32 + lane);
                    e_nxt_k = __ldg(args.tile_k + tn);
                    e_nxt_rs = row_factor(tn);
                }
            } else {
                // identity rows (compression / expansion): the tile's segment
                // gives the row of this lane in its input and its output
                const int tt = item_tile(item);
                long r = (long)tt * kTileM + q * 32 + lane;
                long mrows = args.m_rows, obase = 0;
                if (args.n_segs > 0) {
                    const RowSeg sg = args.segs[find_seg(tt)];
                    r = (long)(tt - sg.tile_begin) * kTileM + q * 32 + lane;
                    mrows = sg.m_rows;
                    obase = sg.out_row;
                    e_dbase = sg.D;
                    e_alpha = sg.alpha;
                    e_beta = sg.beta;
                }
                orow = r < mrows ? (EMODE == E_SPLIT ? obase + r : r) : -1;
                // FP16 pieces: this row times its power of two
                if (EMODE == E_SPLIT && args.dp_f16 && orow >= 0) rsc = 1.f / __ldg(args.dp_row_inv + orow);
            }
            const int n0 = item_n0(item), nthis = item_nthis(item);
            const int nch = (nthis + 31) / 32;
            const int c_beg = half ? (nch + 1) / 2 : 0, c_end = half ? nch : (nch + 1) / 2;
            float sums[96];
#pragma unroll
            for (int j = 0; j < 96; ++j) sums[j] = 0.f;
            for (int kc = 0; kc < KC; kc += L.drain) {
                const int ps = pcount & 1;
                const bool got = mbar_wait(&sm->part_full[ps], (uint32_t)(pcount >> 1) & 1u, sm, args.error_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t pcol = (uint32_t)(ps * (L.dhilo ? 2 : 1) * args.n_chunk);
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) {
                    const int c = (c_beg + jj) * 32;
                    if (c_beg + jj < c_end) {
                        // the slot's (0,0) half, then (dhilo) its small products' half
                        for (int hl = 0; hl < (L.dhilo ? 2 : 1); ++hl) {
                            const uint32_t col = pcol + (uint32_t)(hl * args.n_chunk + c);
                            uint32_t r[32];
                            if (c + 32 <= nthis) {
                                tmem_ld32(tmem + lane_base + col, r);
                            } else {
                                tmem_ld16(tmem + lane_base + col, r);
#pragma unroll
                                for (int j = 16; j < 32; ++j) r[j] = 0u;
                            }
                            tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 32; ++j) sums[jj * 32 + j] += __uint_as_float(r[j]);
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&sm->part_empty[ps]);
                ++pcount;
            }
            if (!ok) break;
            if (EMODE == E_RED && args.direct_rows) {
                // every lane reduces its own row segment: 16-byte vector
                // atomics at D[orow][n0 + c ..], no shared-memory transpose
                if (orow >= 0) {
                    const float f = oscale * rsc;
                    float* drow = args.D + orow * args.ldd + n0;
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) {
                        const int c = (c_beg + jj) * 32;
                        if (c_beg + jj < c_end) {
                            const int ncols = c + 32 <= nthis ? 32 : 16;
#pragma unroll
                            for (int qq = 0; qq < 8; ++qq)
                                if (4 * qq < ncols)
                                    red_add_v4(drow + c + 4 * qq, __float_as_uint(f * sums[jj * 32 + 4 * qq]),
                                               __float_as_uint(f * sums[jj * 32 + 4 * qq + 1]),
                                               __float_as_uint(f * sums[jj * 32 + 4 * qq + 2]),
                                               __float_as_uint(f * sums[jj * 32 + 4 * qq + 3]));
                        }
                    }
                }
                continue;
            }
            if (EMODE == E_RED && args.red_bulk) {
                // every lane hands its own row segment to the TMA unit: one bulk
                // reduction of 32 (or 16) FP32 values per chunk, staged in the
                // lane's row of the transpose buffer
                float* my = trans + lane * kTransStride;
                const float f = oscale * rsc;
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) {
                    const int c = (c_beg + jj) * 32;
                    if (c_beg + jj < c_end) {
                        const int ncols = c + 32 <= nthis ? 32 : 16;
                        bulk_wait_read_all();  // the previous chunk has left the buffer
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq)
                            if (4 * qq < ncols)
                                *reinterpret_cast<float4*>(my + 4 * qq) =
                                    make_float4(f * sums[jj * 32 + 4 * qq], f * sums[jj * 32 + 4 * qq + 1],
                                                f * sums[jj * 32 + 4 * qq + 2], f * sums[jj * 32 + 4 * qq + 3]);
                        fence_proxy_async();
                        if (orow >= 0) {
                            bulk_reduce_add_f32(args.D + orow * args.ldd + n0 + c, smem_u32(my), (uint32_t)ncols * 4u);
                            bulk_commit();
                        }
                    }
                }
                continue;
            }
            long prow[8];
#pragma unroll
            for (int pass = 0; pass < 8; ++pass) prow[pass] = __shfl_sync(0xffffffffu, orow, pass * 4 + lane / 8);
            const int c4 = lane % 8;
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                const int c = (c_beg + jj) * 32;
                if (c_beg + jj < c_end) {
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq)
                        *reinterpret_cast<float4*>(trans + lane * kTransStride + 4 * qq) =
                            make_float4(rsc * sums[jj * 32 + 4 * qq], rsc * sums[jj * 32 + 4 * qq + 1],
                                        rsc * sums[jj * 32 + 4 * qq + 2], rsc * sums[jj * 32 + 4 * qq + 3]);
                    __syncwarp();
                    const int ncols = c + 32 <= nthis ? 32 : 16;
#pragma unroll
                    for (int pass = 0; pass < 8; ++pass) {
                        const int rr = pass * 4 + lane / 8;
                        const long grow = prow[pass];
                        if (grow < 0 || 4 * c4 >= ncols) continue;
                        float4 x = *reinterpret_cast<const float4*>(trans + rr * kTransStride + 4 * c4);
                        const int col = n0 + c + 4 * c4;
                        if (EMODE == E_RED) {
                            red_add_v4(args.D + grow * args.ldd + col, __float_as_uint(oscale * x.x),
                                       __float_as_uint(oscale * x.y), __float_as_uint(oscale * x.z),
                                       __float_as_uint(oscale * x.w));
                        } else if (EMODE == E_STORE) {
                            if (col < args.n_valid) {
                                float4* dp = reinterpret_cast<float4*>(e_dbase + grow * args.ldd + col);
                                float4 y = make_float4(e_alpha * x.x, e_alpha * x.y, e_alpha * x.z, e_alpha * x.w);
                                if (e_beta != 0.f) {
                                    const float4 o = *dp;
                                    y.x = fmaf(e_beta, o.x, y.x);
                                    y.y = fmaf(e_beta, o.y, y.y);
                                    y.z = fmaf(e_beta, o.z, y.z);
                                    y.w = fmaf(e_beta, o.w, y.w);
                                }
                                *dp = y;
                            }
                        } else {  // E_SPLIT
                            x.x *= e_alpha;
                            x.y *= e_alpha;
                            x.z *= e_alpha;
                            x.w *= e_alpha;
                            if (args.Df) *reinterpret_cast<float4*>(args.Df + grow * args.ldd + col) = x;
                            if (args.Z)
                                *reinterpret_cast<float4*>(args.Z + grow * args.ldd + col) = make_float4(0.f, 0.f, 0.f, 0.f);
                            uint32_t lo[3], hi[3];
                            if (args.dp_f16) {
                                const __half2 a = __floats2half2_rn(x.x, x.y), b = __floats2half2_rn(x.z, x.w);
                                const __half2 al = __floats2half2_rn(x.x - __low2float(a), x.y - __high2float(a));
                                const __half2 bl = __floats2half2_rn(x.z - __low2float(b), x.w - __high2float(b));
                                lo[0] = *reinterpret_cast<const uint32_t*>(&a);
                                hi[0] = *reinterpret_cast<const uint32_t*>(&b);
                                lo[1] = *reinterpret_cast<const uint32_t*>(&al);
                                hi[1] = *reinterpret_cast<const uint32_t*>(&bl);
                                lo[2] = hi[2] = 0u;
                            } else {
                                split3x2(x.x, x.y, lo, args.dp_pieces);
                                split3x2(x.z, x.w, hi, args.dp_pieces);
                            }
#pragma unroll
                            for (int pc = 0; pc < 3; ++pc) {
                                if (pc >= args.dp_pieces) break;
                                *reinterpret_cast<uint2*>(args.Dp + pc * args.dp_piece_stride + grow * args.ldd + col) =
                                    make_uint2(lo[pc], hi[pc]);
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        }
        if (EMODE == E_RED && args.red_bulk) bulk_wait_all();  // reductions complete before teardown
    } else {
        // ================= epilogue =================
        float* trans = reinterpret_cast<float*>(smem_raw + L.trans_off) + warp * 32 * kTransStride;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const bool has_lo = args.hilo && args.n_products > 1;
        int tcount = 0, pcount = 0;
        int e_nxt_row = -1, e_nxt_k = 0;
        float e_nxt_rs = 1.f;  // per-row factor of the A row (row_scale), this lane's row
        auto row_factor = [&](int t) -> float {
            if (!args.row_scale) return 1.f;
            const int sr = __ldg(args.row_src + (long)t * kTileM + warp * 32 + lane);
            return sr >= 0 ? __ldg(args.row_scale + sr) : 0.f;
        };
        if (AMODE == A_GATHER && i_beg < i_end) {
            const int t0 = item_tile(i_beg);
            e_nxt_row = __ldg(args.row_dst + (long)t0 * kTileM + warp * 32 + lane);
            e_nxt_k = __ldg(args.tile_k + t0);
            e_nxt_rs = row_factor(t0);
        }
        for (int item = i_beg; item < i_end; item += i_step, ++tcount) {
            const int acc = tcount % L.n_acc;
            const uint32_t aph = (uint32_t)(tcount / L.n_acc) & 1u;
            const int n0 = item_n0(item), nthis = item_nthis(item);
            // this lane's output row (tile row warp*32 + lane); -1 = none
            long orow = -1;
            float oscale = 1.0f, rsc = 1.0f;
            float* e_dbase = args.D;
            float e_alpha = args.alpha, e_beta = args.beta;
            if (AMODE == A_GATHER) {
                orow = e_nxt_row;
                oscale = args.scale_table ? __ldg(args.scale_table + (e_nxt_k >> 16))
                                          : args.level_scale[(e_nxt_k >> 16) & 31];
                rsc = e_nxt_rs;
                if (item + i_step < i_end) {  // prefetch the next item's rows
                    const int tn = item_tile(item + i_step);
                    e_nxt_row = __ldg(args.row_dst + (long)tn * kTileM + warp * 32 + lane);
                    e_nxt_k = __ldg(args.tile_k + tn);
                    e_nxt_rs = row_factor(tn);
                }
            } else if (args.n_segs > 0) {
                const RowSeg sg = args.segs[find_seg(item_tile(item))];
                const long r = (long)(item_tile(item) - sg.tile_begin) * kTileM + warp * 32 + lane;
                if (r < sg.m_rows) orow = (EMODE == E_SPLIT) ? sg.out_row + r : r;
                e_dbase = sg.D;
                e_alpha = sg.alpha;
                e_beta = sg.beta;
            } else {
                const long r = (long)item_tile(item) * kTileM + warp * 32 + lane;
                if (r < args.m_rows) orow = r;
            }
            const uint32_t col_hi = (uint32_t)(acc * L.acc_cols);
            const uint32_t col_lo = col_hi + (uint32_t)args.n_chunk;
            // rows modes: sum the per-K-chunk partials of the (0,0) product in
            // registers (round to nearest), then add the lo slot
            float sums[kMaxRowsChunk];
            if (AMODE == A_ROWS) {
#pragma unroll
                for (int j = 0; j < kMaxRowsChunk; ++j) sums[j] = 0.f;
                bool got_all = true;
                for (int kc = 0; kc < KC; kc += kPartChunks) {
                    const int ps = pcount % 2;
                    const uint32_t pph = (uint32_t)(pcount / 2) & 1u;
                    const bool gp = mbar_wait(&sm->part_full[ps], pph, sm, args.error_flag);
                    if (!__all_sync(0xffffffffu, gp)) {
                        got_all = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t pcol = (uint32_t)(ps * args.n_chunk);
#pragma unroll
                    for (int c = 0; c < kMaxRowsChunk; c += 32) {
                        if (c >= nthis) break;
                        uint32_t r[32];
                        if (c + 32 <= nthis)
                            tmem_ld32(tmem + lane_base + pcol + (uint32_t)c, r);
                        else
                            tmem_ld16(tmem + lane_base + pcol + (uint32_t)c, r);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (c + j < nthis) sums[c + j] += __uint_as_float(r[j]);
                    }
                    tc_fence_before();
                    mbar_arrive(&sm->part_empty[ps]);
                    ++pcount;
                }
                if (!got_all) break;
            }
            // the whole item (lo slot, or the core's accumulator) is complete
            const bool got = mbar_wait(&sm->tmem_full[acc], aph, sm, args.error_flag);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            const uint32_t col_lo_rows = (uint32_t)((2 + acc) * args.n_chunk);
            // output rows of the 8 transpose passes of this lane (pass p
            // serves tile row 4 p + lane / 8)
            long prow[8];
#pragma unroll
            for (int pass = 0; pass < 8; ++pass) prow[pass] = __shfl_sync(0xffffffffu, orow, pass * 4 + lane / 8);
            const int c4 = lane % 8;
            for (int c = 0; c < nthis; c += 32) {
                uint32_t r[32], r2[32];
                const bool full32 = c + 32 <= nthis;
                float val[32];
                // issue the TMEM loads of this chunk together, then wait once
                const uint32_t a0 = tmem + lane_base + (AMODE == A_ROWS ? col_lo_rows : col_hi) + (uint32_t)c;
                if (full32) tmem_ld32(a0, r);
                else tmem_ld16(a0, r);
                if (AMODE != A_ROWS && has_lo) {
                    if (full32) tmem_ld32(tmem + lane_base + col_lo + (uint32_t)c, r2);
                    else tmem_ld16(tmem + lane_base + col_lo + (uint32_t)c, r2);
                }
                tmem_wait_ld();
                if (AMODE == A_ROWS) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        // sums[] is indexed by a loop-invariant offset c (0, 32, 64)
                        float sv = 0.f;
#pragma unroll
                        for (int cc = 0; cc < kMaxRowsChunk; cc += 32)
                            if (cc == c && cc + j < kMaxRowsChunk) sv = sums[cc + j];
                        val[j] = sv + __uint_as_float(r[j]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) val[j] = __uint_as_float(r[j]);
                    if (has_lo) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) val[j] += __uint_as_float(r2[j]);
                    }
                }
                // transpose through shared memory: lane -> row (16-byte stores),
                // then 8 lanes per row (16-byte loads)
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *reinterpret_cast<float4*>(trans + lane * kTransStride + 4 * q) =
                        make_float4(rsc * val[4 * q], rsc * val[4 * q + 1], rsc * val[4 * q + 2], rsc * val[4 * q + 3]);
                __syncwarp();
                const int ncols = full32 ? 32 : 16;
#pragma unroll
                for (int pass = 0; pass < 8; ++pass) {
                    const int rr = pass * 4 + lane / 8;
                    const long grow = prow[pass];
                    if (grow < 0 || 4 * c4 >= ncols) continue;
                    float4 x = *reinterpret_cast<const float4*>(trans + rr * kTransStride + 4 * c4);
                    const int col = n0 + c + 4 * c4;
                    if (EMODE == E_RED) {
                        // one tile = one level: every lane holds the same scale
                        red_add_v4(args.D + grow * args.ldd + col, __float_as_uint(oscale * x.x),
                                   __float_as_uint(oscale * x.y), __float_as_uint(oscale * x.z),
                                   __float_as_uint(oscale * x.w));
                    } else if (EMODE == E_STORE) {
                        if (col < args.n_valid) {
                            float4* dp = reinterpret_cast<float4*>(e_dbase + grow * args.ldd + col);
                            float4 y = make_float4(e_alpha * x.x, e_alpha * x.y, e_alpha * x.z, e_alpha * x.w);
                            if (e_beta != 0.f) {
                                const float4 o = *dp;
                                y.x = fmaf(e_beta, o.x, y.x);
                                y.y = fmaf(e_beta, o.y, y.y);
                                y.z = fmaf(e_beta, o.z, y.z);
                                y.w = fmaf(e_beta, o.w, y.w);
                            }
                            *dp = y;
                        }
                    } else {  // E_SPLIT
                        x.x *= e_alpha;
                        x.y *= e_alpha;
                        x.z *= e_alpha;
                        x.w *= e_alpha;
                        if (args.Df)
                            *reinterpret_cast<float4*>(args.Df + grow * args.ldd + col) = x;
                        if (args.Z)
                            *reinterpret_cast<float4*>(args.Z + grow * args.ldd + col) = make_float4(0.f, 0.f, 0.f, 0.f);
                        uint32_t lo[3], hi[3];
                        split3x2(x.x, x.y, lo, args.dp_pieces);
                        split3x2(x.z, x.w, hi, args.dp_pieces);
#pragma unroll
                        for (int pc = 0; pc < 3; ++pc) {
                            if (pc >= args.dp_pieces) break;
                            uint2 pk = make_uint2(lo[pc], hi[pc]);
                            *reinterpret_cast<uint2*>(args.Dp + pc * args.dp_piece_stride + grow * args.ldd + col) = pk;
                        }
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            mbar_arrive(&sm->tmem_empty[acc]);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kEpiWarps + kProdWarps) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}


// ---------------------------------------------------------------------------
// Core GEMM with the A tile resident in shared memory (split6 with hilo).
//
// With hilo, one 128-row tile needs 2 N TMEM columns (hi and lo); for
// N = r_pad = 192 that is 384 of the 512 columns, so the classic kernel has
// one accumulator slot and each tile's epilogue (bounded by the L2's
// reduction rate) runs between two tiles' MMAs.  Here the A tile (all K,
// 3 pieces: 144 KB for K = 192) stays in shared memory for the whole tile and
// K~_o is streamed in NB column blocks of width BN <= 128: a block's hi and
// lo take 2 BN columns, two blocks ping-pong in TMEM, and the epilogue of one
// block overlaps the MMAs of the next.  Per output element the sums run in
// the same order as in the classic kernel.
//
// Warp roles (384 threads):
//   warps 0-3   epilogue (as in the classic kernel, per N block)
//   warps 4-9   A producers: warp 4 + w gathers the K-chunks j = w (mod 6)
//               of every tile into A slot j (cp.async, 64-byte swizzle)
//   warp 10     B producer: one thread TMA-loads the (block, K-chunk) tiles
//               of K~_o through a ring of SB slots
//   warp 11     TMEM allocation and the MMA-issuing thread
// A slot j is released (for the next tile) by the MMA commit that follows
// the last block's use of it.
constexpr int kResAWarps = 6, kResBWarp = 10, kResMmaWarp = 11;
constexpr int kResMaxKC = 8, kResMaxSB = 4;

struct RSmem {
    uint64_t a_full[kResMaxKC], a_empty[kResMaxKC];
    uint64_t b_full[kResMaxSB], b_empty[kResMaxSB];
    uint64_t t_full[2], t_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    volatile int abort_flag;
    unsigned long long wait_ns;  // bound of every mbarrier wait of this launch
};

struct RLayout {
    int kc_count;            // K chunks of 32 = A slots
    int nb, bn;              // N blocks, block width (last block may be narrower)
    int sb;                  // B ring slots
    int n_items;             // tiles
    uint32_t b_off;          // B ring offset from the A region (= A bytes)
    uint32_t b_piece_bytes;  // bn * 64
    uint32_t trans_off;      // transpose buffers, from the A region
};

__global__ void __launch_bounds__(kThreads, 1)
    core_resident_kernel(const __grid_constant__ CUtensorMap bmap, const UmmaArgs args, const RLayout L) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    uint8_t* smem_raw = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    RSmem* sm = reinterpret_cast<RSmem*>(smem_raw);
    uint8_t* a_region = smem_raw + 1024;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr int CH = 32, RB = 64;
    constexpr uint32_t kAPiece = kTileM * CH * 2;  // 8 KB
    const int KC = L.kc_count, NB = L.nb, BN = L.bn, SB = L.sb;
    const bool contig = args.contiguous != 0;
    const int i_beg = contig ? (int)((long)L.n_items * blockIdx.x / gridDim.x) : (int)blockIdx.x;
    const int i_end = contig ? (int)((long)L.n_items * (blockIdx.x + 1) / gridDim.x) : L.n_items;
    const int i_step = contig ? 1 : (int)gridDim.x;

    if (threadIdx.x == 0) {
        for (int j = 0; j < KC; ++j) {
            mbar_init(&sm->a_full[j], 32);
            mbar_init(&sm->a_empty[j], 1);
        }
        for (int b = 0; b < SB; ++b) {
            mbar_init(&sm->b_full[b], 1);
            mbar_init(&sm->b_empty[b], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sm->t_full[a], 1);
            mbar_init(&sm->t_empty[a], kEpiWarps * 32);
        }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        sm->wait_ns = args.wait_ns ? args.wait_ns : kWaitNs;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kResMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&sm->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;
    auto a_slot = [&](int j, int piece) -> uint32_t {
        return smem_u32(a_region + (size_t)(j * 3 + piece) * kAPiece);
    };
    auto b_slot = [&](int b, int piece) -> uint32_t {
        return smem_u32(a_region + L.b_off + (size_t)(b * 3 + piece) * L.b_piece_bytes);
    };

    if (warp >= kEpiWarps && warp < kEpiWarps + kResAWarps) {
        // ================= A producers =================
        const int aw = warp - kEpiWarps;
        constexpr int CPR = CH / 8, RPI = 32 / CPR, NR = kTileM / RPI;
        const int cch = lane % CPR, rl = lane / CPR;
        bool ok = true;
        int ic = 0;
        int nrow[NR];
        if (aw < KC && i_beg < i_end) {
#pragma unroll
            for (int i = 0; i < NR; ++i) nrow[i] = __ldg(args.row_src + (long)i_beg * kTileM + rl + RPI * i);
        }
        for (int item = i_beg; item < i_end && ok && aw < KC; item += i_step, ++ic) {
            const __nv_bfloat16* rowp[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) rowp[i] = args.A + (long)(nrow[i] < 0 ? args.zero_row : nrow[i]) * args.kdim;
            if (item + i_step < i_end) {
#pragma unroll
                for (int i = 0; i < NR; ++i)
                    nrow[i] = __ldg(args.row_src + (long)(item + i_step) * kTileM + rl + RPI * i);
            }
            for (int j = aw; j < KC; j += kResAWarps) {
                if (!mbar_wait(&sm->a_empty[j], (uint32_t)(ic & 1) ^ 1u, sm, args.error_flag)) {
                    ok = false;
                    break;
                }
                const int col = j * CH + cch * 8;
                const uint32_t bytes = col < args.kdim ? 16u : 0u;
                const int colc = col < args.kdim ? col : 0;
#pragma unroll
                for (int pc = 0; pc < 3; ++pc) {
                    const uint32_t sbase = a_slot(j, pc);
                    const long poff = pc * args.a_piece_stride + colc;
#pragma unroll
                    for (int i = 0; i < NR; ++i) cp_async16(sbase + swz<CH>(rl + RPI * i, cch), rowp[i] + poff, bytes);
                }
                cp_async_commit();
                cp_async_wait_0();
                fence_proxy_async();
                mbar_arrive(&sm->a_full[j]);
            }
        }
        cp_async_wait_0();
    } else if (warp == kResBWarp) {
        // ================= B producer =================
        if (lane == 0) {
            int b = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int item = i_beg; item < i_end && ok; item += i_step) {
                const int group = __ldg(args.tile_k + item) & 0xFFFF;
                for (int nb = 0; nb < NB && ok; ++nb) {
                    for (int kc = 0; kc < KC; ++kc) {
                        if (!mbar_wait(&sm->b_empty[b], ph ^ 1u, sm, args.error_flag)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&sm->b_full[b], 3u * L.b_piece_bytes);
#pragma unroll
                        for (int pc = 0; pc < 3; ++pc)
                            tma_load_2d(b_slot(b, pc), &bmap, kc * CH, (pc * args.b_groups + group) * args.ndim + nb * BN,
                                        &sm->b_full[b]);
                        if (++b == SB) {
                            b = 0;
                            ph ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                const unsigned long long t0 = global_ns();
                while (global_ns() - t0 < 1000000ull) {
                }
            }
        }
    } else if (warp == kResMmaWarp) {
        // ================= MMA issuer =================
        if (lane == 0) {
            const uint64_t adesc0 = umma_desc<CH>(a_slot(0, 0));
            const uint64_t bdesc0 = umma_desc<CH>(b_slot(0, 0));
            const uint32_t a_u = kAPiece >> 4, bp_u = L.b_piece_bytes >> 4;
            int b = 0, bc = 0, ic = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int item = i_beg; item < i_end && ok; item += i_step, ++ic) {
                for (int nb = 0; nb < NB && ok; ++nb, ++bc) {
                    const int slot = bc & 1;
                    if (!mbar_wait(&sm->t_empty[slot], (uint32_t)((bc >> 1) & 1) ^ 1u, sm, args.error_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int nthis = min(BN, args.ndim - nb * BN);
                    const uint32_t idesc = umma_idesc_bf16(nthis);
                    const uint32_t d_hi = tmem + (uint32_t)(slot * 2 * BN), d_lo = d_hi + (uint32_t)BN;
                    bool hi_on = false, lo_on = false;
                    for (int kc = 0; kc < KC; ++kc) {
                        if (nb == 0 && !mbar_wait(&sm->a_full[kc], (uint32_t)(ic & 1), sm, args.error_flag)) {
                            ok = false;
                            break;
                        }
                        if (!mbar_wait(&sm->b_full[b], ph, sm, args.error_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const bool two = args.kdim - kc * CH >= 32;
                        const uint64_t ad = adesc0 + (uint64_t)((uint32_t)(kc * 3) * a_u);
                        const uint64_t bd = bdesc0 + (uint64_t)((uint32_t)(b * 3) * bp_u);
                        constexpr int8_t kA[6] = {2, 1, 0, 1, 0, 0}, kB[6] = {0, 1, 2, 0, 1, 0};
                        if (two) {
                            // common case, kept free of branches between the MMAs
#pragma unroll
                            for (int pi = 0; pi < 6; ++pi) {
                                const bool to_hi = kA[pi] == 0 && kB[pi] == 0;
                                const uint32_t d = to_hi ? d_hi : d_lo;
                                const uint64_t pa = ad + (uint64_t)(kA[pi] * a_u), pb = bd + (uint64_t)(kB[pi] * bp_u);
                                umma_bf16(d, pa, pb, idesc, (to_hi ? hi_on : lo_on) ? 1u : 0u);
                                umma_bf16(d, pa + 2, pb + 2, idesc, 1u);
                                if (to_hi) hi_on = true;
                                else lo_on = true;
                            }
                        } else {
#pragma unroll
                            for (int pi = 0; pi < 6; ++pi) {
                                const bool to_hi = kA[pi] == 0 && kB[pi] == 0;
                                const uint32_t d = to_hi ? d_hi : d_lo;
                                const uint64_t pa = ad + (uint64_t)(kA[pi] * a_u), pb = bd + (uint64_t)(kB[pi] * bp_u);
                                umma_bf16(d, pa, pb, idesc, (to_hi ? hi_on : lo_on) ? 1u : 0u);
                                if (to_hi) hi_on = true;
                                else lo_on = true;
                            }
                        }
                        umma_commit(&sm->b_empty[b]);
                        if (nb == NB - 1) umma_commit(&sm->a_empty[kc]);
                        if (++b == SB) {
                            b = 0;
                            ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    umma_commit(&sm->t_full[slot]);
                }
            }
            umma_commit(&sm->drain);
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&sm->drain, 0u) && global_ns() - t0 < kWaitNs) {
            }
        }
        __syncwarp();
    } else if (warp < kEpiWarps) {
        // ================= epilogue =================
        float* trans = reinterpret_cast<float*>(a_region + L.trans_off) + warp * 32 * kTransStride;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        int bc = 0;
        int e_nxt_row = -1, e_nxt_k = 0;
        if (i_beg < i_end) {
            e_nxt_row = __ldg(args.row_dst + (long)i_beg * kTileM + warp * 32 + lane);
            e_nxt_k = __ldg(args.tile_k + i_beg);
        }
        bool ok = true;
        for (int item = i_beg; item < i_end && ok; item += i_step) {
            const long orow = e_nxt_row;
            const float oscale = args.scale_table ? __ldg(args.scale_table + (e_nxt_k >> 16))
                                                  : args.level_scale[(e_nxt_k >> 16) & 31];
            if (item + i_step < i_end) {
                e_nxt_row = __ldg(args.row_dst + (long)(item + i_step) * kTileM + warp * 32 + lane);
                e_nxt_k = __ldg(args.tile_k + item + i_step);
            }
            long prow[8];
#pragma unroll
            for (int pass = 0; pass < 8; ++pass) prow[pass] = __shfl_sync(0xffffffffu, orow, pass * 4 + lane / 8);
            const int c4 = lane % 8;
            for (int nb = 0; nb < NB; ++nb, ++bc) {
                const int slot = bc & 1;
                const bool got = mbar_wait(&sm->t_full[slot], (uint32_t)((bc >> 1) & 1), sm, args.error_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int nthis = min(BN, args.ndim - nb * BN);
                const uint32_t col_hi = (uint32_t)(slot * 2 * BN), col_lo = col_hi + (uint32_t)BN;
                for (int c = 0; c < nthis; c += 32) {
                    uint32_t r[32], r2[32];
                    const bool full32 = c + 32 <= nthis;
                    if (full32) {
                        tmem_ld32(tmem + lane_base + col_hi + (uint32_t)c, r);
                        tmem_ld32(tmem + lane_base + col_lo + (uint32_t)c, r2);
                    } else {
                        tmem_ld16(tmem + lane_base + col_hi + (uint32_t)c, r);
                        tmem_ld16(tmem + lane_base + col_lo + (uint32_t)c, r2);
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4*>(trans + lane * kTransStride + 4 * q) = make_float4(
                            __uint_as_float(r[4 * q]) + __uint_as_float(r2[4 * q]),
                            __uint_as_float(r[4 * q + 1]) + __uint_as_float(r2[4 * q + 1]),
                            __uint_as_float(r[4 * q + 2]) + __uint_as_float(r2[4 * q + 2]),
                            __uint_as_float(r[4 * q + 3]) + __uint_as_float(r2[4 * q + 3]));
                    __syncwarp();
                    const int ncols = full32 ? 32 : 16;
#pragma unroll
                    for (int pass = 0; pass < 8; ++pass) {
                        const int rr = pass * 4 + lane / 8;
                        const long grow = prow[pass];
                        if (grow < 0 || 4 * c4 >= ncols) continue;
                        const float4 x = *reinterpret_cast<const float4*>(trans + rr * kTransStride + 4 * c4);
                        red_add_v4(args.D + grow * args.ldd + nb * BN + c + 4 * c4, __float_as_uint(oscale * x.x),
                                   __float_as_uint(oscale * x.y), __float_as_uint(oscale * x.z),
                                   __float_as_uint(oscale * x.w));
                    }
                    __syncwarp();
                }
                tc_fence_before();
                mbar_arrive(&sm->t_empty[slot]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kResMmaWarp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}


// ---------------------------------------------------------------------------
// Stage-2 core (Sec. 3.2, Eq. (17)).  With K~_o = Uhat_o Vhat_o (rank k_o,
// rounded up to k16 <= 96), a tile's product is two skinny GEMMs:
//   T = Q~_rows Vhat_o^T   (128 x k16, K = r_pad)     split products, hi/lo
//   P = T Uhat_o^T         (128 x r_pad, K = k16)     split products
// T never leaves the SM: the epilogue warps read it from TMEM, add hi and lo,
// split it into BF16 pieces and store them, 64B-swizzled, as the A operand of
// the second GEMM.  P is reduced into p~ as in the other cores.
//
// Warp roles (384 threads):
//   warps 0-3   epilogue: T split, then the reduction of P
//   warps 4-6   producers, one ring slot each: the first GEMM's stages (q~
//               rows by cp.async, Vhat_o by TMA) and the second GEMM's stages
//               (Uhat_o by TMA, one 96-row part of N per stage)
//   warp 11     TMEM allocation and the MMA-issuing thread
// TMEM columns: T hi [0, 96), T lo [96, 192), P [192, 192 + r_pad).
// The next tile's first GEMM runs while the epilogue reduces P.
constexpr int kS2Prod = 3, kS2MaxStages = 6, kS2Kmax = 96, kS2Part = 96;
constexpr int kOffsetsHost = KIFMM_N_OFFSETS;

struct S2Smem {
    uint64_t full[kS2MaxStages], empty[kS2MaxStages];
    uint64_t t_full, t_empty, tsplit, tbuf_free, p_full, p_empty, drain;
    uint64_t tinv_full[2], tinv_empty[2];  // the T rows' powers of two, T warps -> P warps (f16x3)
    uint32_t tmem_base;
    volatile int abort_flag;
    unsigned long long wait_ns;  // bound of every mbarrier wait of this launch
};

struct S2Layout {
    int kc1;                 // K chunks of the first GEMM (r_pad / 32, rounded up)
    int nh;                  // 96-row parts of N in the second GEMM
    int n_items;             // tiles
    int stages;              // ring stages (at least the 3 producer warps, at most kS2MaxStages)
    uint32_t stage_bytes;    // A pieces (pieces x 8 KB) + B pieces (pieces x 96 rows x 64 B)
    uint32_t tbuf_off;       // T pieces [3 chunks][pieces][128 x 64 B], from the stage ring base
    uint32_t trans_off;      // epilogue transpose buffers (one per P-draining warp), from the stage ring base
    uint32_t tmax_off;       // the T rows' inverse powers of two, 2 slots of 128 floats
};

template <int NP>
__global__ void __launch_bounds__(kThreads, 1)
    core_stage2_kernel(const __grid_constant__ CUtensorMap vmap, const __grid_constant__ CUtensorMap umap,
                       const UmmaArgs args, const S2Layout L) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    uint8_t* smem_raw = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    S2Smem* sm = reinterpret_cast<S2Smem*>(smem_raw);
    uint8_t* ring = smem_raw + 1024;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr int CH = 32, RB = 64;
    constexpr int PC = NP == 6 ? 3 : (NP == 3 ? 2 : 1);  // BF16 pieces
    constexpr int P0 = 6 - NP;
    constexpr bool HILO = NP > 1;
    // epilogue warps: 8 (warps 0-3 split T, the idle producer warps 7-10
    // drain P) for 1 or 2 pieces; split6 keeps one set of 4 doing both
    constexpr int EW = NP == 6 ? 4 : 8;
    constexpr uint32_t kAPiece = kTileM * CH * 2;            // 8 KB
    constexpr uint32_t kBPiece = kS2Kmax * RB;               // 6 KB
    constexpr uint32_t kBOff = PC * kAPiece;                 // B pieces follow the A pieces
    const int S = L.stages, KC1 = L.kc1, NH = L.nh;
    const bool contig = args.contiguous != 0;
    const int i_beg = contig ? (int)((long)L.n_items * blockIdx.x / gridDim.x) : (int)blockIdx.x;
    const int i_end = contig ? (int)((long)L.n_items * (blockIdx.x + 1) / gridDim.x) : L.n_items;
    const int i_step = contig ? 1 : (int)gridDim.x;

    if (threadIdx.x == 0) {
        for (int b = 0; b < S; ++b) {
            mbar_init(&sm->full[b], 33);
            mbar_init(&sm->empty[b], 1);
        }
        mbar_init(&sm->t_full, 1);
        mbar_init(&sm->t_empty, kEpiWarps * 32);
        mbar_init(&sm->tsplit, kEpiWarps * 32);
        mbar_init(&sm->tbuf_free, 1);
        mbar_init(&sm->p_full, 1);
        mbar_init(&sm->p_empty, kEpiWarps * 32);
        for (int sl = 0; sl < 2; ++sl) {
            mbar_init(&sm->tinv_full[sl], kEpiWarps * 32);
            mbar_init(&sm->tinv_empty[sl], kEpiWarps * 32);
        }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        sm->wait_ns = args.wait_ns ? args.wait_ns : kWaitNs;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kEpiWarps + kProdWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&sm->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;
    auto stage_base = [&](int b) -> uint8_t* { return ring + (size_t)b * L.stage_bytes; };
    auto tbuf = [&](int c2, int pc) -> uint8_t* { return ring + L.tbuf_off + (size_t)(c2 * PC + pc) * kAPiece; };
    auto k16_of = [&](int item) -> int { return __ldg(args.s2_k16 + (__ldg(args.tile_k + item) & 0xFFFF)); };

    if (warp >= kEpiWarps && warp < kEpiWarps + kS2Prod) {
        // ================= producers =================
        const int pw = warp - kEpiWarps;
        constexpr int CPR = CH / 8, RPI = 32 / CPR, NR = kTileM / RPI;
        const int cch = lane % CPR, rl = lane / CPR;
        int it = 0;
        bool ok = true;
        // stages in the MMA thread's order: GEMM 1 of every tile, and (with
        // EW = 8) GEMM 1 of tile s + 1 before GEMM 2 of tile s
        auto produce = [&](int item, bool first_gemm) {
            const int group = __ldg(args.tile_k + item) & 0xFFFF;
            const int k16 = __ldg(args.s2_k16 + group);
            const int nst = first_gemm ? KC1 : ((k16 + 31) / 32) * NH;
            int srow[NR];
            if (first_gemm) {
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const int r = __ldg(args.row_src + (long)item * kTileM + rl + RPI * i);
                    srow[i] = r < 0 ? args.zero_row : r;
                }
            }
            for (int j = 0; j < nst && ok; ++j, ++it) {
                if (it % kS2Prod != pw) continue;
                const int b = it % S;
                const uint32_t ph = (uint32_t)(it / S) & 1u;
                if (!mbar_wait(&sm->empty[b], ph ^ 1u, sm, args.error_flag)) {
                    ok = false;
                    break;
                }
                uint8_t* sb = stage_base(b);
                if (first_gemm) {
                    const int col = j * CH + cch * 8;
                    const uint32_t bytes = col < args.kdim ? 16u : 0u;
                    const int colc = col < args.kdim ? col : 0;
#pragma unroll
                    for (int pc = 0; pc < PC; ++pc) {
                        const __nv_bfloat16* base = args.A + pc * args.a_piece_stride + colc;
                        const uint32_t sa = smem_u32(sb + pc * kAPiece);
#pragma unroll
                        for (int i = 0; i < NR; ++i)
                            cp_async16(sa + swz<CH>(rl + RPI * i, cch), base + (long)srow[i] * args.kdim, bytes);
                    }
                    if (lane == 0) {
                        mbar_arrive_expect_tx(&sm->full[b], (uint32_t)(PC * k16 * RB));
                        for (int pc = 0; pc < PC; ++pc)
                            for (int rb = 0; rb < k16; rb += 16)
                                tma_load_2d(smem_u32(sb + kBOff + pc * kBPiece + rb * RB), &vmap, j * CH,
                                            (pc * KIFMM_N_OFFSETS + group) * kS2Kmax + rb, &sm->full[b]);
                    }
                    // the lanes arrive as their copies land (the MMA thread
                    // fences them into the async proxy), so a warp keeps
                    // several stages in flight
                    cp_async_mbar_arrive(&sm->full[b]);
                } else {
                    const int c2 = j / NH, h = j % NH;
                    if (lane == 0) {
                        mbar_arrive_expect_tx(&sm->full[b], (uint32_t)(PC * kBPiece));
                        for (int pc = 0; pc < PC; ++pc)
                            tma_load_2d(smem_u32(sb + kBOff + pc * kBPiece), &umap, c2 * CH,
                                        (pc * KIFMM_N_OFFSETS + group) * args.ndim + h * kS2Part, &sm->full[b]);
                    }
                    mbar_arrive(&sm->full[b]);
                }
            }
        };
        if (EW == 8) {
            if (i_beg < i_end) produce(i_beg, true);
            for (int item = i_beg; item < i_end && ok; item += i_step) {
                if (item + i_step < i_end) produce(item + i_step, true);
                if (ok) produce(item, false);
            }
        } else {
            for (int item = i_beg; item < i_end && ok; item += i_step) {
                produce(item, true);
                if (ok) produce(item, false);
            }
        }
        cp_async_wait_0();
        if (!ok && lane == 0) {
            const unsigned long long t0 = global_ns();
            while (global_ns() - t0 < 1000000ull) {
            }
        }
    } else if (warp == kEpiWarps + kProdWarps) {
        // ================= MMA issuer =================
        if (lane == 0) {
            const uint64_t ring_desc = umma_desc<CH>(smem_u32(ring));
            const uint32_t stage_u = L.stage_bytes >> 4, a_u = kAPiece >> 4, bo_u = kBOff >> 4, bp_u = kBPiece >> 4;
            const uint64_t tdesc = umma_desc<CH>(smem_u32(ring + L.tbuf_off));
            int b = 0;
            uint32_t ph = 0;
            bool ok = true;
            constexpr int8_t kA[6] = {2, 1, 0, 1, 0, 0}, kB[6] = {0, 1, 2, 0, 1, 0};
            auto gemm1 = [&](int item, int ic) -> bool {
                const int k16 = k16_of(item);
                // first GEMM: T = Q~ Vhat^T
                if (!mbar_wait(&sm->t_empty, (uint32_t)(ic & 1) ^ 1u, sm, args.error_flag)) return false;
                tc_fence_after();
                const uint32_t idT = umma_idesc(k16, args.f16);
                const uint32_t d_hi = tmem, d_lo = HILO ? tmem + (uint32_t)kS2Kmax : tmem;
                bool hi_on = false, lo_on = false;
                for (int kc = 0; kc < KC1; ++kc) {
                    if (!mbar_wait(&sm->full[b], ph, sm, args.error_flag)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();  // cp.async data -> tensor-core reads
                    tc_fence_after();
                    const uint64_t sd = ring_desc + (uint64_t)((uint32_t)b * stage_u);
                    if (args.kdim - kc * CH >= 32) {
#pragma unroll
                        for (int pi = P0; pi < 6; ++pi) {
                            const bool to_hi = (kA[pi] == 0 && kB[pi] == 0) || !HILO;
                            const uint32_t d = to_hi ? d_hi : d_lo;
                            const uint64_t ad = sd + (uint64_t)(kA[pi] * a_u), bd = sd + (uint64_t)(bo_u + kB[pi] * bp_u);
                            umma_bf16(d, ad, bd, idT, (to_hi ? hi_on : lo_on) ? 1u : 0u);
                            umma_bf16(d, ad + 2, bd + 2, idT, 1u);
                            hi_on = hi_on || to_hi;
                            lo_on = lo_on || !to_hi;
                        }
                    } else {
#pragma unroll
                        for (int pi = P0; pi < 6; ++pi) {
                            const bool to_hi = (kA[pi] == 0 && kB[pi] == 0) || !HILO;
                            const uint32_t d = to_hi ? d_hi : d_lo;
                            const uint64_t ad = sd + (uint64_t)(kA[pi] * a_u), bd = sd + (uint64_t)(bo_u + kB[pi] * bp_u);
                            umma_bf16(d, ad, bd, idT, (to_hi ? hi_on : lo_on) ? 1u : 0u);
                            hi_on = hi_on || to_hi;
                            lo_on = lo_on || !to_hi;
                        }
                    }
                    umma_commit(&sm->empty[b]);
                    if (++b == S) {
                        b = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) return false;
                umma_commit(&sm->t_full);
                return true;
            };
            auto gemm2 = [&](int item, int ic) -> bool {
                const int k16 = k16_of(item);
                const int nc2 = (k16 + 31) / 32;
                // second GEMM: P = T Uhat^T, T pieces from shared memory
                if (!mbar_wait(&sm->tsplit, (uint32_t)(ic & 1), sm, args.error_flag) ||
                    !mbar_wait(&sm->p_empty, (uint32_t)(ic & 1) ^ 1u, sm, args.error_flag))
                    return false;
                tc_fence_after();
                uint32_t p_on = 0;  // bit h: part h of P has been written
                for (int c2 = 0; c2 < nc2 && ok; ++c2) {
                    const bool two = k16 - c2 * CH >= 32;
                    for (int h = 0; h < NH; ++h) {
                        if (!mbar_wait(&sm->full[b], ph, sm, args.error_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int nh_cols = min(kS2Part, args.ndim - h * kS2Part);
                        const uint32_t idP = umma_idesc(nh_cols, args.f16);
                        const uint32_t dP = tmem + (uint32_t)(2 * kS2Kmax + h * kS2Part);
                        const uint64_t sd = ring_desc + (uint64_t)((uint32_t)b * stage_u);
                        const uint64_t td = tdesc + (uint64_t)((uint32_t)(c2 * PC) * a_u);
#pragma unroll
                        for (int pi = P0; pi < 6; ++pi) {
                            const uint64_t ad = td + (uint64_t)(kA[pi] * a_u), bd = sd + (uint64_t)(bo_u + kB[pi] * bp_u);
                            umma_bf16(dP, ad, bd, idP, ((p_on >> h) & 1u) ? 1u : 0u);
                            p_on |= 1u << h;
                            if (two) umma_bf16(dP, ad + 2, bd + 2, idP, 1u);
                        }
                        umma_commit(&sm->empty[b]);
                        if (++b == S) {
                            b = 0;
                            ph ^= 1u;
                        }
                    }
                }
                if (!ok) return false;
                umma_commit(&sm->p_full);
                umma_commit(&sm->tbuf_free);
                return true;
            };
            // EW = 8: GEMM 1 of tile i + 1 runs while the T warps split tile i
            // (they free the TMEM T columns as soon as they have read them)
            int ic = 0;
            if (EW == 8 && i_beg < i_end) ok = gemm1(i_beg, 0);
            for (int item = i_beg; item < i_end && ok; item += i_step, ++ic) {
                if (EW == 8) {
                    if (item + i_step < i_end) ok = gemm1(item + i_step, ic + 1);
                } else {
                    ok = gemm1(item, ic);
                }
                if (ok) ok = gemm2(item, ic);
            }
            umma_commit(&sm->drain);
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&sm->drain, 0u) && global_ns() - t0 < kWaitNs) {
            }
        }
        __syncwarp();
    } else if (warp < kEpiWarps || (EW == 8 && warp >= kEpiWarps + kS2Prod && warp < kEpiWarps + kProdWarps)) {
        // ================= epilogue =================
        // Warp w < 4 and (EW = 8) warp 7-10 read TMEM lane quarter w mod 4,
        // one whole tile row per lane.  With EW = 4 each warp splits T and
        // then drains P, tile after tile.  With EW = 8 the roles run side by
        // side: warps 0-3 split T (and hand each row's power of two to the P
        // warps through a 2-slot ring of shared-memory rows), warps 7-10
        // drain P, so the split of tile i + 1 overlaps the drain of tile i.
        const int q = warp & 3;
        const bool t_role = EW == 4 || warp < kEpiWarps;
        const bool p_role = EW == 4 || warp >= kEpiWarps;
        float* trans = reinterpret_cast<float*>(ring + L.trans_off) + q * 32 * kTransStride;
        float* tinv_rows = reinterpret_cast<float*>(ring + L.tmax_off);  // [2 slots][128 rows]
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int m = q * 32 + lane;  // tile row = TMEM lane
        const bool f16t = NP == 3 && args.f16 != 0;
        int ic = 0;
        bool ok = true;
        for (int item = i_beg; item < i_end && ok; item += i_step, ++ic) {
            const int code = __ldg(args.tile_k + item);
            const int k16 = __ldg(args.s2_k16 + (code & 0xFFFF));
            float tinv = 1.f;
            if (EW == 8 && t_role) {
                // T: TMEM -> registers (hi + lo), the TMEM columns released at
                // once for the next tile's GEMM 1, then pieces in shared memory
                // once GEMM 2 of the previous tile has read them
                bool got = mbar_wait(&sm->t_full, (uint32_t)(ic & 1), sm, args.error_flag);
                if (f16t)
                    got = got && mbar_wait(&sm->tinv_empty[ic & 1], (uint32_t)((ic >> 1) & 1) ^ 1u, sm,
                                           args.error_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                float tv[kS2Kmax];
                float mx = 0.f;
#pragma unroll
                for (int c = 0; c < kS2Kmax; c += 16) {
                    if (c < k16) {
                        uint32_t r[16], r2[16];
                        tmem_ld8(tmem + lane_base + (uint32_t)c, r);
                        tmem_ld8(tmem + lane_base + (uint32_t)(c + 8), r + 8);
                        if (HILO) {
                            tmem_ld8(tmem + lane_base + (uint32_t)(kS2Kmax + c), r2);
                            tmem_ld8(tmem + lane_base + (uint32_t)(kS2Kmax + c + 8), r2 + 8);
                        }
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            tv[c + j] = __uint_as_float(r[j]) + (HILO ? __uint_as_float(r2[j]) : 0.f);
                            mx = fmaxf(mx, fabsf(tv[c + j]));
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) tv[c + j] = 0.f;
                    }
                }
                tc_fence_before();
                mbar_arrive(&sm->t_empty);
                float tsc = 1.f;
                if (f16t) {
                    int e = mx > 0.f ? ((__float_as_int(mx) >> 23) & 0xFF) - 127 : 0;
                    e = max(-112, min(127, e));  // tsc and tinv both normal powers of two
                    tsc = __int_as_float((127 + 14 - e) << 23);
                    tinv = __int_as_float((127 + e - 14) << 23);
                }
                if (!__all_sync(0xffffffffu,
                                mbar_wait(&sm->tbuf_free, (uint32_t)(ic & 1) ^ 1u, sm, args.error_flag))) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int c = 0; c < kS2Kmax; c += 32) {
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        if (c + 8 * qq < k16) {
                            uint32_t pk[3][4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float x = tv[c + 8 * qq + 2 * e], y = tv[c + 8 * qq + 2 * e + 1];
                                uint32_t hh[3];
                                if (f16t) {
                                    const float xs = x * tsc, ys = y * tsc;
                                    const __half2 h = __floats2half2_rn(xs, ys);
                                    const __half2 l = __floats2half2_rn(xs - __low2float(h), ys - __high2float(h));
                                    hh[0] = *reinterpret_cast<const uint32_t*>(&h);
                                    hh[1] = *reinterpret_cast<const uint32_t*>(&l);
                                    hh[2] = 0u;
                                } else {
                                    split3x2(x, y, hh, PC);
                                }
#pragma unroll
                                for (int pc = 0; pc < 3; ++pc) pk[pc][e] = hh[pc];
                            }
#pragma unroll
                            for (int pc = 0; pc < PC; ++pc)
                                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                                                 smem_u32(tbuf(c / 32, pc)) + swz<CH>(m, qq)),
                                             "r"(pk[pc][0]), "r"(pk[pc][1]), "r"(pk[pc][2]), "r"(pk[pc][3])
                                             : "memory");
                        }
                    }
                }
                fence_proxy_async();
                mbar_arrive(&sm->tsplit);
                if (f16t) {
                    tinv_rows[(ic & 1) * kTileM + m] = tinv;
                    mbar_arrive(&sm->tinv_full[ic & 1]);
                }
            } else if (t_role) {
                // T: TMEM -> hi + lo -> pieces in shared memory
                bool got = mbar_wait(&sm->tbuf_free, (uint32_t)(ic & 1) ^ 1u, sm, args.error_flag);
                got = got && mbar_wait(&sm->t_full, (uint32_t)(ic & 1), sm, args.error_flag);
                if (EW == 8 && f16t)
                    got = got && mbar_wait(&sm->tinv_empty[ic & 1], (uint32_t)((ic >> 1) & 1) ^ 1u, sm,
                                           args.error_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // FP16 pieces (f16x3): this row of T scaled by the power of two
                // tsc that puts its largest entry in [2^14, 2^15), undone by
                // tinv on the row of P
                float tsc = 1.f;
                if (f16t) {
                    float mx = 0.f;
                    for (int c = 0; c < k16; c += 16) {
                        uint32_t r[32], r2[32];
                        tmem_ld16(tmem + lane_base + (uint32_t)c, r);
                        tmem_ld16(tmem + lane_base + (uint32_t)(kS2Kmax + c), r2);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            mx = fmaxf(mx, fabsf(__uint_as_float(r[j]) + __uint_as_float(r2[j])));
                    }
                    int e = mx > 0.f ? ((__float_as_int(mx) >> 23) & 0xFF) - 127 : 0;
                    e = max(-112, min(127, e));  // tsc and tinv both normal powers of two
                    tsc = __int_as_float((127 + 14 - e) << 23);
                    tinv = __int_as_float((127 + e - 14) << 23);
                }
                for (int c = 0; c < k16; c += 32) {
                    uint32_t r[32], r2[32];
                    const bool full32 = c + 32 <= k16;
                    if (full32) tmem_ld32(tmem + lane_base + (uint32_t)c, r);
                    else tmem_ld16(tmem + lane_base + (uint32_t)c, r);
                    if (HILO) {
                        if (full32) tmem_ld32(tmem + lane_base + (uint32_t)(kS2Kmax + c), r2);
                        else tmem_ld16(tmem + lane_base + (uint32_t)(kS2Kmax + c), r2);
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        if (!full32 && qq >= 2) break;
                        uint32_t pk[3][4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float x = __uint_as_float(r[8 * qq + 2 * e]), y = __uint_as_float(r[8 * qq + 2 * e + 1]);
                            if (HILO) {
                                x += __uint_as_float(r2[8 * qq + 2 * e]);
                                y += __uint_as_float(r2[8 * qq + 2 * e + 1]);
                            }
                            uint32_t hh[3];
                            if (f16t) {
                                const float xs = x * tsc, ys = y * tsc;
                                const __half2 h = __floats2half2_rn(xs, ys);
                                const __half2 l = __floats2half2_rn(xs - __low2float(h), ys - __high2float(h));
                                hh[0] = *reinterpret_cast<const uint32_t*>(&h);
                                hh[1] = *reinterpret_cast<const uint32_t*>(&l);
                                hh[2] = 0u;
                            } else {
                                split3x2(x, y, hh, PC);
                            }
#pragma unroll
                            for (int pc = 0; pc < 3; ++pc) pk[pc][e] = hh[pc];
                        }
#pragma unroll
                        for (int pc = 0; pc < PC; ++pc)
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(tbuf(c / 32, pc)) +
                                                                                            swz<CH>(m, qq)),
                                         "r"(pk[pc][0]), "r"(pk[pc][1]), "r"(pk[pc][2]), "r"(pk[pc][3])
                                         : "memory");
                    }
                }
                tc_fence_before();
                mbar_arrive(&sm->t_empty);
                fence_proxy_async();
                mbar_arrive(&sm->tsplit);
                if (EW == 8 && f16t) {
                    tinv_rows[(ic & 1) * kTileM + m] = tinv;
                    mbar_arrive(&sm->tinv_full[ic & 1]);
                }
            }
            if (p_role) {
                // P: TMEM -> transpose -> reductions into p~
                const long orow = __ldg(args.row_dst + (long)item * kTileM + m);
                const float oscale =
                    args.scale_table ? __ldg(args.scale_table + (code >> 16)) : args.level_scale[(code >> 16) & 31];
                // this row's factor besides s_l: the FP16 scaling of its q~ row
                // (row_scale) and of its T row (tinv)
                float qf = 1.f;
                if (args.row_scale) {
                    const int sr = __ldg(args.row_src + (long)item * kTileM + m);
                    qf = sr >= 0 ? __ldg(args.row_scale + sr) : 0.f;
                }
                bool got = true;
                if (EW == 8 && f16t) {
                    got = mbar_wait(&sm->tinv_full[ic & 1], (uint32_t)(ic >> 1) & 1u, sm, args.error_flag);
                    if (got) {
                        tinv = tinv_rows[(ic & 1) * kTileM + m];
                        mbar_arrive(&sm->tinv_empty[ic & 1]);
                    }
                }
                got = got && mbar_wait(&sm->p_full, (uint32_t)(ic & 1), sm, args.error_flag);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const float rowf = qf * tinv;
                long prow[8];
#pragma unroll
                for (int pass = 0; pass < 8; ++pass) prow[pass] = __shfl_sync(0xffffffffu, orow, pass * 4 + lane / 8);
                const int c4 = lane % 8;
                for (int c = 0; c < args.ndim; c += 32) {
                    uint32_t r[32];
                    const bool full32 = c + 32 <= args.ndim;
                    const uint32_t a0 = tmem + lane_base + (uint32_t)(2 * kS2Kmax + c);
                    if (full32) tmem_ld32(a0, r);
                    else tmem_ld16(a0, r);
                    tmem_wait_ld();
#pragma unroll
                    for (int qv = 0; qv < 8; ++qv)
                        *reinterpret_cast<float4*>(trans + lane * kTransStride + 4 * qv) =
                            make_float4(rowf * __uint_as_float(r[4 * qv]), rowf * __uint_as_float(r[4 * qv + 1]),
                                        rowf * __uint_as_float(r[4 * qv + 2]), rowf * __uint_as_float(r[4 * qv + 3]));
                    __syncwarp();
                    const int ncols = full32 ? 32 : 16;
#pragma unroll
                    for (int pass = 0; pass < 8; ++pass) {
                        const int rr = pass * 4 + lane / 8;
                        const long grow = prow[pass];
                        if (grow < 0 || 4 * c4 >= ncols) continue;
                        const float4 x = *reinterpret_cast<const float4*>(trans + rr * kTransStride + 4 * c4);
                        red_add_v4(args.D + grow * args.ldd + c + 4 * c4, __float_as_uint(oscale * x.x),
                                   __float_as_uint(oscale * x.y), __float_as_uint(oscale * x.z),
                                   __float_as_uint(oscale * x.w));
                    }
                    __syncwarp();
                }
                tc_fence_before();
                mbar_arrive(&sm->p_empty);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kEpiWarps + kProdWarps) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Host-side state cached across launches (the per-call host work is a
// visible share of a small level's apply): the largest dynamic shared memory
// already granted to each kernel instantiation on each device, each device's
// opt-in limit, and encoded tensor maps of the B operands.
std::mutex g_cache_mutex;
int g_smem_granted[10][64] = {};
int g_max_smem[64] = {};
struct MapKey {
    const void* ptr;
    int rows, kdim, ch, box_rows;
    bool operator<(const MapKey& o) const {
        if (ptr != o.ptr) return ptr < o.ptr;
        if (rows != o.rows) return rows < o.rows;
        if (kdim != o.kdim) return kdim < o.kdim;
        if (ch != o.ch) return ch < o.ch;
        return box_rows < o.box_rows;
    }
};

std::map<MapKey, CUtensorMap> g_maps;

// A BF16 matrix viewed as a 2D tensor [rows][cols], boxes of ch x box_rows,
// 64-byte (ch = 32) or 32-byte (ch = 16) swizzle.
cudaError_t get_map2d(const __nv_bfloat16* ptr, cuuint64_t rows, int cols, int ch, int box_rows,
                      EncodeTiledFn encode, CUtensorMap* out) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    const MapKey key{ptr, (int)rows, cols, ch, box_rows};
    auto it = g_maps.find(key);
    if (it != g_maps.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    const cuuint64_t gdim[2] = {(cuuint64_t)cols, rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)ch, (cuuint32_t)box_rows};
    const cuuint32_t estride[2] = {1, 1};
    CUresult cr = encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), gdim, gstride, box,
                         estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         ch == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    if (g_maps.size() > 256) g_maps.clear();
    g_maps.emplace(key, *out);
    return cudaSuccess;
}

// B pieces viewed as a 2D tensor [rows_total][kdim].
cudaError_t get_bmap(const UmmaArgs& a, cuuint64_t rows_total, int ch, int box_rows, EncodeTiledFn encode,
                     CUtensorMap* out) {
    return get_map2d(a.B, rows_total, a.kdim, ch, box_rows, encode, out);
}

template <int AM, int EM>
cudaError_t launch_t(const CUtensorMap& bmap, const CUtensorMap& amap, const UmmaArgs& a, const Layout& L, size_t smem,
                     int grid, cudaStream_t stream, int dev) {
    const int inst = AM == A_GATHER ? (EM == E_RED ? 0 : (EM == E_STORE ? 7 : 8)) : (EM == E_STORE ? 1 : 2);
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        if (g_smem_granted[inst][dev] < (int)smem) {
            cudaError_t e =
                cudaFuncSetAttribute(umma_kernel<AM, EM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            g_smem_granted[inst][dev] = (int)smem;
        }
    }
    umma_kernel<AM, EM><<<grid, kThreads, smem, stream>>>(bmap, amap, a, L);
    return cudaGetLastError();
}

// The A-resident core (split6 with hilo); cudaErrorNotSupported when the
// A tile or the B ring does not fit in shared memory.
cudaError_t launch_core_resident(const UmmaArgs& a, int num_sms, cudaStream_t stream, EncodeTiledFn encode) {
    if (a.n_products != 6 || !a.hilo) return cudaErrorNotSupported;
    const int KC = (a.kdim + 31) / 32;
    if (KC > kResMaxKC) return cudaErrorNotSupported;
    // N blocks: two slots of hi + lo (4 BN columns) fit in 512
    int nb = 1, bn = (a.ndim + 15) / 16 * 16;
    while (4 * bn > 512) {
        ++nb;
        bn = ((a.ndim + nb - 1) / nb + 15) / 16 * 16;
    }
    int dev = 0, max_smem = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return ce;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        if (!g_max_smem[dev]) {
            ce = cudaDeviceGetAttribute(&g_max_smem[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            if (ce != cudaSuccess) return ce;
        }
        max_smem = g_max_smem[dev];
    }
    RLayout L{};
    L.kc_count = KC;
    L.nb = nb;
    L.bn = bn;
    L.n_items = a.n_tiles;
    const uint32_t a_bytes = (uint32_t)KC * 3u * (uint32_t)(kTileM * 32 * 2);
    const uint32_t trans_bytes = kEpiWarps * 32 * kTransStride * 4;
    L.b_off = a_bytes;
    L.b_piece_bytes = (uint32_t)bn * 64u;
    const long avail = (long)max_smem - 2048 - (long)a_bytes - (long)trans_bytes;
    int sb = (int)(avail / (long)(3u * L.b_piece_bytes));
    if (sb > kResMaxSB) sb = kResMaxSB;
    if (sb < 2) return cudaErrorNotSupported;
    L.sb = sb;
    L.trans_off = a_bytes + (uint32_t)sb * 3u * L.b_piece_bytes;
    if (L.n_items <= 0) return cudaSuccess;
    const size_t smem = 2048 + (size_t)L.trans_off + trans_bytes;
    CUtensorMap bmap;
    ce = get_bmap(a, (cuuint64_t)3 * a.b_groups * a.ndim, 32, bn, encode, &bmap);
    if (ce != cudaSuccess) return ce;
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        if (g_smem_granted[3][dev] < (int)smem) {
            ce = cudaFuncSetAttribute(core_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (ce != cudaSuccess) return ce;
            g_smem_granted[3][dev] = (int)smem;
        }
    }
    const int grid = num_sms < L.n_items ? num_sms : L.n_items;
    core_resident_kernel<<<grid, kThreads, smem, stream>>>(bmap, a, L);
    return cudaGetLastError();
}

// The stage-2 core (Sec. 3.2).
cudaError_t launch_core_stage2(const UmmaArgs& a, int num_sms, cudaStream_t stream, EncodeTiledFn encode) {
    if (!a.s2_V || !a.s2_U || !a.s2_k16) return cudaErrorInvalidValue;
    if (a.ndim % 16 != 0 || a.ndim < 16 || a.ndim > 512 - 2 * kS2Kmax || a.kdim % 16 != 0 || a.kdim <= 0)
        return cudaErrorInvalidValue;
    int dev = 0, max_smem = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return ce;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        if (!g_max_smem[dev]) {
            ce = cudaDeviceGetAttribute(&g_max_smem[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            if (ce != cudaSuccess) return ce;
        }
        max_smem = g_max_smem[dev];
    }
    S2Layout L{};
    L.kc1 = (a.kdim + 31) / 32;
    L.nh = (a.ndim + kS2Part - 1) / kS2Part;
    L.n_items = a.n_tiles;
    const uint32_t pc = a.n_products == 6 ? 3u : (a.n_products == 3 ? 2u : 1u);  // pieces
    L.stage_bytes = pc * (kTileM * 32u * 2u + kS2Kmax * 64u);
    // the fixed part: T pieces, transpose buffers, T row maxima; the ring
    // takes the rest (3 to kS2MaxStages stages)
    const uint32_t fixed = 3u * pc * kTileM * 32u * 2u + kEpiWarps * 32 * kTransStride * 4 + 2u * kTileM * 4u;
    L.stages = (int)std::min<long>(kS2MaxStages, ((long)max_smem - 2048 - (long)fixed) / (long)L.stage_bytes);
    if (L.stages < kS2Prod) return cudaErrorInvalidConfiguration;
    L.tbuf_off = (uint32_t)L.stages * L.stage_bytes;
    L.trans_off = L.tbuf_off + 3u * pc * kTileM * 32u * 2u;
    L.tmax_off = L.trans_off + kEpiWarps * 32 * kTransStride * 4;
    const size_t smem = 2048 + (size_t)L.tmax_off + 2u * kTileM * 4u;
    if ((long)smem > (long)max_smem) return cudaErrorInvalidConfiguration;
    if (L.n_items <= 0) return cudaSuccess;
    CUtensorMap vmap, umap;
    ce = get_map2d(a.s2_V, (cuuint64_t)3 * kOffsetsHost * kS2Kmax, a.kdim, 32, 16, encode, &vmap);
    if (ce != cudaSuccess) return ce;
    ce = get_map2d(a.s2_U, (cuuint64_t)3 * kOffsetsHost * a.ndim, kS2Kmax, 32, kS2Part, encode, &umap);
    if (ce != cudaSuccess) return ce;
    const int grid = num_sms < L.n_items ? num_sms : L.n_items;
    auto go = [&](auto kern, int slot) -> cudaError_t {
        {
            std::lock_guard<std::mutex> lock(g_cache_mutex);
            if (g_smem_granted[slot][dev] < (int)smem) {
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                g_smem_granted[slot][dev] = (int)smem;
            }
        }
        // round-robin tiles: the per-offset ranks k_o make tile costs uneven
        // along the offset-major list, so contiguous runs would not balance
        UmmaArgs b = a;
        b.contiguous = 0;
        kern<<<grid, kThreads, smem, stream>>>(vmap, umap, b, L);
        return cudaGetLastError();
    };
    if (a.n_products == 6) return go(core_stage2_kernel<6>, 4);
    if (a.n_products == 3) return go(core_stage2_kernel<3>, 5);
    return go(core_stage2_kernel<1>, 6);
}

}  // namespace

cudaError_t tma_map_2d(const void* ptr, uint64_t rows, int cols, int ch, int box_rows, CUtensorMap* out) {
    EncodeTiledFn encode = get_encode_fn();
    if (!encode) return cudaErrorNotSupported;
    return get_map2d(static_cast<const __nv_bfloat16*>(ptr), (cuuint64_t)rows, cols, ch, box_rows, encode, out);
}

cudaError_t launch_umma(int amode, int emode, const UmmaArgs& a, int num_sms, cudaStream_t stream) {
    if (a.kdim % 16 != 0 || a.kdim <= 0 || a.ndim % 16 != 0 || a.ndim < 16 || a.n_chunk % 16 != 0 ||
        a.n_chunk < 16 || a.n_chunk > 512)
        return cudaErrorInvalidValue;
    if (a.n_products != 1 && a.n_products != 3 && a.n_products != 6) return cudaErrorInvalidValue;
    const bool gather = amode == A_GATHER;
    if (!((gather && (emode == E_RED || a.row_identity)) || (!gather && (emode == E_STORE || emode == E_SPLIT))))
        return cudaErrorInvalidValue;
    if (!gather && (a.k_valid % 4 != 0 || a.lda % 4 != 0 || a.k_valid > a.kdim)) return cudaErrorInvalidValue;
    if (a.ldd % 4 != 0) return cudaErrorInvalidValue;
    EncodeTiledFn encode = get_encode_fn();
    if (!encode) return cudaErrorNotSupported;
    // FP16 operands and per-row factors: the gather kernel's classic and drain
    // paths and the 3-product stage-2 core only
    if ((a.f16 || a.row_scale) && (!gather || (a.s2_on && a.n_products != 3) || (a.row_scale && emode != E_RED)))
        return cudaErrorNotSupported;
    if (gather && a.s2_on) return launch_core_stage2(a, num_sms, stream, encode);
    if (gather && a.core_resident && !a.f16 && !a.row_scale) {
        const cudaError_t e = launch_core_resident(a, num_sms, stream, encode);
        if (e != cudaErrorNotSupported) return e;
    }

    Layout L{};
    L.na = a.n_products == 1 ? 1 : (a.n_products == 3 ? 2 : 3);
    L.nc = L.na;
    L.n_chunks = (a.ndim + a.n_chunk - 1) / a.n_chunk;
    const int ch = chunk_of(amode);
    L.kc_count = (a.kdim + ch - 1) / ch;
    L.c_rows_alloc = (a.n_chunk + kCBoxRows - 1) / kCBoxRows * kCBoxRows;
    L.a_bytes = kTileM * ch * 2;
    L.c_bytes = (uint32_t)L.c_rows_alloc * ch * 2;
    L.stage_bytes = (uint32_t)L.na * L.a_bytes + (uint32_t)L.nc * L.c_bytes;
    if (gather) {
        L.acc_cols = a.n_chunk * ((a.hilo && a.n_products > 1) ? 2 : 1);
        if (L.acc_cols > 512) return cudaErrorInvalidValue;
        L.n_acc = 2 * L.acc_cols <= 512 ? 2 : 1;
    } else {
        // two partial slots + two lo slots, partial sums of <= 96 columns in registers
        if (a.n_chunk > kMaxRowsChunk) return cudaErrorInvalidValue;
        L.acc_cols = a.n_chunk;
        L.n_acc = 2;
    }
    const long row_tiles = gather ? a.n_tiles : (a.n_segs > 0 ? (long)a.seg_tiles : ((long)a.m_rows + kTileM - 1) / kTileM);
    if (gather && a.row_identity && a.n_tiles != (a.n_segs > 0 ? a.seg_tiles : (a.m_rows + kTileM - 1) / kTileM))
        return cudaErrorInvalidValue;
    if (row_tiles * L.n_chunks > INT32_MAX) return cudaErrorInvalidValue;
    L.n_items = (int)(row_tiles * L.n_chunks);
    if (L.n_items <= 0) return cudaSuccess;

    int dev = 0, max_smem = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return ce;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        if (!g_max_smem[dev]) {
            ce = cudaDeviceGetAttribute(&g_max_smem[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            if (ce != cudaSuccess) return ce;
        }
        max_smem = g_max_smem[dev];
    }
    if (gather && emode == E_RED && a.core_bres && !a.row_identity) {
        const cudaError_t e = launch_core_stage(a, num_sms, max_smem, dev, stream);
        if (e != cudaErrorNotSupported) return e;
    }
    // drain mode (split6 core): 8 epilogue warps, which needs at most 3
    // producer warps (= stages) and N <= 192 per item (96 sums per thread)
    L.drain = gather && a.core_drain > 0 && (a.n_products == 6 || a.n_products == 3) && a.n_chunk <= 192
                  ? std::min(a.core_drain, 3)
                  : 0;
    // compression / expansion with hilo: the (0,0) product gets its own half
    // of each partial slot (two slots of 2 N columns in the 512), so a partial
    // may span several K-chunks with only 2 full-magnitude MMAs per chunk;
    // where the slots do not fit, one K-chunk per partial
    L.dhilo = 0;
    if (L.drain && gather && emode != E_RED && a.hilo && a.n_products > 1) {
        if (4 * a.n_chunk <= 512) L.dhilo = 1;
        else L.drain = 1;
    }
    // the drained core that reduces rows straight from registers (direct_rows)
    // needs no transpose buffers: their room goes to the ring
    const bool no_trans = L.drain && gather && emode == E_RED && a.direct_rows;
    uint32_t trans_bytes = no_trans ? 0u : (L.drain ? 2u : 1u) * kEpiWarps * 32 * kTransStride * 4;
    int avail = max_smem - 2048 - (int)trans_bytes;
    L.stages = avail / (int)L.stage_bytes;
    if (L.drain && L.stages < 2) {
        L.drain = 0;
        trans_bytes = kEpiWarps * 32 * kTransStride * 4;
        avail = max_smem - 2048 - (int)trans_bytes;
        L.stages = avail / (int)L.stage_bytes;
    }
    // identity-row gathers (compression / expansion) have only the drained epilogue
    if (gather && emode != E_RED && !L.drain) return cudaErrorNotSupported;
    if (L.stages > 8) L.stages = 8;
    if (L.stages < 2) return cudaErrorInvalidConfiguration;
    // gather mode: producer warps 4-10 (4-6 when warps 7-10 drain), each
    // taking every P-th ring slot with its copies in flight asynchronously
    L.prod_warps = gather ? std::min(L.stages, L.drain ? 3 : kProdWarps) : L.stages;
    L.trans_off = 1024 + (uint32_t)L.stages * L.stage_bytes;
    const size_t smem = 1024 + (size_t)L.trans_off + trans_bytes;

    // B pieces viewed as a 2D tensor [pieces * b_groups * ndim rows][kdim]
    CUtensorMap bmap;
    ce = get_bmap(a, (cuuint64_t)L.nc * a.b_groups * a.ndim, ch, kCBoxRows, encode, &bmap);
    if (ce != cudaSuccess) return ce;

    const int grid = num_sms < L.n_items ? num_sms : L.n_items;
    // identity-row gathers read the A pieces as TMA boxes of 128 rows: the
    // pieces [na][a_rows][kdim] as one 2D tensor
    CUtensorMap amap = bmap;
    L.a_tma = 0;
    if (gather && a.row_identity && a.a_piece_stride % a.kdim == 0) {
        L.a_rows = (int)(a.a_piece_stride / a.kdim);
        ce = get_map2d(a.A, (cuuint64_t)L.na * L.a_rows, a.kdim, ch, kTileM, encode, &amap);
        if (ce != cudaSuccess) return ce;
        L.a_tma = 1;
    }
    if (gather && emode == E_STORE) return launch_t<A_GATHER, E_STORE>(bmap, amap, a, L, smem, grid, stream, dev);
    if (gather && emode == E_SPLIT) return launch_t<A_GATHER, E_SPLIT>(bmap, amap, a, L, smem, grid, stream, dev);
    if (gather) return launch_t<A_GATHER, E_RED>(bmap, amap, a, L, smem, grid, stream, dev);
    if (emode == E_STORE) return launch_t<A_ROWS, E_STORE>(bmap, amap, a, L, smem, grid, stream, dev);
    return launch_t<A_ROWS, E_SPLIT>(bmap, amap, a, L, smem, grid, stream, dev);
}

}  // namespace kifmm
