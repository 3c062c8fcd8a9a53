// The core products of the compressed M2L (Sec. 3.1, Eq. (14):
// p~^t += s_l K~_o q~^s over every box pair (t, s = t - o)), with the
// scatter into p~ handed to the TMA unit.
//
// Work: the offset-major tile list of 128 (pair, rhs) rows, split in N parts
// of at most 192 columns, gives (part, tile) items; each CTA takes one
// contiguous run of them, part-major, so consecutive items share the
// offset's K~_o (L2-resident, read by TMA per K stage with the A rows).
//
// Groups: one launch may cover up to kMaxGroups operators at once (the plans
// of a batch: several expansion orders p, or one plan per level for a kernel
// that is not homogeneous).  Each group brings its own q~ pieces, cores K~_o
// (a tensor map of its own), rank, tile list, scale table and p~; the items
// of all groups form one sequence and every CTA takes a contiguous run of
// it whose cost (K-chunks x part width per item) is an equal share of the
// total.  The ring stages and TMEM slots are sized for the widest part.
//
// Arithmetic: A and B as 1 piece (bf16) or 2 pieces (split3, f16x3; the
// products hi*lo and lo*hi before hi*hi), tcgen05.mma kind::f16 with FP32
// accumulation in TMEM.  The products of every 3 K-chunks (18 MMAs of
// K = 16 for 2 pieces) go to one of two TMEM partial slots, which the
// epilogue drains into FP32 registers (round to nearest) while the MMAs fill
// the other slot, so no accumulator chain is longer than 18 MMA steps and
// the tensor pipe never waits for an epilogue that keeps pace.
//
// Epilogue: eight warps (warp w: TMEM lanes 32 (w % 4) .. + 31, column half
// w / 4) add the item's partials in registers, apply the level scale s_l
// (and for f16x3 the source row's power-of-two factor) and write each row
// into a shared-memory staging row; one lane per row then hands the row to
// the TMA unit as one bulk reduction (cp.reduce.async.bulk .add.f32) into
// p~.  The unit performs the scattered adds while the warps move on, at the
// L2 rate of the best register-issued form (8 lanes per 128 contiguous
// bytes) without its shared-memory transposes.
//
// Warp roles (384 threads, one CTA per SM):
//   warps 0-7   epilogue (as above); warp w < 4 issues the bulk reductions of
//               rows 32 w .. + 31 after a named barrier with warp w + 4
//   warps 8-10  producers: a stage belongs to warp 8 + it % P; its lanes
//               gather the A rows (cp.async, 64B swizzle, arriving on the
//               stage's full barrier as they land) and lane 0 loads the
//               stage's K~_o pieces by TMA
//   warp 11     TMEM allocation; lane 0 issues the MMAs
//
// Every wait is bounded (the launch's wait_ns, 2 s by default); on timeout
// the error flag is raised, every role stops, copies, reductions and MMAs in
// flight are waited for, and TMEM is freed.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "kernels.h"
#include "umma_ptx.h"

namespace kifmm {

namespace {

using namespace ptx;

constexpr int kEpiW = 8;                 // epilogue warps
constexpr int kProdW = 3;                // producer warps
constexpr int kMmaW = kEpiW + kProdW;    // TMEM / MMA warp
constexpr int kThr = (kMmaW + 1) * 32;   // 384
constexpr int kMaxS = 8;                 // ring stages
constexpr int kCh = 32;                  // K elements per stage (64-byte rows, 64-byte swizzle)
constexpr int kRowB = 64;                // bytes per shared-memory row of a stage
constexpr int kPieceA = kTileM * kRowB;  // 8 KB: one A piece of one stage
constexpr int kMaxPart = 192;            // N per part of the common kernel (96 running sums per epilogue thread)
constexpr int kMaxPartWide = 224;        // N per part of the wide kernel (112 sums, drained 16 columns at a time)
constexpr int kPartK = 3;                // K-chunks per TMEM partial
constexpr int kOffsetsC = 316;

struct CSmem {
    uint64_t full[kMaxS], empty[kMaxS];
    uint64_t part_full[2], part_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    volatile int abort_flag;
    unsigned long long wait_ns;
};

// One operator of a launch.
struct CGroup {
    const __nv_bfloat16* A;  // q~ pieces: piece 0 [rows][kdim], piece i at A + i * a_piece_stride
    long a_piece_stride;     // elements
    const int* row_src;      // tile t: A rows row_src[128 t + i] (-1: the zero row)
    const int* row_dst;      // tile t: p~ rows row_dst[128 t + i] (-1: none)
    const int* tile_k;       // tile t: offset | (scale index << 16)
    const float* scale_table;  // s_l by scale index (null: the launch's level_scale)
    const float* row_scale;    // f16x3: factor of A row r (null: 1)
    float* D;                  // p~ [*][ldd]
    long ldd;
    long item_beg;   // first item of the group in the launch's item sequence
    long n_items;    // n_parts * n_tiles
    long cost_beg;   // cost of the items before the group
    int cost;        // cost of one item
    int kdim, ndim;  // K (multiple of 16) and N (multiple of 16) of the group's cores
    int kc, n_parts, ni;  // K-chunks, N parts, columns per part (the last may be narrower)
    int box_rows;    // rows per TMA box of K~_o (divides every part width)
    int n_tiles, zero_row;
};

constexpr int kMaxGroups = 8;

struct CParams {
    CUtensorMap map[kMaxGroups];  // K~_o of each group: rows (piece, offset, n), columns k
    CGroup g[kMaxGroups];
    float level_scale[32];        // groups without a scale table
    int n_groups;
    int f16;                      // A and B pieces are FP16 (else BF16)
    long n_items, total_cost;
    int* error_flag;
    unsigned long long wait_ns;
};

struct CLayout {
    int stages, prod, pieces;  // ring stages, producer warps in use, pieces
    int ni;                    // widest part over the groups: TMEM slot width and B rows per stage
    uint32_t stage_bytes;      // pieces * (8 KB of A + ni * 64 of B)
    uint32_t st_stride;        // bytes per staging row: (ni + 4) * 4
};

__device__ __forceinline__ void named_sync(int id, int n) {
    // every participant reaches it: the pair leaves its loop only together
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// First item whose cost offset is >= c (the launch's item count when none).
__device__ __forceinline__ long item_at_cost(const CParams& P, long c) {
    for (int g = 0; g < P.n_groups; ++g) {
        const CGroup& G = P.g[g];
        if (c < G.cost_beg + G.n_items * (long)G.cost) return G.item_beg + (c - G.cost_beg + G.cost - 1) / G.cost;
    }
    return P.n_items;
}

// The group of `item`, searching forward from group g (items only increase).
__device__ __forceinline__ int group_of(const CParams& P, long item, int g) {
    while (g + 1 < P.n_groups && item >= P.g[g + 1].item_beg) ++g;
    return g;
}

// HW: the most columns an epilogue thread holds (parts of at most 2 HW).
template <int HW>
__global__ void __launch_bounds__(kThr, 1) core_stage_kernel(const __grid_constant__ CParams P, const CLayout L) {
    constexpr int RW = HW > 96 ? 16 : 48;  // columns per TMEM drain round
    constexpr bool kHalfStage = HW > 96;   // 64 staging rows (room for a third ring stage)
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    uint8_t* base = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    CSmem* sm = reinterpret_cast<CSmem*>(base);
    uint8_t* ring = base + 1024;
    uint8_t* staging = ring + (size_t)L.stages * L.stage_bytes;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int S = L.stages, NP = L.pieces, NI = L.ni;
    const long i_beg = item_at_cost(P, P.total_cost * blockIdx.x / gridDim.x);
    const long i_end = item_at_cost(P, P.total_cost * (blockIdx.x + 1) / gridDim.x);
    const uint32_t a_bytes = (uint32_t)NP * kPieceA;  // A part of a stage
    const uint32_t b_piece = (uint32_t)NI * kRowB;    // one B piece of a stage

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&sm->full[s], 33);  // 32 producer lanes (cp.async arrivals) + the TMA expect_tx arrival
            mbar_init(&sm->empty[s], 1);  // MMA commit
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&sm->part_full[a], 1);
            mbar_init(&sm->part_empty[a], kEpiW * 32);
        }
        mbar_init(&sm->drain, 1);
        sm->abort_flag = 0;
        sm->wait_ns = P.wait_ns ? P.wait_ns : kWaitNs;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&sm->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;

    if (warp >= kEpiW && warp < kMmaW) {
        // ================= producers =================
        const int pw = warp - kEpiW, PW = L.prod;
        constexpr int CPR = kCh / 8;     // 16-byte chunks per row and stage (4)
        constexpr int RPI = 32 / CPR;    // rows per warp instruction (8)
        constexpr int NR = kTileM / RPI; // rows per lane (16)
        const int cch = lane % CPR, rl = lane / CPR;
        int srow[NR], nrow[NR], ngroup = 0;
        int g = 0, gn = 0;  // group of the current item and of the prefetched one
        auto load_rows = [&](long item) {
            gn = group_of(P, item, gn);
            const CGroup& G = P.g[gn];
            const int t = (int)((item - G.item_beg) % G.n_tiles);
#pragma unroll
            for (int i = 0; i < NR; ++i) nrow[i] = __ldg(G.row_src + (long)t * kTileM + rl + RPI * i);
            ngroup = __ldg(G.tile_k + t) & 0xFFFF;
        };
        bool ok = true;
        long it = 0;
        if (pw < PW && i_beg < i_end) load_rows(i_beg);
        for (long item = i_beg; item < i_end && ok; ++item) {
            g = group_of(P, item, g);
            const CGroup& G = P.g[g];
            const int part = (int)((item - G.item_beg) / G.n_tiles);
            const int nw = min(G.ni, G.ndim - part * G.ni);
            const int KC = G.kc, kdim = G.kdim;
            int k = 0;
            if (pw < PW) {
#pragma unroll
                for (int i = 0; i < NR; ++i) srow[i] = nrow[i] < 0 ? G.zero_row : nrow[i];
                k = ngroup;
                if (item + 1 < i_end) load_rows(item + 1);
            }
            for (int kc = 0; kc < KC; ++kc, ++it) {
                if (pw >= PW || it % PW != pw) continue;
                const int s = (int)(it % S);
                const uint32_t ph = (uint32_t)(it / S) & 1u;
                if (!mbar_wait(&sm->empty[s], ph ^ 1u, sm, P.error_flag)) {
                    ok = false;
                    break;
                }
                const uint32_t st = smem_u32(ring + (size_t)s * L.stage_bytes);
                if (lane == 0) {
                    // the stage's K~_o columns: every piece, this part's rows
                    mbar_arrive_expect_tx(&sm->full[s], (uint32_t)NP * nw * kRowB);
                    for (int pc = 0; pc < NP; ++pc) {
                        const int row0 = (pc * kOffsetsC + k) * G.ndim + part * G.ni;
                        for (int rb = 0; rb < nw; rb += G.box_rows)
                            tma_load_2d(st + a_bytes + pc * b_piece + rb * kRowB, &P.map[g], kc * kCh, row0 + rb,
                                        &sm->full[s]);
                    }
                }
                const int col = kc * kCh + cch * 8;
                const uint32_t bytes = col < kdim ? 16u : 0u;
                const int colc = col < kdim ? col : 0;
                for (int pc = 0; pc < NP; ++pc) {
                    const __nv_bfloat16* src = G.A + pc * G.a_piece_stride + colc;
                    const uint32_t dst = st + pc * kPieceA;
#pragma unroll
                    for (int i = 0; i < NR; ++i)
                        cp_async16(dst + swz<kCh>(rl + RPI * i, cch), src + (long)srow[i] * kdim, bytes);
                }
                cp_async_mbar_arrive(&sm->full[s]);
            }
        }
        cp_async_wait_0();
        if (!ok && lane == 0) {
            // TMA loads of a stage this warp filled may still be in flight
            const unsigned long long t0 = global_ns();
            while (global_ns() - t0 < 1000000ull) {
            }
        }
    } else if (warp == kMmaW) {
        // ================= MMA issuer =================
        if (lane == 0) {
            const uint64_t desc0 = umma_desc<kCh>(smem_u32(ring));
            const uint32_t stage_u = L.stage_bytes >> 4, apiece_u = kPieceA >> 4;
            const uint32_t b_u = a_bytes >> 4, bpiece_u = b_piece >> 4;
            int s = 0, pcount = 0, g = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (long item = i_beg; item < i_end && ok; ++item) {
                g = group_of(P, item, g);
                const CGroup& G = P.g[g];
                const int part = (int)((item - G.item_beg) / G.n_tiles);
                const int nw = min(G.ni, G.ndim - part * G.ni);
                const int KC = G.kc, kdim = G.kdim;
                const uint32_t idesc = umma_idesc(nw, P.f16);
                uint32_t d = tmem;
                for (int kc = 0; kc < KC; ++kc) {
                    const bool p_first = kc % kPartK == 0;
                    if (p_first) {
                        // the partial slot has been drained by the epilogue
                        const int ps = pcount & 1;
                        if (!mbar_wait(&sm->part_empty[ps], ((uint32_t)(pcount >> 1) & 1u) ^ 1u, sm,
                                       P.error_flag)) {
                            ok = false;
                            break;
                        }
                        d = tmem + (uint32_t)(ps * NI);
                    }
                    if (!mbar_wait(&sm->full[s], ph, sm, P.error_flag)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();  // cp.async data -> tensor-core reads
                    tc_fence_after();
                    const uint64_t sd = desc0 + (uint64_t)((uint32_t)s * stage_u);
                    const uint64_t bd = sd + b_u;
                    const bool two = kdim - kc * kCh >= 32;  // K steps of 16 in this chunk: 2 or 1
                    const uint32_t first = p_first ? 0u : 1u;
                    if (NP == 2) {
                        // hi*lo and lo*hi (small terms first), then hi*hi
                        umma_bf16(d, sd + apiece_u, bd, idesc, first);
                        if (two) umma_bf16(d, sd + apiece_u + 2, bd + 2, idesc, 1u);
                        umma_bf16(d, sd, bd + bpiece_u, idesc, 1u);
                        if (two) umma_bf16(d, sd + 2, bd + bpiece_u + 2, idesc, 1u);
                        umma_bf16(d, sd, bd, idesc, 1u);
                        if (two) umma_bf16(d, sd + 2, bd + 2, idesc, 1u);
                    } else {
                        umma_bf16(d, sd, bd, idesc, first);
                        if (two) umma_bf16(d, sd + 2, bd + 2, idesc, 1u);
                    }
                    umma_commit(&sm->empty[s]);
                    if (kc % kPartK == kPartK - 1 || kc == KC - 1) {
                        umma_commit(&sm->part_full[pcount & 1]);
                        ++pcount;
                    }
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            // cleanup (fixed bound): every MMA issued has completed before
            // TMEM is released
            umma_commit(&sm->drain);
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&sm->drain, 0u) && global_ns() - t0 < kWaitNs) {
            }
        }
        __syncwarp();
    } else {
        // ================= epilogue =================
        const int q = warp & 3, half = warp >> 2;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        // the wide kernel stages 64 rows: lane quarters q and q ^ 2 share rows
        uint8_t* my_row = staging + (size_t)((kHalfStage ? (q & 1) : q) * 32 + lane) * L.st_stride;
        int pcount = 0, g = 0, gn = 0;
        bool ok = true;
        long nx_row = -1;
        float nx_f = 1.f;
        // the next item's output row and factor s_l (times the f16x3 row factor)
        auto fetch = [&](long item) {
            gn = group_of(P, item, gn);
            const CGroup& G = P.g[gn];
            const int t = (int)((item - G.item_beg) % G.n_tiles);
            const long r = (long)t * kTileM + q * 32 + lane;
            nx_row = __ldg(G.row_dst + r);
            const int k = __ldg(G.tile_k + t);
            float rs = 1.f;
            if (G.row_scale) {
                const int sr = __ldg(G.row_src + r);
                rs = sr >= 0 ? __ldg(G.row_scale + sr) : 0.f;
            }
            nx_f = (G.scale_table ? __ldg(G.scale_table + (k >> 16)) : P.level_scale[(k >> 16) & 31]) * rs;
        };
        if (i_beg < i_end) fetch(i_beg);
        for (long item = i_beg; item < i_end && ok; ++item) {
            g = group_of(P, item, g);
            const CGroup& G = P.g[g];
            const long orow = nx_row;
            const float f = nx_f;
            if (item + 1 < i_end) fetch(item + 1);
            const int part = (int)((item - G.item_beg) / G.n_tiles);
            const int nw = min(G.ni, G.ndim - part * G.ni);
            const int KC = G.kc;
            const int hw = nw / 2;  // columns of this warp (a multiple of 8, <= HW)
            const int c_beg = half * hw;
            // partials -> FP32 running sums, RW columns per TMEM round
            float sums[HW];
#pragma unroll
            for (int j = 0; j < HW; ++j) sums[j] = 0.f;
            bool got = true;
            for (int kc = 0; kc < KC; kc += kPartK) {
                const int ps = pcount & 1;
                got = __all_sync(0xffffffffu, mbar_wait(&sm->part_full[ps], (uint32_t)(pcount >> 1) & 1u, sm,
                                                        P.error_flag));
                if (!got) break;
                tc_fence_after();
                const uint32_t col = tmem + lane_base + (uint32_t)(ps * NI + c_beg);
#pragma unroll
                for (int r0 = 0; r0 < HW; r0 += RW) {
                    if (r0 < hw) {
                        uint32_t v[RW];
#pragma unroll
                        for (int c = 0; c < RW; c += 8)
                            if (r0 + c < hw) tmem_ld8(col + (uint32_t)(r0 + c), v + c);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < RW; ++j)
                            if (r0 + j < hw) sums[r0 + j] += __uint_as_float(v[j]);
                    }
                }
                tc_fence_before();
                mbar_arrive(&sm->part_empty[ps]);
                ++pcount;
            }
            auto stage_row = [&]() {
#pragma unroll
                for (int j = 0; j < HW; j += 4)
                    if (j < hw)
                        *reinterpret_cast<float4*>(my_row + (size_t)(c_beg + j) * 4) =
                            make_float4(f * sums[j], f * sums[j + 1], f * sums[j + 2], f * sums[j + 3]);
                fence_proxy_async();  // staging writes -> the TMA unit's reads
            };
            auto reduce_row = [&]() {
                bulk_reduce_add_f32(G.D + orow * G.ldd + part * G.ni, smem_u32(my_row), (uint32_t)nw * 4u);
                bulk_commit();
            };
            if constexpr (!kHalfStage) {
                // this lane's staging row is free once its last bulk reduction
                // has read it (issued by the lane of warp q)
                if (half == 0) bulk_wait_read_all();
                named_sync(1 + q, 64);
                if (got) stage_row();
                // both warps of the pair leave together when either one gave up
                if (named_sync_or(1 + q, 64, !got)) {
                    ok = false;
                    break;
                }
                if (half == 0 && orow >= 0) reduce_row();
            } else {
                // quarters q < 2 stage first, then q + 2 into the same rows; the
                // four warps of the row set pass the same four barriers every item
                const int set = q & 1;
                const bool first = q < 2;
                if (!first && half == 0) bulk_wait_read_all();  // the previous item's rows were read
                named_sync(1 + set, 128);
                if (first && got) stage_row();
                const bool fail1 = named_sync_or(1 + set, 128, !got);
                if (first && half == 0) {
                    if (!fail1 && orow >= 0) reduce_row();
                    bulk_wait_read_all();  // read before the second quarter overwrites the rows
                }
                named_sync(1 + set, 128);
                if (!first && got) stage_row();
                const bool fail2 = named_sync_or(1 + set, 128, !got);
                if (fail1 || fail2) {
                    ok = false;
                    break;
                }
                if (!first && half == 0 && orow >= 0) reduce_row();
            }
        }
        if (half == 0) bulk_wait_all();  // reductions complete before the CTA's shared memory goes away
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaW) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

int gcd_int(int a, int b) { return b == 0 ? a : gcd_int(b, a % b); }

std::mutex g_stage_mutex;
int g_stage_granted[2][64] = {};

// Shared memory of a launch whose widest part has ni columns (0: too large);
// parts wider than 192 columns stage 64 rows at a time.
size_t stage_smem_ni(int pieces, int ni, int max_smem, int* stages_out) {
    const size_t stage = (size_t)pieces * (kPieceA + (size_t)ni * kRowB);
    const size_t staging = (size_t)(ni > kMaxPart ? kTileM / 2 : kTileM) * (ni + 4) * 4;
    const size_t fixed = 2048 + staging;
    if ((long)max_smem - (long)fixed < 2L * (long)stage) return 0;
    int stages = (int)(((size_t)max_smem - fixed) / stage);
    stages = std::min(stages, kMaxS);
    if (stages_out) *stages_out = stages;
    return fixed + (size_t)stages * stage;
}

}  // namespace

size_t core_stage_smem(int pieces, int kdim, int ndim, int max_smem, int* stages_out) {
    (void)kdim;
    const int n_parts = (ndim + kMaxPart - 1) / kMaxPart;
    const int ni = ((ndim + n_parts - 1) / n_parts + 15) / 16 * 16;
    return stage_smem_ni(pieces, ni, max_smem, stages_out);
}

cudaError_t launch_core_stage_grouped(const UmmaArgs* a, int n_groups, int num_sms, int max_smem, int dev,
                                      cudaStream_t stream) {
    if (n_groups < 1 || n_groups > kMaxGroups) return cudaErrorNotSupported;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int products = a[0].n_products, f16 = a[0].f16;
    if (products != 1 && products != 3) return cudaErrorNotSupported;
    CParams P{};
    CLayout L{};
    L.pieces = products == 1 ? 1 : 2;
    int ng = 0;
    long items = 0, cost = 0;
    for (int i = 0; i < n_groups; ++i) {
        const UmmaArgs& x = a[i];
        // two partial slots of N columns fit the 512 TMEM columns for N <= 192
        if (x.n_products != products || x.f16 != f16 || x.s2_on || x.b_groups != kOffsetsC || x.kdim % 16 != 0 ||
            x.ndim % 16 != 0 || x.ndim < 16 || x.ldd % 4 != 0 || x.n_tiles < 0)
            return cudaErrorNotSupported;
        if (n_groups > 1 && !x.scale_table) return cudaErrorInvalidValue;
        if (x.n_tiles == 0) continue;
        CGroup& G = P.g[ng];
        G.A = x.A;
        G.a_piece_stride = x.a_piece_stride;
        G.row_src = x.row_src;
        G.row_dst = x.row_dst;
        G.tile_k = x.tile_k;
        G.scale_table = x.scale_table;
        G.row_scale = x.row_scale;
        G.D = x.D;
        G.ldd = x.ldd;
        G.kdim = x.kdim;
        G.ndim = x.ndim;
        G.kc = (x.kdim + kCh - 1) / kCh;
        // parts of at most 224 columns: the wide kernel takes N in (192, 224]
        // whole rather than gathering every A row once per part
        G.n_parts = (x.ndim + kMaxPartWide - 1) / kMaxPartWide;
        G.ni = ((x.ndim + G.n_parts - 1) / G.n_parts + 15) / 16 * 16;
        const int last = x.ndim - (G.n_parts - 1) * G.ni;
        G.box_rows = std::min(gcd_int(G.ni, last), 256);
        G.n_tiles = x.n_tiles;
        G.zero_row = x.zero_row;
        G.item_beg = items;
        G.n_items = (long)G.n_parts * x.n_tiles;
        G.cost_beg = cost;
        // per item: every K-chunk gathers 128 A rows and loads ni K~_o rows,
        // every partial is one drain (measured: a 128-row gather costs about
        // as much as 192 B rows, a drain about as much as one more chunk)
        G.cost = G.kc * (G.ni + 192) + (G.kc + kPartK - 1) / kPartK * 192;
        items += G.n_items;
        cost += G.n_items * (long)G.cost;
        L.ni = std::max(L.ni, G.ni);
        const cudaError_t e = tma_map_2d(x.B, (uint64_t)L.pieces * kOffsetsC * x.ndim, x.kdim, kCh, G.box_rows,
                                         &P.map[ng]);
        if (e != cudaSuccess) return e;
        ++ng;
    }
    if (ng == 0) return cudaSuccess;
    if (items > INT32_MAX) return cudaErrorInvalidValue;
    P.n_groups = ng;
    P.n_items = items;
    P.total_cost = cost;
    P.f16 = f16;
    for (int i = 0; i < 32; ++i) P.level_scale[i] = a[0].level_scale[i];
    P.error_flag = a[0].error_flag;
    P.wait_ns = a[0].wait_ns;
    const int wide = L.ni > kMaxPart ? 1 : 0;
    const size_t smem = stage_smem_ni(L.pieces, L.ni, max_smem, &L.stages);
    if (smem == 0) return cudaErrorNotSupported;
    L.prod = std::min(L.stages, kProdW);
    L.stage_bytes = (uint32_t)L.pieces * (kPieceA + (uint32_t)L.ni * kRowB);
    L.st_stride = (uint32_t)(L.ni + 4) * 4;
    {
        std::lock_guard<std::mutex> lock(g_stage_mutex);
        if (g_stage_granted[wide][dev] < (int)smem) {
            const cudaError_t e =
                wide ? cudaFuncSetAttribute(core_stage_kernel<112>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem)
                     : cudaFuncSetAttribute(core_stage_kernel<96>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem);
            if (e != cudaSuccess) return e;
            g_stage_granted[wide][dev] = (int)smem;
        }
    }
    const int grid = (int)std::min<long>(num_sms, items);
    if (wide)
        core_stage_kernel<112><<<grid, kThr, smem, stream>>>(P, L);
    else
        core_stage_kernel<96><<<grid, kThr, smem, stream>>>(P, L);
    return cudaGetLastError();
}

cudaError_t launch_core_stage(const UmmaArgs& a, int num_sms, int max_smem, int dev, cudaStream_t stream) {
    return launch_core_stage_grouped(&a, 1, num_sms, max_smem, dev, stream);
}

}  // namespace kifmm
