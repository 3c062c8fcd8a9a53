// The core products of the compressed M2L (Sec. 3.1, Eq. (14):
// p~^t += s_l K~_o q~^s over every box pair (t, s = t - o)), with the
// scatter into p~ handed to the TMA unit.
//
// Work: the offset-major tile list of 128 (pair, rhs) rows, split in N parts
// of at most 192 columns, gives (part, tile) items; each CTA takes one
// contiguous run of them, part-major, so consecutive items share the
// offset's K~_o (L2-resident, read by TMA per K stage with the A rows).
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
constexpr int kMaxPart = 192;            // N per part (96 running sums per epilogue thread)
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

struct CLayout {
    int stages, prod, pieces, kc;  // ring stages, producer warps in use, pieces, K-chunks
    int n_parts, ni;               // N parts, columns per part (the last may be narrower)
    long n_items;                  // n_parts * n_tiles
    uint32_t stage_bytes;          // pieces * (8 KB of A + ni * 64 of B)
    uint32_t st_stride;            // bytes per staging row: (ni + 4) * 4
    int box_rows;                  // rows per TMA box of K~_o (divides every part width)
};

__device__ __forceinline__ void named_sync(int id, int n) {
    // every participant reaches it: the pair leaves its loop only together
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__global__ void __launch_bounds__(kThr, 1)
    core_stage_kernel(const __grid_constant__ CUtensorMap bmap, const UmmaArgs args, const CLayout L) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    uint8_t* base = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    CSmem* sm = reinterpret_cast<CSmem*>(base);
    uint8_t* ring = base + 1024;
    uint8_t* staging = ring + (size_t)L.stages * L.stage_bytes;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int S = L.stages, NP = L.pieces, KC = L.kc, NI = L.ni;
    const int n_tiles = args.n_tiles;
    const long i_beg = L.n_items * blockIdx.x / gridDim.x;
    const long i_end = L.n_items * (blockIdx.x + 1) / gridDim.x;
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
        sm->wait_ns = args.wait_ns ? args.wait_ns : kWaitNs;
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

    auto part_width = [&](int part) { return min(NI, args.ndim - part * NI); };

    if (warp >= kEpiW && warp < kMmaW) {
        // ================= producers =================
        const int pw = warp - kEpiW, P = L.prod;
        constexpr int CPR = kCh / 8;     // 16-byte chunks per row and stage (4)
        constexpr int RPI = 32 / CPR;    // rows per warp instruction (8)
        constexpr int NR = kTileM / RPI; // rows per lane (16)
        const int cch = lane % CPR, rl = lane / CPR;
        int srow[NR], nrow[NR], ngroup = 0;
        auto load_rows = [&](long item) {
            const int t = (int)(item % n_tiles);
#pragma unroll
            for (int i = 0; i < NR; ++i) nrow[i] = __ldg(args.row_src + (long)t * kTileM + rl + RPI * i);
            ngroup = __ldg(args.tile_k + t) & 0xFFFF;
        };
        bool ok = true;
        long it = 0;
        if (pw < P && i_beg < i_end) load_rows(i_beg);
        for (long item = i_beg; item < i_end && ok; ++item) {
            const int part = (int)(item / n_tiles);
            const int nw = part_width(part);
            int k = 0;
            if (pw < P) {
#pragma unroll
                for (int i = 0; i < NR; ++i) srow[i] = nrow[i] < 0 ? args.zero_row : nrow[i];
                k = ngroup;
                if (item + 1 < i_end) load_rows(item + 1);
            }
            for (int kc = 0; kc < KC; ++kc, ++it) {
                if (pw >= P || it % P != pw) continue;
                const int s = (int)(it % S);
                const uint32_t ph = (uint32_t)(it / S) & 1u;
                if (!mbar_wait(&sm->empty[s], ph ^ 1u, sm, args.error_flag)) {
                    ok = false;
                    break;
                }
                const uint32_t st = smem_u32(ring + (size_t)s * L.stage_bytes);
                if (lane == 0) {
                    // the stage's K~_o columns: every piece, this part's rows
                    mbar_arrive_expect_tx(&sm->full[s], (uint32_t)NP * nw * kRowB);
                    for (int pc = 0; pc < NP; ++pc) {
                        const int row0 = (pc * kOffsetsC + k) * args.ndim + part * NI;
                        for (int rb = 0; rb < nw; rb += L.box_rows)
                            tma_load_2d(st + a_bytes + pc * b_piece + rb * kRowB, &bmap, kc * kCh, row0 + rb,
                                        &sm->full[s]);
                    }
                }
                const int col = kc * kCh + cch * 8;
                const uint32_t bytes = col < args.kdim ? 16u : 0u;
                const int colc = col < args.kdim ? col : 0;
                for (int pc = 0; pc < NP; ++pc) {
                    const __nv_bfloat16* src = args.A + pc * args.a_piece_stride + colc;
                    const uint32_t dst = st + pc * kPieceA;
#pragma unroll
                    for (int i = 0; i < NR; ++i)
                        cp_async16(dst + swz<kCh>(rl + RPI * i, cch), src + (long)srow[i] * args.kdim, bytes);
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
            int s = 0, pcount = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (long item = i_beg; item < i_end && ok; ++item) {
                const int nw = part_width((int)(item / n_tiles));
                const uint32_t idesc = umma_idesc(nw, args.f16);
                uint32_t d = tmem;
                for (int kc = 0; kc < KC; ++kc) {
                    const bool p_first = kc % kPartK == 0;
                    if (p_first) {
                        // the partial slot has been drained by the epilogue
                        const int ps = pcount & 1;
                        if (!mbar_wait(&sm->part_empty[ps], ((uint32_t)(pcount >> 1) & 1u) ^ 1u, sm,
                                       args.error_flag)) {
                            ok = false;
                            break;
                        }
                        d = tmem + (uint32_t)(ps * NI);
                    }
                    if (!mbar_wait(&sm->full[s], ph, sm, args.error_flag)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async();  // cp.async data -> tensor-core reads
                    tc_fence_after();
                    const uint64_t sd = desc0 + (uint64_t)((uint32_t)s * stage_u);
                    const uint64_t bd = sd + b_u;
                    const bool two = args.kdim - kc * kCh >= 32;  // K steps of 16 in this chunk: 2 or 1
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
        uint8_t* my_row = staging + (size_t)(q * 32 + lane) * L.st_stride;
        int pcount = 0;
        bool ok = true;
        long nx_row = -1;
        int nx_k = 0;
        float nx_rs = 1.f;
        auto fetch = [&](long item) {
            const int t = (int)(item % n_tiles);
            const long r = (long)t * kTileM + q * 32 + lane;
            nx_row = __ldg(args.row_dst + r);
            nx_k = __ldg(args.tile_k + t);
            nx_rs = 1.f;
            if (args.row_scale) {
                const int sr = __ldg(args.row_src + r);
                nx_rs = sr >= 0 ? __ldg(args.row_scale + sr) : 0.f;
            }
        };
        if (i_beg < i_end) fetch(i_beg);
        for (long item = i_beg; item < i_end && ok; ++item) {
            const long orow = nx_row;
            const float f = (args.scale_table ? __ldg(args.scale_table + (nx_k >> 16))
                                              : args.level_scale[(nx_k >> 16) & 31]) *
                            nx_rs;
            if (item + 1 < i_end) fetch(item + 1);
            const int part = (int)(item / n_tiles);
            const int nw = part_width(part);
            const int hw = nw / 2;  // columns of this warp (a multiple of 8, <= 96)
            const int c_beg = half * hw;
            // partials -> FP32 running sums, 48 columns per TMEM round
            float sums[kMaxPart / 2];
#pragma unroll
            for (int j = 0; j < kMaxPart / 2; ++j) sums[j] = 0.f;
            bool got = true;
            for (int kc = 0; kc < KC; kc += kPartK) {
                const int ps = pcount & 1;
                got = __all_sync(0xffffffffu, mbar_wait(&sm->part_full[ps], (uint32_t)(pcount >> 1) & 1u, sm,
                                                        args.error_flag));
                if (!got) break;
                tc_fence_after();
                const uint32_t col = tmem + lane_base + (uint32_t)(ps * NI + c_beg);
#pragma unroll
                for (int r0 = 0; r0 < kMaxPart / 2; r0 += 48) {
                    if (r0 < hw) {
                        uint32_t v[48];
#pragma unroll
                        for (int c = 0; c < 48; c += 8)
                            if (r0 + c < hw) tmem_ld8(col + (uint32_t)(r0 + c), v + c);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 48; ++j)
                            if (r0 + j < hw) sums[r0 + j] += __uint_as_float(v[j]);
                    }
                }
                tc_fence_before();
                mbar_arrive(&sm->part_empty[ps]);
                ++pcount;
            }
            // this lane's staging row is free once its last bulk reduction
            // has read it (issued by the lane of warp q)
            if (half == 0) bulk_wait_read_all();
            named_sync(1 + q, 64);
            if (got) {
#pragma unroll
                for (int j = 0; j < kMaxPart / 2; j += 4)
                    if (j < hw)
                        *reinterpret_cast<float4*>(my_row + (size_t)(c_beg + j) * 4) =
                            make_float4(f * sums[j], f * sums[j + 1], f * sums[j + 2], f * sums[j + 3]);
                fence_proxy_async();  // staging writes -> the TMA unit's reads
            }
            // both warps of the pair leave together when either one gave up
            if (named_sync_or(1 + q, 64, !got)) {
                ok = false;
                break;
            }
            if (half == 0 && orow >= 0) {
                bulk_reduce_add_f32(args.D + orow * args.ldd + part * NI, smem_u32(my_row), (uint32_t)nw * 4u);
                bulk_commit();
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
int g_stage_granted[64] = {};

}  // namespace

size_t core_stage_smem(int pieces, int kdim, int ndim, int max_smem, int* stages_out) {
    (void)kdim;
    const int n_parts = (ndim + kMaxPart - 1) / kMaxPart;
    const int ni = ((ndim + n_parts - 1) / n_parts + 15) / 16 * 16;
    const size_t stage = (size_t)pieces * (kPieceA + (size_t)ni * kRowB);
    const size_t staging = (size_t)kTileM * (ni + 4) * 4;
    const size_t fixed = 2048 + staging;
    if ((long)max_smem - (long)fixed < 2L * (long)stage) return 0;
    int stages = (int)(((size_t)max_smem - fixed) / stage);
    stages = std::min(stages, kMaxS);
    if (stages_out) *stages_out = stages;
    return fixed + (size_t)stages * stage;
}

cudaError_t launch_core_stage(const UmmaArgs& a, int num_sms, int max_smem, int dev, cudaStream_t stream) {
    if (a.n_products != 1 && a.n_products != 3) return cudaErrorNotSupported;
    // two partial slots of N columns fit the 512 TMEM columns for N <= 192
    if (a.s2_on || a.b_groups != kOffsetsC || a.kdim % 16 != 0 || a.ndim % 16 != 0 || a.ndim < 16 || a.ldd % 4 != 0)
        return cudaErrorNotSupported;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    CLayout L{};
    L.pieces = a.n_products == 1 ? 1 : 2;
    L.kc = (a.kdim + kCh - 1) / kCh;
    L.n_parts = (a.ndim + kMaxPart - 1) / kMaxPart;
    L.ni = ((a.ndim + L.n_parts - 1) / L.n_parts + 15) / 16 * 16;
    const size_t smem = core_stage_smem(L.pieces, a.kdim, a.ndim, max_smem, &L.stages);
    if (smem == 0) return cudaErrorNotSupported;
    L.prod = std::min(L.stages, kProdW);
    L.stage_bytes = (uint32_t)L.pieces * (kPieceA + (uint32_t)L.ni * kRowB);
    L.st_stride = (uint32_t)(L.ni + 4) * 4;
    const int last = a.ndim - (L.n_parts - 1) * L.ni;
    L.box_rows = std::min(gcd_int(L.ni, last), 256);
    L.n_items = (long)L.n_parts * a.n_tiles;
    if (L.n_items <= 0) return cudaSuccess;
    if (L.n_items > INT32_MAX) return cudaErrorInvalidValue;
    CUtensorMap bmap;
    cudaError_t e = tma_map_2d(a.B, (uint64_t)L.pieces * kOffsetsC * a.ndim, a.kdim, kCh, L.box_rows, &bmap);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(g_stage_mutex);
        if (g_stage_granted[dev] < (int)smem) {
            e = cudaFuncSetAttribute(core_stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            g_stage_granted[dev] = (int)smem;
        }
    }
    const int grid = (int)std::min<long>(num_sms, L.n_items);
    core_stage_kernel<<<grid, kThr, smem, stream>>>(bmap, a, L);
    return cudaGetLastError();
}

}  // namespace kifmm
