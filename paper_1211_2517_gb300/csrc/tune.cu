// kifmm_m2l_autotune: picks the tensor-core core launch's work assignment on
// the caller's own workload.
//
// Candidates change only how the core's (tile, N-chunk) work items are laid
// out over the persistent CTAs, never the arithmetic of an output element:
//   contiguous   0: item i goes to CTA i mod grid (neighbouring tiles, which
//                   share the offset and so the core matrix, run at the same
//                   time on different SMs and hit the same L2 lines);
//                1: each CTA takes one contiguous run of items (its own
//                   offsets, fewer core-matrix switches per CTA).
//   n_chunk      the plan's default N per item, or half of it (more, smaller
//                items: better balance, but every A row is gathered once per
//                N part).
//   variant      split6 only: 0 the classic core (hi and lo accumulators per
//                tile, epilogue after the tile's MMAs); 1 the core that keeps
//                each tile's A rows in shared memory and streams K~_o in
//                column blocks whose epilogues overlap the next block's MMAs
//                (n_chunk does not apply); 2 and 3 partial sums of two K-chunks
//                (2) or one (3) drained into registers by eight epilogue
//                warps while the next partial's MMAs run; 4 and 5 as 2 and 3
//                with the rows reduced into p~ by TMA bulk reductions instead
//                of vector atomics; 6 (f16x3 only) partials of three K-chunks;
//                9 and 10 (f16x3 only) as 2 and 6 with two K-chunks of a
//                partial issued per MMA step, 11 (f16x3 only) with all three,
//                12 (f16x3 only) as 11 with every epilogue lane reducing its
//                own row segment into p~ (no shared-memory transpose);
//                13 (1 or 2 pieces) the core that keeps K~_o in shared memory
//                while a CTA's contiguous run of tiles shares it, and streams
//                only the gathered A rows.
//                The FP16 split (f16x3) has no variant 1.
// Each candidate is timed with CUDA events around the core launch of
// kifmm_m2l_apply_levels.  With $KIFMM_M2L_AUTOTUNE_CACHE naming a file,
// results are kept there as a JSON object keyed by operator, device and
// workload, and a later call with the same key reads the choice back without
// timing anything.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "kifmm_internal.h"
#include "plan.h"

using namespace kifmm;

namespace {

std::mutex g_tune_mutex;

std::string tune_key(kifmm_m2l_plan plan, const MultiState* ms, int nrhs, int lo, int hi) {
    int64_t pairs = 0;
    for (const auto& g : ms->groups) pairs += g.count;
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, plan->device);
    char buf[512];
    std::snprintf(buf, sizeof(buf), "p=%d eps=%.6e d=%.6g prec=%d sm=%d%d sms=%d levels=%d-%d nrhs=%d boxes=%lld pairs=%lld",
                  plan->prm.p, plan->prm.eps, plan->prm.d, plan->prm.precision, prop.major, prop.minor, plan->num_sms,
                  lo, hi, nrhs, (long long)ms->total_boxes, (long long)pairs);
    std::string key = buf;
    if (plan->prm.kernel_id != KIFMM_KERNEL_LAPLACE) {
        // another operator (and rank) on the same boxes: its own entry
        std::snprintf(buf, sizeof(buf), " kernel=%d kh=%.17g", plan->prm.kernel_id, kernel_kh(plan->prm));
        key += buf;
    }
    return key;
}

// The cache file holds one entry per line:
//   "<key>": {"n_chunk": N, "contiguous": C, "variant": V, "core_ms": T},
// inside one pair of braces, so that it is a JSON object.
std::map<std::string, std::string> read_cache(const char* path) {
    std::map<std::string, std::string> out;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t a = line.find('"');
        if (a == std::string::npos) continue;
        const size_t b = line.find('"', a + 1);
        if (b == std::string::npos) continue;
        const size_t c = line.find('{', b);
        const size_t d = line.find('}', c == std::string::npos ? b : c);
        if (c == std::string::npos || d == std::string::npos) continue;
        out[line.substr(a + 1, b - a - 1)] = line.substr(c, d - c + 1);
    }
    return out;
}

bool parse_entry(const std::string& v, int* chunk, int* contig, int* variant, double* ms) {
    const char* s = v.c_str();
    const char* pc = std::strstr(s, "\"n_chunk\":");
    const char* pg = std::strstr(s, "\"contiguous\":");
    const char* pr = std::strstr(s, "\"variant\":");
    const char* pm = std::strstr(s, "\"core_ms\":");
    if (!pc || !pg || !pr || !pm) return false;
    *chunk = std::atoi(pc + 10);
    *contig = std::atoi(pg + 13);
    *variant = std::atoi(pr + 10);
    *ms = std::atof(pm + 10);
    return true;
}

int write_cache(const char* path, const std::map<std::string, std::string>& entries) {
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return -1;
        f << "{\n";
        size_t i = 0;
        for (const auto& e : entries) {
            f << "\"" << e.first << "\": " << e.second << (++i < entries.size() ? ",\n" : "\n");
        }
        f << "}\n";
        if (!f) return -1;
    }
    return std::rename(tmp.c_str(), path);
}

}  // namespace

extern "C" int kifmm_m2l_autotune(kifmm_m2l_plan plan, int instance, int level_lo, int level_hi, int nrhs,
                                  const float* q_up, float* p_down, int reps, kifmm_m2l_tune_result* result,
                                  void* stream) {
    if (!plan) {
        set_error("plan is NULL");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (reps < 1 || reps > 1000 || nrhs < 1) {
        set_error("reps must be in [1, 1000] and nrhs >= 1");
        return KIFMM_ERR_INVALID_ARG;
    }
    if (plan->prm.precision == KIFMM_PREC_FP32) {
        set_error("FP32 plans run the SIMT core, which has no launch choices to tune");
        return KIFMM_ERR_UNSUPPORTED;
    }
    int st = check_device(plan);
    if (st != KIFMM_OK) return st;
    MultiState* ms = nullptr;
    st = get_multi_state(plan, instance, level_lo, level_hi, false, &ms);
    if (st != KIFMM_OK) return st;
    const std::string key = tune_key(plan, ms, nrhs, level_lo, level_hi);
    const char* path = std::getenv("KIFMM_M2L_AUTOTUNE_CACHE");
    if (path && *path) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        const auto entries = read_cache(path);
        auto it = entries.find(key);
        int c = 0, g = 0, rs = 0;
        double t = 0;
        if (it != entries.end() && parse_entry(it->second, &c, &g, &rs, &t) && c >= 16 && c % 16 == 0 &&
            c <= 512 && (g == 0 || g == 1) && rs >= 0 && rs <= 13) {
            plan->tune_chunk = c == core_chunk_default(plan) ? 0 : c;
            plan->tune_contig = g;
            plan->tune_variant = rs;
            if (result) *result = {c, g, rs, t, 1};
            return KIFMM_OK;
        }
    }

    // candidates (n_chunk, contiguous, variant)
    struct Cand {
        int chunk, contig, variant;
    };
    const int c0 = core_chunk_default(plan);
    const int c1 = (c0 / 2 + 15) / 16 * 16;
    std::vector<Cand> cands;
    for (int g = 0; g < 2; ++g) {
        if (plan->core_hilo) {
            cands.push_back({c0, g, 2});
            cands.push_back({c0, g, 3});
            cands.push_back({c0, g, 4});
            cands.push_back({c0, g, 5});
            cands.push_back({c0, g, 9});
            if (plan->prm.precision != KIFMM_PREC_F16X3) {
                cands.push_back({c0, g, 1});  // A-resident: BF16 only
            } else {
                cands.push_back({c0, g, 6});  // three-K-chunk partials: short enough chains for 3 products
                cands.push_back({c0, g, 10});
                cands.push_back({c0, g, 11});
                cands.push_back({c0, g, 12});
            }
        }
        if (plan->products <= 3 && g == 1) cands.push_back({c0, g, 13});  // K~_o resident (contiguous runs only)
        cands.push_back({c0, g, 0});
        if (c1 >= 16 && c1 < c0) cands.push_back({c1, g, 0});
    }
    const bool was_profiling = plan->profile;
    kifmm_m2l_profile_read(plan, nullptr, nullptr);  // drop pending records
    plan->profile = true;
    double best = 1e300;
    Cand bestc = cands[0];
    st = KIFMM_OK;
    for (const Cand& cd : cands) {
        if (st != KIFMM_OK) break;
        plan->tune_chunk = cd.chunk == c0 ? 0 : cd.chunk;
        plan->tune_contig = cd.contig;
        plan->tune_variant = cd.variant;
        // one untimed pass (tile tables, first launch), then reps timed ones
        st = kifmm_m2l_apply_levels(plan, instance, level_lo, level_hi, nrhs, q_up, p_down, 0.0f, stream);
        if (st == KIFMM_OK) st = kifmm_m2l_profile_read(plan, nullptr, nullptr);
        for (int r = 0; r < reps && st == KIFMM_OK; ++r)
            st = kifmm_m2l_apply_levels(plan, instance, level_lo, level_hi, nrhs, q_up, p_down, 0.0f, stream);
        double t[3] = {0, 0, 0};
        if (st == KIFMM_OK) st = kifmm_m2l_profile_read(plan, t, nullptr);
        if (st == KIFMM_OK) st = kifmm_m2l_sync(plan, stream);
        if (st == KIFMM_OK && t[1] / reps < best) {
            best = t[1] / reps;
            bestc = cd;
        }
    }
    plan->profile = was_profiling;
    if (st != KIFMM_OK) {
        plan->tune_chunk = 0;
        plan->tune_contig = 0;
        plan->tune_variant = 2;
        return st;
    }
    plan->tune_chunk = bestc.chunk == c0 ? 0 : bestc.chunk;
    plan->tune_contig = bestc.contig;
    plan->tune_variant = bestc.variant;
    if (result) *result = {bestc.chunk, bestc.contig, bestc.variant, best, 0};
    if (path && *path) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto entries = read_cache(path);
        char v[160];
        std::snprintf(v, sizeof(v), "{\"n_chunk\": %d, \"contiguous\": %d, \"variant\": %d, \"core_ms\": %.6f}",
                      bestc.chunk, bestc.contig, bestc.variant, best);
        entries[key] = v;
        if (write_cache(path, entries) != 0) {
            set_error(std::string("could not write the autotune cache ") + path);
            return KIFMM_ERR_INVALID_ARG;
        }
    }
    return KIFMM_OK;
}
