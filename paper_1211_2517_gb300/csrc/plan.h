// Internal plan object of the C ABI (include/kifmm_m2l.h), shared by the
// translation units that implement its entry points.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "kernels.h"
#include "kifmm_internal.h"

namespace kifmm {

constexpr int kTileRows = 128;

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

struct PairSet {
    DevBuf<int> src, dst;
    std::vector<int64_t> off_begin;  // [317] prefix by offset
    std::map<int, std::unique_ptr<DevBuf<Tile>>> tiles;  // per nrhs
    std::map<int, int> n_tiles;
};

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
    kifmm::DevBuf<float> C, K;
    kifmm::DevBuf<__nv_bfloat16> Cb, Rtb, Ub;  // 3 BF16 pieces each
    kifmm::DevBuf<int> err_flag;
    std::map<std::pair<int, int>, std::unique_ptr<kifmm::LevelState>> levels;
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
    ~kifmm_m2l_plan_s() {
        for (auto& r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : event_pool) cudaEventDestroy(e);
    }
    // scratch shared by all levels (apply calls on one plan are serialised)
    kifmm::DevBuf<float> qt, pt;
    kifmm::DevBuf<__nv_bfloat16> qb;
};


namespace kifmm {

// The registered level, or nullptr.
LevelState* find_level(kifmm_m2l_plan plan, int instance, int level);
// KIFMM_OK when the current device is the plan's device.
int check_device(kifmm_m2l_plan plan);
// N per work item of the compression / expansion GEMMs.
int chunk_for(int ndim);

}  // namespace kifmm
