// Internal: the handle behind gspca_t, shared by the translation units of the
// library (never part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>

#include "../../include/gspca.h"
#include "workspace.cuh"
#include "workspace64.cuh"

namespace gspca {

// Records the error text for gspca_last_cuda_error; true on cudaSuccess.
bool cuda_ok(cudaError_t e);

struct BatchCtl;

// Launch plan of the batched kernel for one team size and maximum problem size.
struct BatchPlan {
    int C = 0;          // CTAs per team (cluster)
    int clusters = 0;   // co-resident clusters (persistent grid)
    int ldk = 0, max_slice = 0, ring_bytes = 0;
    size_t dyn = 0;
    WsDims dims{};
    size_t stride = 0;  // bytes of one team's workspace
};

// Batched form: workspace of the teams, per-call counters, autotuner cache.
struct BatchState {
    void* ws = nullptr;
    size_t ws_bytes = 0;
    BatchCtl* ctl = nullptr;                 // device
    BatchCtl* h_ctl = nullptr;               // pinned copy read after a synchronous call
    std::map<uint64_t, int> tuned;           // shape-list key -> team size (CTAs per cluster)
    std::map<uint64_t, BatchPlan> plans;     // (team size, maximum sizes) -> plan
    cudaEvent_t e0 = nullptr, e1 = nullptr;  // bracket the launches of a synchronous call
    unsigned long long* timing_dev = nullptr;  // phase times (instrumented builds only)
};

// Release what the batched form allocated (called by gspca_destroy).
void batch_release(BatchState& b);

}  // namespace gspca

struct gspca_handle;

namespace gspca {
// Allocate the FP64 workspace of a GSPCA_F64 handle (fit64_api.cu).
gspca_status create_ws64(gspca_handle* h);
// Release what gspca_fit_block allocated (block_api.cu).
gspca_status block_release(gspca_handle* h);
}  // namespace gspca

#define GS_CUDA(call)                                     \
    do {                                                  \
        if (!gspca::cuda_ok(call)) return GSPCA_ERR_CUDA; \
    } while (0)

struct gspca_handle {
    int device = 0;
    long max_M = 0, max_N = 0;
    int max_K = 0;
    gspca_dtype dtype = GSPCA_F32;
    int num_sms = 0;
    void* ws_base = nullptr;
    gspca::Workspace ws{};
    int* h_info = nullptr;                     // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // bracket the persistent kernel
    // host-buffer entry point staging (allocated on first use)
    void* stage = nullptr;
    float *sX = nullptr, *sT = nullptr, *sP = nullptr, *sR = nullptr;
    double* slam = nullptr;
    int* siters = nullptr;
    gspca_info last{};
    gspca::BatchState batch;
    void* ws_train = nullptr;       // scratch of gspca_ws_train_step (grown on demand)
    size_t ws_train_bytes = 0;
    void* ws64_base = nullptr;      // GSPCA_F64 handles: the FP64 workspace (instead of ws)
    gspca::Workspace64 ws64{};
    void* blk_base = nullptr;       // gspca_fit_block: block workspace (allocated on first use)
    void* cublas = nullptr;         // its cuBLAS handle
    int* h_blk = nullptr;           // pinned flag word
};
