// Host side of the learned warm start's C ABI (gspca_ws_features,
// gspca_ws_forward, gspca_ws_train_step): argument checks and launches of the
// kernels in warmstart.cuh.  The warm start inside a fit is driven by
// gspca_fit / gspca_fit_batched (opts->warm).
#include <cuda_runtime.h>

#include "../../include/gspca.h"
#include "handle.h"
#include "warmstart_kernels.cuh"

using namespace gspca;

static_assert(kWsParams == GSPCA_WS_PARAMS, "parameter count of the C ABI");
static_assert(kWsIn == GSPCA_WS_FEATURES && kWsSketch == GSPCA_WS_SKETCH, "feature sizes of the C ABI");

namespace {

constexpr int kWsWarps = 8;  // warps per block of the per-column kernels

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" {

gspca_status gspca_ws_features(void* stream, const float* X, long ldx, int M, int N, const float* T, const float* P,
                               int k, const float* G, float* feat) {
    if (!X || !G || !feat || M < 1 || N < 1 || ldx < M || k < 0) return GSPCA_ERR_INVALID_ARG;
    if (k > 0 && (!T || !P)) return GSPCA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ws_raw_features_kernel<<<(N + kWsWarps - 1) / kWsWarps, 32 * kWsWarps, 0, s>>>(X, ldx, M, N, T, P, k, G, feat);
    ws_normalize_kernel<<<1, 1024, 0, s>>>(feat, N);
    GS_CUDA(cudaGetLastError());
    return GSPCA_OK;
}

gspca_status gspca_ws_forward(void* stream, const float* net, const float* feat, long count, float* w) {
    if (!net || !feat || !w || count < 0) return GSPCA_ERR_INVALID_ARG;
    if (count == 0) return GSPCA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const long blocks = (count + kWsWarps - 1) / kWsWarps;
    if (blocks > 0x7fffffffL) return GSPCA_ERR_NOT_SUPPORTED;
    ws_forward_kernel<<<(unsigned)blocks, 32 * kWsWarps, 0, s>>>(net, feat, count, w);
    GS_CUDA(cudaGetLastError());
    return GSPCA_OK;
}

gspca_status gspca_ws_train_step(gspca_t h, void* stream, float* net, float* adam_m, float* adam_v, int step,
                                 float lr, const float* feat, const float* target, const int* offsets, int ninst,
                                 long ncols, float* loss, float* grad) {
    if (!h || !net || !feat || !target || !offsets || ninst < 1 || ncols < 1 || step < 1 || !(lr >= 0.f))
        return GSPCA_ERR_INVALID_ARG;
    if (lr > 0.f && (!adam_m || !adam_v)) return GSPCA_ERR_INVALID_ARG;
    if (ncols > 0x7fffffffL) return GSPCA_ERR_NOT_SUPPORTED;
    GS_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: Z1, Z2, D1, D2 (64 x ncols each), w, g (ncols), block partials, instance losses
    const long cols_per_blk = 2048;
    const int nblk = (int)((ncols + cols_per_blk - 1) / cols_per_blk);
    const size_t act = up256(sizeof(float) * kWsH * (size_t)ncols);
    const size_t vec = up256(sizeof(float) * (size_t)ncols);
    const size_t part = up256(sizeof(float) * kWsParams * (size_t)nblk);
    const size_t inst = up256(sizeof(float) * (size_t)ninst);
    const size_t need = 4 * act + 2 * vec + part + inst;
    if (need > h->ws_train_bytes) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return GSPCA_ERR_NOT_SUPPORTED;
        GS_CUDA(cudaStreamSynchronize(s));
        if (h->ws_train) GS_CUDA(cudaFree(h->ws_train));
        h->ws_train = nullptr;
        h->ws_train_bytes = 0;
        cudaError_t e = cudaMalloc(&h->ws_train, need);
        if (e != cudaSuccess) {
            cuda_ok(e);
            h->ws_train = nullptr;
            return e == cudaErrorMemoryAllocation ? GSPCA_ERR_OOM : GSPCA_ERR_CUDA;
        }
        h->ws_train_bytes = need;
    }
    char* b = static_cast<char*>(h->ws_train);
    WsTrainScratch sc{};
    sc.Z1 = (float*)b;
    sc.Z2 = (float*)(b + act);
    sc.D1 = (float*)(b + 2 * act);
    sc.D2 = (float*)(b + 3 * act);
    sc.w = (float*)(b + 4 * act);
    sc.g = (float*)(b + 4 * act + vec);
    sc.part = (float*)(b + 4 * act + 2 * vec);
    sc.inst = (float*)(b + 4 * act + 2 * vec + part);
    sc.nblk = nblk;
    const unsigned cb = (unsigned)((ncols + 127) / 128);
    ws_train_fwd_kernel<<<cb, 128, 0, s>>>(net, feat, ncols, sc);
    ws_loss_kernel<<<ninst, 256, 0, s>>>(target, offsets, ninst, sc);
    ws_train_bwd_kernel<<<cb, 128, 0, s>>>(net, ncols, sc);
    ws_wgrad_kernel<<<nblk, kWsGradThreads, 0, s>>>(feat, ncols, cols_per_blk, sc);
    ws_adam_kernel<<<(kWsParams + 255) / 256, 256, 0, s>>>(net, adam_m, adam_v, sc, ninst, step, lr, 0.9f, 0.999f,
                                                          1e-8f, grad, loss, lr > 0.f ? 1 : 0);
    GS_CUDA(cudaGetLastError());
    return GSPCA_OK;
}

}  // extern "C"
