// Host side of the C ABI declared in include/gspca.h: handles and their
// workspace, argument checks, and the launch sequence of one fit
//   [centring means] -> pack X into R panels -> persistent fit kernel
//   -> epilogue (T, P, lambda, iters) -> [unpack R_out]
// all enqueued on the caller's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/gspca.h"
#include "handle.h"
#include "launch_common.cuh"

using namespace gspca;

namespace {

char g_cuda_err[256] = "no CUDA error";
#ifdef GSPCA_PHASE_TIMING
unsigned long long* g_timing_dev = nullptr;  // instrumented builds only
#endif

}  // namespace

bool gspca::cuda_ok(cudaError_t e) {
    if (e == cudaSuccess) return true;
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return false;
}

namespace {

gspca_status check_fit_args(gspca_t h, const void* X, gspca_layout layout, long ldx, int M, int N, int K,
                            double tol, int max_iter, gspca_algo algo, const void* T, const void* P,
                            const void* lambda, const gspca_opts* opts) {
    if (!h || !X || !T || !P || !lambda) return GSPCA_ERR_INVALID_ARG;
    if (h->dtype == GSPCA_F64) return GSPCA_ERR_INVALID_ARG;  // FP64 handles take gspca_fit_f64
    if (M < 1 || N < 1 || K < 1 || K > M || K > N) return GSPCA_ERR_INVALID_ARG;
    if (M > h->max_M || N > h->max_N || K > h->max_K) return GSPCA_ERR_INVALID_ARG;
    if (!(tol > 0.0) || max_iter < 1) return GSPCA_ERR_INVALID_ARG;
    if (algo != GSPCA_NIPALS && algo != GSPCA_GS) return GSPCA_ERR_INVALID_ARG;
    if (layout == GSPCA_COL_MAJOR) {
        if (ldx < M) return GSPCA_ERR_INVALID_ARG;
    } else if (layout == GSPCA_ROW_MAJOR) {
        if (ldx < N) return GSPCA_ERR_INVALID_ARG;
    } else {
        return GSPCA_ERR_INVALID_ARG;
    }
    const gspca_status ost = check_opts(opts, K);
    if (ost != GSPCA_OK) return ost;
    if (opts) {
        if (opts->warm) {
            const gspca_warm_start* w = opts->warm;
            if (!w->net || !w->G || w->G_rows < M) return GSPCA_ERR_INVALID_ARG;
            if (algo != GSPCA_GS || cpt_for(N) > kWarmMaxCpt) return GSPCA_ERR_NOT_SUPPORTED;
            if (opts->gs_passes == 2) return GSPCA_ERR_NOT_SUPPORTED;  // no kernel has both
        }
    }
    return GSPCA_OK;
}

// Give the handle's workspace the buffers of the learned warm start (once).
gspca_status ensure_warm(gspca_t h) {
    if (h->ws.wsF) return GSPCA_OK;
    WsDims dims{(h->max_M + 3) / 4 * 4, (int)h->max_N, h->max_K, h->num_sms, true};
    const Workspace probe = carve(nullptr, dims);
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, probe.bytes);
    if (e != cudaSuccess) {
        cuda_ok(e);
        return e == cudaErrorMemoryAllocation ? GSPCA_ERR_OOM : GSPCA_ERR_CUDA;
    }
    if (!cuda_ok(cudaMemset(base, 0, probe.bytes))) {
        cudaFree(base);
        return GSPCA_ERR_CUDA;
    }
    GS_CUDA(cudaDeviceSynchronize());  // no work of an earlier call may still use the old workspace
    GS_CUDA(cudaFree(h->ws_base));
    h->ws_base = base;
    h->ws = carve(base, dims);
    return GSPCA_OK;
}

// Enqueue one fit on device buffers.  Does not synchronise.
gspca_status enqueue_fit(gspca_t h, cudaStream_t s, const float* X, gspca_layout layout, long ldx, int M, int N,
                         int K, double tol, int max_iter, gspca_algo algo, float* T, float* P, double* lambda,
                         int* iters, float* R_out, const gspca_opts* opts) {
    const int center = opts ? opts->center : 0;
    const double timeout = (opts && opts->timeout_s > 0) ? opts->timeout_s : 2.0;
    const int np = (M + 3) / 4;
    const int nxpart = ((N + 31) / 32) * ((np + 31) / 32);
    if (nxpart > h->ws.xcap) return GSPCA_ERR_NOT_SUPPORTED;
    const gspca_warm_start* warm = opts ? opts->warm : nullptr;
    if (warm) {
        const gspca_status ws = ensure_warm(h);
        if (ws != GSPCA_OK) return ws;
    }
    Plan plan{};
    GS_CUDA(plan_fit(h->device, h->num_sms, h->ws.G, M, N, K, cell_bytes(h->dtype), algo == GSPCA_GS, h->ws.ld,
                     opts, &plan));
    const int* lock_dev = nullptr;
    if (opts && opts->iters_lock) {
        GS_CUDA(cudaMemcpyAsync(h->ws.lock, opts->iters_lock, sizeof(int) * K, cudaMemcpyHostToDevice, s));
        lock_dev = h->ws.lock;
    }
    FitArgs a = make_args(h->ws, plan, M, N, K, tol, max_iter, algo, lock_dev, timeout, nxpart);
    if (opts && opts->test_stall) a.stall_word = h->ws.abort + 2;  // a word nothing sets
    if (opts) a.coef_trace = opts->coef_trace;
    if (warm) {
        a.ws_net = warm->net;
        a.ws_G = warm->G;
        a.wsF = h->ws.wsF;
        a.wsP0 = h->ws.wsP0;
        a.pC = h->ws.pC;
        a.wsPart = h->ws.wsPart;
        a.wsInit = h->ws.wsInit;
        a.ws_choice = warm->choice;
    }
#ifdef GSPCA_PHASE_TIMING
    if (!g_timing_dev) cudaMalloc(&g_timing_dev, 16 * sizeof(unsigned long long));
    cudaMemsetAsync(g_timing_dev, 0, 16 * sizeof(unsigned long long), s);
    a.timing = g_timing_dev;
#endif
    int launches = 0;
    GS_CUDA(enqueue_sequence(h->ws, plan, a, s, X, layout, ldx, center, T, P, lambda, iters, R_out, h->ev0, h->ev1,
                             &launches));
    h->last.grid_ctas = plan.G;
    h->last.team_ctas = plan.G;
    h->last.batch_pass = 0;
    h->last.block_threads = kBlock;
    h->last.kernel_launches = launches;
    return GSPCA_OK;
}

// Algorithmic bytes of the persistent kernel for a finished fit: per pass one
// read of R (M x N values of elem_bytes each); per component one extra write
// of R (the fused deflation); GS-PCA reads the FP32 factors V_(k) twice (b',
// v') and U_(k) twice, W_(k) once per iteration.
// With two Gram-Schmidt passes (CGS2) every iteration reads V_(k) and U_(k)
// twice more (the second pass's coefficients and its subtraction).
double alg_bytes(int M, int N, int found, const int* iters, bool gs, double elem_bytes, int gs_passes) {
    const double mn = (double)M * N * elem_bytes;
    double b = 0.0;
    for (int k = 0; k < found; ++k) {
        const double passes = (double)iters[k] + 1.0;
        b += passes * mn + (k > 0 ? mn : 0.0);
        if (gs && k > 0) b += (double)iters[k] * (2.0 * M * k + 3.0 * N * k) * 4.0;
        if (gs && k > 0 && gs_passes == 2) b += (double)iters[k] * (2.0 * M * k + 2.0 * N * k) * 4.0;
    }
    return b;
}

gspca_status finish(gspca_t h, cudaStream_t s, int K, gspca_algo algo, int M, int N, const gspca_opts* opts) {
    GS_CUDA(cudaMemcpyAsync(h->h_info, h->ws.info, sizeof(int) * kInfoWords, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaMemcpyAsync(h->h_info + kInfoWords, h->ws.abort, sizeof(int), cudaMemcpyDeviceToHost, s));
    int* hiters = h->h_info + kInfoWords + 4;
    GS_CUDA(cudaMemcpyAsync(hiters, h->ws.iters, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    GS_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->last.kernel_ms = ms;
    if (h->h_info[kInfoWords] != 0) return GSPCA_ERR_TIMEOUT;
#ifdef GSPCA_PHASE_TIMING
    {
        unsigned long long t[16];
        cudaMemcpy(t, g_timing_dev, sizeof(t), cudaMemcpyDeviceToHost);
        std::fprintf(stderr, "PHASES");
        for (int i = 0; i < 16; ++i) std::fprintf(stderr, " %llu", t[i]);
        std::fprintf(stderr, "\n");
    }
#endif
    const int st = h->h_info[kInfoStatus];
    h->last.found = h->h_info[kInfoFound];
    h->last.total_iters = (long long)h->h_info[kInfoItersLo] + ((long long)h->h_info[kInfoItersHi] << 31);
    h->last.alg_bytes = alg_bytes(M, N, h->last.found, hiters, algo == GSPCA_GS, cell_bytes(h->dtype) / 4.0,
                                  (opts && opts->gs_passes == 2) ? 2 : 1);
    if (st == kStDegenerate) return GSPCA_ERR_DEGENERATE;
    if (st == kStNotConverged) return GSPCA_WARN_NOT_CONVERGED;
    return GSPCA_OK;
}

}  // namespace

extern "C" {

gspca_status gspca_create(gspca_t* out, int device, long max_M, long max_N, int max_K, gspca_dtype dtype) {
    if (!out) return GSPCA_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_M < 1 || max_N < 1 || max_K < 1 || max_K > max_N || max_K > max_M) return GSPCA_ERR_INVALID_ARG;
    if (dtype != GSPCA_F32 && dtype != GSPCA_BF16 && dtype != GSPCA_F64) return GSPCA_ERR_INVALID_ARG;
    if (max_N > kMaxCols) return GSPCA_ERR_NOT_SUPPORTED;
    GS_CUDA(cudaSetDevice(device));
    gspca_handle* h = new (std::nothrow) gspca_handle();
    if (!h) return GSPCA_ERR_OOM;
    h->device = device;
    h->max_M = max_M;
    h->max_N = max_N;
    h->max_K = max_K;
    h->dtype = dtype;
    if (!cuda_ok(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device))) {
        delete h;
        return GSPCA_ERR_CUDA;
    }
    if (!cuda_ok(cudaMallocHost((void**)&h->h_info, sizeof(int) * (kInfoWords + 4 + (size_t)max_K))) ||
        !cuda_ok(cudaEventCreate(&h->ev0)) || !cuda_ok(cudaEventCreate(&h->ev1))) {
        gspca_destroy(h);
        return GSPCA_ERR_CUDA;
    }
    if (dtype == GSPCA_F64) {  // the FP64 storage path has a workspace of its own
        const gspca_status st = create_ws64(h);
        if (st != GSPCA_OK) {
            gspca_destroy(h);
            return st;
        }
        *out = h;
        return GSPCA_OK;
    }
    const WsDims dims{(max_M + 3) / 4 * 4, (int)max_N, max_K, h->num_sms};
    const Workspace probe = carve(nullptr, dims);
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, probe.bytes);
    if (e != cudaSuccess) {
        cuda_ok(e);
        gspca_destroy(h);
        return e == cudaErrorMemoryAllocation ? GSPCA_ERR_OOM : GSPCA_ERR_CUDA;
    }
    h->ws_base = base;
    h->ws = carve(base, dims);
    if (!cuda_ok(cudaMemset(base, 0, probe.bytes))) {
        gspca_destroy(h);
        return GSPCA_ERR_CUDA;
    }
    *out = h;
    return GSPCA_OK;
}

gspca_status gspca_fit(gspca_t h, void* stream, const float* X, gspca_layout layout, long ldx, int M, int N, int K,
                       double tol, int max_iter, gspca_algo algo, float* T, float* P, double* lambda, int* iters,
                       float* R_out, const gspca_opts* opts) {
    gspca_status st = check_fit_args(h, X, layout, ldx, M, N, K, tol, max_iter, algo, T, P, lambda, opts);
    if (st != GSPCA_OK) return st;
    GS_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = enqueue_fit(h, s, X, layout, ldx, M, N, K, tol, max_iter, algo, T, P, lambda, iters, R_out, opts);
    if (st != GSPCA_OK) return st;
    return finish(h, s, K, algo, M, N, opts);
}

gspca_status gspca_fit_host(gspca_t h, void* stream, const float* X, gspca_layout layout, long ldx, int M, int N,
                            int K, double tol, int max_iter, gspca_algo algo, float* T, float* P, double* lambda,
                            int* iters, float* R_out, const gspca_opts* opts) {
    gspca_status st = check_fit_args(h, X, layout, ldx, M, N, K, tol, max_iter, algo, T, P, lambda, opts);
    if (st != GSPCA_OK) return st;
    GS_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->stage) {
        const size_t xs = align_up(sizeof(float) * (size_t)h->max_M * h->max_N, 256);
        const size_t ts = align_up(sizeof(float) * (size_t)h->max_M * h->max_K, 256);
        const size_t ps = align_up(sizeof(float) * (size_t)h->max_N * h->max_K, 256);
        const size_t ls = align_up(sizeof(double) * (size_t)h->max_K, 256);
        const size_t is = align_up(sizeof(int) * (size_t)h->max_K, 256);
        const size_t rs = xs;
        void* b = nullptr;
        cudaError_t e = cudaMalloc(&b, xs + ts + ps + ls + is + rs);
        if (e != cudaSuccess) {
            cuda_ok(e);
            return e == cudaErrorMemoryAllocation ? GSPCA_ERR_OOM : GSPCA_ERR_CUDA;
        }
        h->stage = b;
        char* c = (char*)b;
        h->sX = (float*)c;
        h->sT = (float*)(c + xs);
        h->sP = (float*)(c + xs + ts);
        h->slam = (double*)(c + xs + ts + ps);
        h->siters = (int*)(c + xs + ts + ps + ls);
        h->sR = (float*)(c + xs + ts + ps + ls + is);
    }
    const size_t xbytes = layout == GSPCA_COL_MAJOR ? sizeof(float) * ((size_t)ldx * (N - 1) + M)
                                                    : sizeof(float) * ((size_t)ldx * (M - 1) + N);
    if (xbytes > sizeof(float) * (size_t)h->max_M * h->max_N) {
        // a padded leading dimension larger than the staging buffer: copy tightly packed
        if (layout == GSPCA_COL_MAJOR)
            GS_CUDA(cudaMemcpy2DAsync(h->sX, sizeof(float) * M, X, sizeof(float) * ldx, sizeof(float) * M, N,
                                      cudaMemcpyHostToDevice, s));
        else
            GS_CUDA(cudaMemcpy2DAsync(h->sX, sizeof(float) * N, X, sizeof(float) * ldx, sizeof(float) * N, M,
                                      cudaMemcpyHostToDevice, s));
        ldx = layout == GSPCA_COL_MAJOR ? M : N;
    } else {
        GS_CUDA(cudaMemcpyAsync(h->sX, X, xbytes, cudaMemcpyHostToDevice, s));
    }
    st = enqueue_fit(h, s, h->sX, layout, ldx, M, N, K, tol, max_iter, algo, h->sT, h->sP, h->slam, h->siters,
                     R_out ? h->sR : nullptr, opts);
    if (st != GSPCA_OK) return st;
    GS_CUDA(cudaMemcpyAsync(T, h->sT, sizeof(float) * (size_t)M * K, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaMemcpyAsync(P, h->sP, sizeof(float) * (size_t)N * K, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaMemcpyAsync(lambda, h->slam, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    if (iters) GS_CUDA(cudaMemcpyAsync(iters, h->siters, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
    if (R_out) GS_CUDA(cudaMemcpyAsync(R_out, h->sR, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToHost, s));
    return finish(h, s, K, algo, M, N, opts);
}

gspca_status gspca_get_info(gspca_t h, gspca_info* info) {
    if (!h || !info) return GSPCA_ERR_INVALID_ARG;
    *info = h->last;
    return GSPCA_OK;
}

gspca_status gspca_destroy(gspca_t h) {
    if (!h) return GSPCA_OK;
    cudaSetDevice(h->device);
    gspca_status st = GSPCA_OK;
    if (h->stage && !cuda_ok(cudaFree(h->stage))) st = GSPCA_ERR_CUDA;
    if (h->ws_base && !cuda_ok(cudaFree(h->ws_base))) st = GSPCA_ERR_CUDA;
    if (h->ws64_base && !cuda_ok(cudaFree(h->ws64_base))) st = GSPCA_ERR_CUDA;
    if (block_release(h) != GSPCA_OK) st = GSPCA_ERR_CUDA;
    if (h->ws_train && !cuda_ok(cudaFree(h->ws_train))) st = GSPCA_ERR_CUDA;
    if (h->h_info && !cuda_ok(cudaFreeHost(h->h_info))) st = GSPCA_ERR_CUDA;
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    batch_release(h->batch);
    delete h;
    return st;
}

const char* gspca_status_string(gspca_status s) {
    switch (s) {
        case GSPCA_OK: return "ok";
        case GSPCA_ERR_INVALID_ARG: return "invalid argument";
        case GSPCA_ERR_CUDA: return "CUDA error";
        case GSPCA_ERR_OOM: return "out of device memory";
        case GSPCA_WARN_NOT_CONVERGED: return "at least one component reached max_iter without converging";
        case GSPCA_ERR_DEGENERATE: return "rank exhausted: fewer than K components found";
        case GSPCA_ERR_TIMEOUT: return "a bounded device wait timed out";
        case GSPCA_ERR_NOT_SUPPORTED: return "not supported by this build";
    }
    return "unknown status";
}

const char* gspca_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"
