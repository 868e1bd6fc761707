// Host side of the FP64 storage path: gspca_fit_f64 on a GSPCA_F64 handle.
//   [centring means] -> pack X into the row-major FP64 residual -> persistent
//   FP64 fit kernel -> epilogue (T, P, lambda, iters) -> [R_out]
// all enqueued on the caller's stream.
#include <cuda_runtime.h>

#include <cfloat>
#include <new>

#include "../../include/gspca.h"
#include "fit64_kernel.cuh"
#include "handle.h"
#include "launch_common.cuh"

using namespace gspca;

namespace {

__device__ __forceinline__ double load_x64(const double* X, int layout, long ldx, int r, int c) {
    return layout == 0 ? X[(size_t)c * ldx + r] : X[(size_t)r * ldx + c];
}

__global__ void colmean64_kernel(const double* X, int layout, long ldx, int M, int N, double* mean) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= N) return;
    double s = 0.0;
    for (int r = lane; r < M; r += 32) s += load_x64(X, layout, ldx, r, c);
    s = warp_sum(s);
    if (lane == 0) mean[c] = s / (double)M;
}

__global__ void rowmean64_kernel(const double* X, int layout, long ldx, int M, int N, double* mean) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= M) return;
    double s = 0.0;
    for (int c = lane; c < N; c += 32) s += load_x64(X, layout, ldx, r, c);
    s = warp_sum(s);
    if (lane == 0) mean[r] = s / (double)N;
}

// R (row-major) <- X, centred as asked (Eq. 1 / the prose of Sec. 2.1); one
// ||R||_F^2 partial per block (fixed grid, so the sum has a fixed order).  Block
// 0 also clears the barrier counter, the abort words and the info words.
__global__ void __launch_bounds__(256) pack64_kernel(const double* X, int layout, long ldx, int M, int N, int center,
                                                     const double* cmean, const double* rmean, double* R,
                                                     double* xpart, unsigned* flags, int* abort, int* info) {
    __shared__ double red[8];
    const int t = threadIdx.x;
    if (blockIdx.x == 0) {
        if (t < 32) flags[t] = 0u;
        if (t < 4) abort[t] = 0;
        if (t < 8) info[t] = 0;
    }
    const size_t total = (size_t)M * N, stride = (size_t)gridDim.x * blockDim.x;
    double sq = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + t; i < total; i += stride) {
        // walk X in its own storage order (coalesced reads)
        int r, c;
        if (layout == 0) {
            r = (int)(i % M);
            c = (int)(i / M);
        } else {
            r = (int)(i / N);
            c = (int)(i % N);
        }
        double v = load_x64(X, layout, ldx, r, c);
        if (center == 1) v -= cmean[c];
        else if (center == 2) v -= rmean[r];
        R[(size_t)r * N + c] = v;
        sq = fma(v, v, sq);
    }
    sq = warp_sum(sq);
    if ((t & 31) == 0) red[t >> 5] = sq;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        xpart[blockIdx.x] = s;
    }
}

// T (M x K, ld M), P (N x K, ld N), lambda, iters; zero past `found`.  T = V lambda
// (GS) or the scores t (NIPALS); svd: the unit score directions (V, or t / lambda).
__global__ void epilogue64_kernel(const double* V, const double* U, int ld, const double* lam_ws, const int* iters_ws,
                                  const int* info, int M, int N, int K, int gs, int svd, double* T, double* P,
                                  double* lambda, int* iters) {
    const int found = info[1];
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)M * K; i += stride) {
        const int r = (int)(i % M), k = (int)(i / M);
        double v = 0.0;
        if (k < found) {
            v = V[(size_t)r * ld + k];
            if (gs && !svd) v *= lam_ws[k];
            else if (!gs && svd) v /= lam_ws[k];
        }
        T[i] = v;
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)N * K; i += stride) {
        const int n = (int)(i % N), k = (int)(i / N);
        P[i] = k < found ? U[(size_t)n * ld + k] : 0.0;
    }
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            lambda[k] = k < found ? lam_ws[k] : 0.0;
            if (iters) iters[k] = k < found ? iters_ws[k] : 0;
        }
}

// R_out (M x N, ld M) from the row-major residual; when every component was found,
// the deflation of the last one (Eq. 3) is applied here, as the fit applies it
// inside the next component's first sweep.
__global__ void unpack64_kernel(const double* R, const double* V, const double* U, int ld, const double* lam_ws,
                                const int* info, int M, int N, int K, int gs, double* Rout) {
    const bool defl = info[1] == K;
    const double lamf = gs ? lam_ws[K - 1] : 1.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)M * N; i += stride) {
        const int r = (int)(i % M), c = (int)(i / M);
        double v = R[(size_t)r * N + c];
        if (defl) v = fma(-lamf * V[(size_t)r * ld + (K - 1)], U[(size_t)c * ld + (K - 1)], v);
        Rout[i] = v;
    }
}

// Rows per staged chunk and dynamic shared memory for N columns; rc = 0 when
// even one row does not fit.
cudaError_t plan64(int device, int N, int ldk, int G, int* rc, size_t* dyn) {
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, fit64_kernel)) != cudaSuccess) return e;
    const int max_slice = (N + G - 1) / G + 1;
    const long avail = (long)optin - (long)fa.sharedSizeBytes - 1024;
    int r = 0;
    while (r < kMaxRc64 && (long)smem64_bytes(N, r + 1, ldk, max_slice) <= avail) ++r;
    *rc = r;
    *dyn = smem64_bytes(N, r > 0 ? r : 1, ldk, max_slice);
    return cudaSuccess;
}

}  // namespace

gspca_status gspca::create_ws64(gspca_handle* h) {
    if (h->max_N > kMaxCols) return GSPCA_ERR_NOT_SUPPORTED;
    const Workspace64 probe = carve64_ws(nullptr, h->max_M, (int)h->max_N, h->max_K, h->num_sms);
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
    h->ws64_base = base;
    h->ws64 = carve64_ws(base, h->max_M, (int)h->max_N, h->max_K, h->num_sms);
    return GSPCA_OK;
}

extern "C" gspca_status gspca_fit_f64(gspca_t h, void* stream, const double* X, gspca_layout layout, long ldx, int M,
                                      int N, int K, double tol, int max_iter, gspca_algo algo, double* T, double* P,
                                      double* lambda, int* iters, double* R_out, const gspca_opts* opts) {
    if (!h || !X || !T || !P || !lambda) return GSPCA_ERR_INVALID_ARG;
    if (h->dtype != GSPCA_F64) return GSPCA_ERR_INVALID_ARG;
    if (M < 1 || N < 1 || K < 1 || K > M || K > N) return GSPCA_ERR_INVALID_ARG;
    if (M > h->max_M || N > h->max_N || K > h->max_K) return GSPCA_ERR_INVALID_ARG;
    if (!(tol > 0.0) || max_iter < 1) return GSPCA_ERR_INVALID_ARG;
    if (algo != GSPCA_NIPALS && algo != GSPCA_GS) return GSPCA_ERR_INVALID_ARG;
    if ((layout == GSPCA_COL_MAJOR && ldx < M) || (layout == GSPCA_ROW_MAJOR && ldx < N) ||
        (layout != GSPCA_COL_MAJOR && layout != GSPCA_ROW_MAJOR))
        return GSPCA_ERR_INVALID_ARG;
    const gspca_status ost = check_opts(opts, K);
    if (ost != GSPCA_OK) return ost;
    if (opts && (opts->warm || opts->gs_passes == 2 || opts->coef_trace)) return GSPCA_ERR_NOT_SUPPORTED;
    GS_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const Workspace64& w = h->ws64;
    int G = h->num_sms < M ? h->num_sms : M;
    if (opts && opts->grid_ctas > 0 && opts->grid_ctas < G) G = opts->grid_ctas;
    const int ldk = w.ld;
    int rc = 0;
    size_t dyn = 0;
    GS_CUDA(plan64(h->device, N, ldk, G, &rc, &dyn));
    if (rc < 1) return GSPCA_ERR_NOT_SUPPORTED;
    GS_CUDA(cudaFuncSetAttribute(fit64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int bps = 0;
    GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fit64_kernel, kBlock64, dyn));
    if (bps < 1) return GSPCA_ERR_NOT_SUPPORTED;

    const int center = opts ? opts->center : 0;
    const double timeout = (opts && opts->timeout_s > 0) ? opts->timeout_s : 2.0;
    const int* lock_dev = nullptr;
    if (opts && opts->iters_lock) {
        GS_CUDA(cudaMemcpyAsync(w.lock, opts->iters_lock, sizeof(int) * K, cudaMemcpyHostToDevice, s));
        lock_dev = w.lock;
    }
    int launches = 0;
    if (center == 1) {
        colmean64_kernel<<<(N + 7) / 8, 256, 0, s>>>(X, (int)layout, ldx, M, N, w.cmean);
        ++launches;
    } else if (center == 2) {
        rowmean64_kernel<<<(M + 7) / 8, 256, 0, s>>>(X, (int)layout, ldx, M, N, w.rmean);
        ++launches;
    }
    pack64_kernel<<<kPack64Blocks, 256, 0, s>>>(X, (int)layout, ldx, M, N, center, w.cmean, w.rmean, w.R, w.xpart,
                                                w.flags, w.abort, w.info);
    ++launches;
    GS_CUDA(cudaGetLastError());

    Fit64Args a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.algo = (int)algo;
    a.max_iter = max_iter;
    a.tol = tol;
    a.eps_thresh = 64.0 * DBL_EPSILON;
    a.xpart = w.xpart;
    a.nxpart = kPack64Blocks;
    a.R = w.R;
    a.V = w.V;
    a.U = w.U;
    a.W = w.W;
    a.ldk = ldk;
    a.vraw = w.vraw;
    a.vcorr = w.vcorr;
    a.ut = w.ut;
    a.upre = w.upre;
    a.partS = w.partS;
    a.LS = w.LS;
    a.partA = w.partA;
    a.scal = w.scal;
    a.lam = w.lam;
    a.iters = w.iters;
    a.info = w.info;
    a.flags = w.flags;
    a.abort = w.abort;
    a.iters_lock = lock_dev;
    a.timeout_ns = (unsigned long long)(timeout * 1e9);
    a.rc = rc;
    void* args[] = {&a};
    GS_CUDA(cudaEventRecord(h->ev0, s));
    GS_CUDA(cudaLaunchCooperativeKernel((const void*)fit64_kernel, dim3(G), dim3(kBlock64), args, dyn, s));
    ++launches;
    GS_CUDA(cudaEventRecord(h->ev1, s));
    epilogue64_kernel<<<256, 256, 0, s>>>(w.V, w.U, ldk, w.lam, w.iters, w.info, M, N, K, algo == GSPCA_GS,
                                          (opts && opts->svd_form == 1) ? 1 : 0, T, P, lambda, iters);
    ++launches;
    if (R_out) {
        unpack64_kernel<<<1024, 256, 0, s>>>(w.R, w.V, w.U, ldk, w.lam, w.info, M, N, K, algo == GSPCA_GS, R_out);
        ++launches;
    }
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaMemcpyAsync(h->h_info, w.info, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaMemcpyAsync(h->h_info + 8, w.abort, sizeof(int), cudaMemcpyDeviceToHost, s));
    int* hiters = h->h_info + 12;
    GS_CUDA(cudaMemcpyAsync(hiters, w.iters, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    GS_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->last.kernel_ms = ms;
    h->last.grid_ctas = G;
    h->last.team_ctas = G;
    h->last.block_threads = kBlock64;
    h->last.batch_pass = 0;
    h->last.kernel_launches = launches;
    if (h->h_info[8] != 0) return GSPCA_ERR_TIMEOUT;
    const int st = h->h_info[0];
    h->last.found = h->h_info[1];
    h->last.total_iters = (long long)h->h_info[2] + ((long long)h->h_info[3] << 31);
    // algorithmic bytes: one FP64 read of R per sweep, the deflation's write per component,
    // GS factor reads (V twice, W, U twice per iteration)
    double b = 0.0;
    const double mn = 8.0 * M * N;
    for (int k = 0; k < h->last.found; ++k) {
        b += ((double)hiters[k] + 1.0) * mn + (k > 0 ? mn : 0.0);
        if (algo == GSPCA_GS && k > 0) b += (double)hiters[k] * (2.0 * M * k + 3.0 * N * k) * 8.0;
    }
    h->last.alg_bytes = b;
    if (st == kStDegenerate) return GSPCA_ERR_DEGENERATE;
    if (st == kStNotConverged) return GSPCA_WARN_NOT_CONVERGED;
    return GSPCA_OK;
}
