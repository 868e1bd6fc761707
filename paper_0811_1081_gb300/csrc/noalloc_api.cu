// gspca_fit_noalloc: the fit of gspca_fit for callers that must not allocate
// device memory.  Its scratch workspace is one file-scope device array; the
// host code below looks up that array's device address once per device and
// carves the workspace of each call out of it.  Nothing here calls
// cudaMalloc, cudaFree or an allocating library routine.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <mutex>

#include "../../include/gspca.h"
#include "fit_kernel.cuh"
#include "prep_kernels.cuh"

using namespace gspca;

// The scratch array.  In host code this name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress, never from &array.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GSPCA_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices];
int g_num_sms[kMaxDevices];

// Once per device, with that device current: resolve the array's device
// address (checked) and the SM count.
gspca_status device_setup(int dev, void** addr, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) return GSPCA_ERR_NOT_SUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return GSPCA_ERR_CUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            return GSPCA_ERR_CUDA;
        g_num_sms[dev] = n;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return GSPCA_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bump allocator over the scratch array (addresses only; no memory is obtained).
struct Carve {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        T* p = reinterpret_cast<T*>(base + off);
        off += up256(sizeof(T) * (count > 0 ? count : 1));
        return p;
    }
};

template <int CPT>
int blocks_per_sm(size_t dyn) {
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fit_kernel<CPT>, kBlock, dyn) != cudaSuccess) return 0;
    return bps;
}

template <int CPT>
cudaError_t launch(const FitArgs& a, int G, size_t dyn, cudaStream_t s) {
    void* args[] = {const_cast<FitArgs*>(&a)};
    return cudaLaunchCooperativeKernel((const void*)fit_kernel<CPT>, dim3(G), dim3(kBlock), args, dyn, s);
}

}  // namespace

extern "C" gspca_status gspca_fit_noalloc(void* stream, const float* X, gspca_layout layout, long ldx, int M, int N,
                                          int K, double tol, int max_iter, gspca_algo algo, float* T, float* P,
                                          double* lambda, int* iters, float* R_out, const gspca_opts* opts) {
    if (!X || !T || !P || !lambda) return GSPCA_ERR_INVALID_ARG;
    if (M < 1 || N < 1 || K < 1 || K > M || K > N) return GSPCA_ERR_INVALID_ARG;
    if (!(tol > 0.0) || max_iter < 1) return GSPCA_ERR_INVALID_ARG;
    if (algo != GSPCA_NIPALS && algo != GSPCA_GS) return GSPCA_ERR_INVALID_ARG;
    if ((layout == GSPCA_COL_MAJOR && ldx < M) || (layout == GSPCA_ROW_MAJOR && ldx < N) ||
        (layout != GSPCA_COL_MAJOR && layout != GSPCA_ROW_MAJOR))
        return GSPCA_ERR_INVALID_ARG;
    if (opts) {
        if (opts->center < 0 || opts->center > 2 || opts->grid_ctas < 0 || opts->timeout_s < 0)
            return GSPCA_ERR_INVALID_ARG;
        if (opts->iters_lock)
            for (int k = 0; k < K; ++k)
                if (opts->iters_lock[k] < 1) return GSPCA_ERR_INVALID_ARG;
    }
    if (N > 16 * kBlock) return GSPCA_ERR_NOT_SUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GSPCA_ERR_CUDA;
    void* scratch = nullptr;
    int sms = 0;
    gspca_status st = device_setup(dev, &scratch, &sms);
    if (st != GSPCA_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // launch shape (same rule as gspca_fit)
    int cpt = 1;
    while (cpt * kBlock < N) cpt *= 2;
    const int ld = (K + 3) / 4 * 4;
    const size_t dyn = sizeof(float) * (size_t)ld;
    int bps = 0;
    switch (cpt) {
        case 1: bps = blocks_per_sm<1>(dyn); break;
        case 2: bps = blocks_per_sm<2>(dyn); break;
        case 4: bps = blocks_per_sm<4>(dyn); break;
        case 8: bps = blocks_per_sm<8>(dyn); break;
        default: bps = blocks_per_sm<16>(dyn); break;
    }
    if (bps < 1) return GSPCA_ERR_CUDA;
    const int np = (M + 3) / 4;
    const int ppr = cpt >= 8 ? 1 : 8 / cpt;
    int G = sms * bps;
    if (G > (np + ppr - 1) / ppr) G = (np + ppr - 1) / ppr;
    if (opts && opts->grid_ctas > 0 && opts->grid_ctas < G) G = opts->grid_ctas;
    if (G < 1) G = 1;

    // workspace for exactly this problem, checked against the array's size
    const size_t Mp = (size_t)np * 4;
    const int L = (N + K + 4 + 3) / 4 * 4;
    const dim3 pgrid((N + 31) / 32, (np + 31) / 32);
    const int nxpart = (int)(pgrid.x * pgrid.y);
    Carve c{static_cast<char*>(scratch)};
    FitArgs a{};
    a.R = c.take<float>(Mp * N);
    a.V = c.take<float>(Mp * ld);
    a.U = c.take<float>((size_t)N * ld);
    a.W = c.take<float>((size_t)N * ld);
    a.vraw = c.take<float>(Mp);
    a.vcorr = c.take<float>(Mp);
    a.ut = c.take<float>(N);
    a.ucur = c.take<float>(N);
    a.upre = c.take<double>(N);
    a.part = c.take<float>((size_t)G * L);
    a.spart = c.take<double>((size_t)G * 4);
    a.red = c.take<double>(L);
    a.reds = c.take<double>(4);
    a.normpart = c.take<double>(G);
    a.lam = c.take<double>(K);
    a.iters = c.take<int>(K);
    a.info = c.take<int>(kInfoWords);
    a.abort = c.take<int>(4);
    a.bar = c.take<unsigned>(4);
    double* xpart = c.take<double>(nxpart);
    double* cmean = c.take<double>(N);
    double* rmean = c.take<double>(Mp);
    int* lock = c.take<int>(K);
    if (c.off > (size_t)GSPCA_NOALLOC_SCRATCH_BYTES) return GSPCA_ERR_NOT_SUPPORTED;

    const int center = opts ? opts->center : 0;
    if (center == 1)
        colmean_kernel<<<(N + 7) / 8, 256, 0, s>>>(X, (int)layout, ldx, M, N, cmean);
    else if (center == 2)
        rowmean_kernel<<<(M + 7) / 8, 256, 0, s>>>(X, (int)layout, ldx, M, N, rmean);
    // pack also clears the barrier, abort flag and status words of this call
    pack_kernel<<<pgrid, kPackThreads, 0, s>>>(X, (int)layout, ldx, M, N, np, center, cmean, rmean, a.R, xpart,
                                               a.bar, a.abort, a.info, kInfoWords);
    if (cudaGetLastError() != cudaSuccess) return GSPCA_ERR_CUDA;
    a.iters_lock = nullptr;
    if (opts && opts->iters_lock) {
        if (cudaMemcpyAsync(lock, opts->iters_lock, sizeof(int) * K, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return GSPCA_ERR_CUDA;
        a.iters_lock = lock;
    }
    a.M = M;
    a.N = N;
    a.K = K;
    a.np = np;
    a.algo = (int)algo;
    a.max_iter = max_iter;
    a.tol = tol;
    a.eps_thresh = 64.0 * (double)FLT_EPSILON;
    a.xpart = xpart;
    a.nxpart = nxpart;
    a.ldv = a.ldu = a.ldw = ld;
    a.L = L;
    const double timeout = (opts && opts->timeout_s > 0) ? opts->timeout_s : 2.0;
    a.timeout_ns = (unsigned long long)(timeout * 1e9);

    cudaError_t e;
    switch (cpt) {
        case 1: e = launch<1>(a, G, dyn, s); break;
        case 2: e = launch<2>(a, G, dyn, s); break;
        case 4: e = launch<4>(a, G, dyn, s); break;
        case 8: e = launch<8>(a, G, dyn, s); break;
        default: e = launch<16>(a, G, dyn, s); break;
    }
    if (e != cudaSuccess) return GSPCA_ERR_CUDA;
    const dim3 egrid((M + 31) / 32 + (N + 31) / 32, (K + 31) / 32);
    epilogue_kernel<<<egrid, 256, 0, s>>>(a.V, ld, a.U, ld, a.lam, a.iters, a.info, M, N, K, algo == GSPCA_GS, T, P,
                                          lambda, iters);
    if (R_out)
        unpack_kernel<<<pgrid, kPackThreads, 0, s>>>(a.R, M, N, np, a.V, ld, a.U, ld, a.lam, a.info, K,
                                                     algo == GSPCA_GS, R_out);
    if (cudaGetLastError() != cudaSuccess) return GSPCA_ERR_CUDA;

    int words[kInfoWords + 1] = {0};
    if (cudaMemcpyAsync(words, a.info, sizeof(int) * kInfoWords, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(words + kInfoWords, a.abort, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GSPCA_ERR_CUDA;
    if (words[kInfoWords] != 0) return GSPCA_ERR_TIMEOUT;
    if (words[kInfoStatus] == kStDegenerate) return GSPCA_ERR_DEGENERATE;
    if (words[kInfoStatus] == kStNotConverged) return GSPCA_WARN_NOT_CONVERGED;
    return GSPCA_OK;
}
