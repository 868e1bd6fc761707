// gspca_fit_noalloc: the fit of gspca_fit for callers that must not allocate
// device memory.  Its scratch workspace is one file-scope device array; every
// call looks up that array's device address for the current device and lays
// the workspace of the call out inside it.  Nothing here calls cudaMalloc,
// cudaFree or an allocating library routine.
#include <cuda_runtime.h>

#include "../../include/gspca.h"
#include "handle.h"
#include "launch_common.cuh"

using namespace gspca;

// The scratch array.  In host code this name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress, never from &array.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GSPCA_NOALLOC_SCRATCH_BYTES];

namespace {

// With the caller's device current: the array's device address (checked) and
// the SM count.  Resolved on every call rather than cached: after a
// cudaDeviceReset (or any teardown of the primary context) the module is
// loaded again and the array can sit at another address.
gspca_status device_setup(int dev, void** addr, int* sms) {
    void* p = nullptr;
    if (!cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch))) return GSPCA_ERR_CUDA;
    if (p == nullptr) return GSPCA_ERR_CUDA;
    int n = 0;
    if (!cuda_ok(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev))) return GSPCA_ERR_CUDA;
    if (n < 1) return GSPCA_ERR_CUDA;
    *addr = p;
    *sms = n;
    return GSPCA_OK;
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
    const gspca_status ost = check_opts(opts, K);
    if (ost != GSPCA_OK) return ost;
    if (opts && opts->warm) return GSPCA_ERR_NOT_SUPPORTED;  // its buffers are not part of the fixed scratch
    if (N > kMaxCols) return GSPCA_ERR_NOT_SUPPORTED;

    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev))) return GSPCA_ERR_CUDA;
    void* scratch = nullptr;
    int sms = 0;
    gspca_status st = device_setup(dev, &scratch, &sms);
    if (st != GSPCA_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // launch shape first (it fixes the grid, hence the partial buffers), then
    // the workspace for exactly this problem, checked against the array's size
    Plan plan{};
    if (!cuda_ok(plan_fit(dev, sms, sms, M, N, K, cell_bytes(GSPCA_F32), algo == GSPCA_GS, ws_ld(K), opts, &plan)))
        return GSPCA_ERR_CUDA;
    const WsDims dims{(long)(M + 3) / 4 * 4, N, K, plan.G};
    if (carve(nullptr, dims).bytes > (size_t)GSPCA_NOALLOC_SCRATCH_BYTES) return GSPCA_ERR_NOT_SUPPORTED;
    const Workspace w = carve(scratch, dims);
    const int np = (M + 3) / 4;
    const int nxpart = ((N + 31) / 32) * ((np + 31) / 32);

    const int* lock_dev = nullptr;
    if (opts && opts->iters_lock) {
        if (!cuda_ok(cudaMemcpyAsync(w.lock, opts->iters_lock, sizeof(int) * K, cudaMemcpyHostToDevice, s)))
            return GSPCA_ERR_CUDA;
        lock_dev = w.lock;
    }
    const double timeout = (opts && opts->timeout_s > 0) ? opts->timeout_s : 2.0;
    FitArgs a = make_args(w, plan, M, N, K, tol, max_iter, algo, lock_dev, timeout, nxpart);
    // a word nothing sets: the pack kernel clears all four abort words
    if (opts && opts->test_stall) a.stall_word = w.abort + 2;
    int launches = 0;
    // the pack kernel, first in the sequence, clears the barrier, abort and status words
    if (!cuda_ok(enqueue_sequence(w, plan, a, s, X, layout, ldx, opts ? opts->center : 0, T, P, lambda, iters, R_out,
                                  nullptr, nullptr, &launches)))
        return GSPCA_ERR_CUDA;

    int words[kInfoWords + 1] = {0};
    if (!cuda_ok(cudaMemcpyAsync(words, w.info, sizeof(int) * kInfoWords, cudaMemcpyDeviceToHost, s)) ||
        !cuda_ok(cudaMemcpyAsync(words + kInfoWords, w.abort, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
        !cuda_ok(cudaStreamSynchronize(s)))
        return GSPCA_ERR_CUDA;
    if (words[kInfoWords] != 0) return GSPCA_ERR_TIMEOUT;
    if (words[kInfoStatus] == kStDegenerate) return GSPCA_ERR_DEGENERATE;
    if (words[kInfoStatus] == kStNotConverged) return GSPCA_WARN_NOT_CONVERGED;
    return GSPCA_OK;
}
