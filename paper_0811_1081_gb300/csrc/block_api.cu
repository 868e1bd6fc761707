// gspca_fit_block: block power iteration (components b at a time), the block
// form of the GS-PCA loop of Sec. 2.3 (not in the paper).  Per block of width
// bw, on the caller's stream:
//   U = R^T R(:, k0 .. k0+bw-1); U -= U_(k0) U_(k0)^T U; U = qr(U)
//   repeat: Y = R U; Y -= V_(k0) V_(k0)^T Y; V = qr(Y)
//           Z = R^T V; Z -= U_(k0) U_(k0)^T Z; s = sqrt(eig(Z^T Z)) (Ritz values)
//           stop when every |s_i - s_i'| < tol s_i (or max_iter / the lock); else U = qr(Z)
//   Rayleigh-Ritz on B = Z^T U; R -= V diag(sigma) U^T.
// The large products are FP32 GEMMs of cuBLAS; qr is Cholesky QR applied twice
// with the Gram matrix accumulated in FP64 (block_kernels.cuh).  The residual
// lives column-major in the handle's R buffer; V and U are kept in the caller's
// T and P (unit columns until the block ends).  One host synchronisation per
// iteration reads the stop and degenerate flags.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/gspca.h"
#include "block_kernels.cuh"
#include "handle.h"
#include "launch_common.cuh"

using namespace gspca;

namespace {

#define BL_CUBLAS(call)                                                       \
    do {                                                                      \
        if ((call) != CUBLAS_STATUS_SUCCESS) {                                \
            cuda_ok(cudaErrorUnknown);                                        \
            return GSPCA_ERR_CUDA;                                            \
        }                                                                     \
    } while (0)

struct BlockWs {
    float *Y, *V, *Z, *U, *tmp, *Sinv, *Yh, *Zh;
    double *part, *G, *Bm, *ev, *evec, *sp, *sigma;
    int* flag;
    size_t bytes;
};

BlockWs carve_block(void* base, long M, int N, int K) {
    BlockWs w{};
    char* b = static_cast<char*>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = (off + 255) / 256 * 256;
        void* p = b ? b + off : nullptr;
        off += bytes > 0 ? bytes : 1;
        return p;
    };
    const size_t B = kBlkMax;
    w.Y = (float*)take(sizeof(float) * (size_t)M * B);
    w.V = (float*)take(sizeof(float) * (size_t)M * B);
    w.Z = (float*)take(sizeof(float) * (size_t)N * B);
    w.U = (float*)take(sizeof(float) * (size_t)N * B);
    w.tmp = (float*)take(sizeof(float) * (size_t)((size_t)K > B ? (size_t)K : B) * B);
    w.Sinv = (float*)take(sizeof(float) * B * B);
    w.Yh = (float*)take(sizeof(float) * B * B);
    w.Zh = (float*)take(sizeof(float) * B * B);
    w.part = (double*)take(sizeof(double) * kGramCtas * B * B);
    w.G = (double*)take(sizeof(double) * B * B);
    w.Bm = (double*)take(sizeof(double) * B * B);
    w.ev = (double*)take(sizeof(double) * B);
    w.evec = (double*)take(sizeof(double) * B * B);
    w.sp = (double*)take(sizeof(double) * B);
    w.sigma = (double*)take(sizeof(double) * B);
    w.flag = (int*)take(sizeof(int) * 4);
    w.bytes = (off + 255) / 256 * 256;
    return w;
}

// Gram matrix out = A^T B (n x m, FP64) of FP32 column-major A (rows x n), B (rows x m).
void gram(cudaStream_t s, const float* A, int lda, const float* B, int ldb, int rows, int n, int m, const BlockWs& w,
          double* out) {
    gram_part_kernel<<<kGramCtas, 1024, 0, s>>>(A, lda, B, ldb, rows, n, m, w.part);
    gram_sum_kernel<<<1, 1024, 0, s>>>(w.part, kGramCtas, n, m, out);
}

// Cholesky QR applied twice: Q (rows x n) = A S1^{-1} S2^{-1}, A left unchanged
// unless Q == A is not required (Q and A distinct buffers).  `have_gram`: w.G
// already holds A^T A.
gspca_status cholqr2(cublasHandle_t cb, cudaStream_t s, const float* A, float* Q, int rows, int n, const BlockWs& w,
                     bool have_gram, int* launches) {
    const float one = 1.f, zero = 0.f;
    if (!have_gram) {
        gram(s, A, rows, A, rows, rows, n, n, w, w.G);
        *launches += 2;
    }
    chol_inv_kernel<<<1, 256, 0, s>>>(w.G, n, w.Sinv, w.flag);
    BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_N, CUBLAS_OP_N, rows, n, n, &one, A, rows, w.Sinv, n, &zero, Q, rows));
    gram(s, Q, rows, Q, rows, rows, n, n, w, w.G);
    chol_inv_kernel<<<1, 256, 0, s>>>(w.G, n, w.Sinv, w.flag);
    // Q <- Q S2^{-1} in place: an upper-triangular factor on the right (column j uses columns <= j)
    BL_CUBLAS(cublasStrmm(cb, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, rows, n,
                          &one, w.Sinv, n, Q, rows, Q, rows));
    *launches += 6;
    return GSPCA_OK;
}

// X (rows x n) -= Q (rows x k) (Q^T X); nothing when k == 0.
gspca_status project_out(cublasHandle_t cb, const float* Q, int rows, int k, float* X, int n, float* tmp) {
    if (k == 0) return GSPCA_OK;
    const float one = 1.f, zero = 0.f, mone = -1.f;
    BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_T, CUBLAS_OP_N, k, n, rows, &one, Q, rows, X, rows, &zero, tmp, k));
    BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_N, CUBLAS_OP_N, rows, n, k, &mone, Q, rows, tmp, k, &one, X, rows));
    return GSPCA_OK;
}

}  // namespace

gspca_status gspca::block_release(gspca_handle* h) {
    gspca_status st = GSPCA_OK;
    if (h->blk_base && cudaFree(h->blk_base) != cudaSuccess) st = GSPCA_ERR_CUDA;
    if (h->cublas) cublasDestroy((cublasHandle_t)h->cublas);
    if (h->h_blk) cudaFreeHost(h->h_blk);
    h->blk_base = nullptr;
    h->cublas = nullptr;
    h->h_blk = nullptr;
    return st;
}

extern "C" gspca_status gspca_fit_block(gspca_t h, void* stream, const float* X, gspca_layout layout, long ldx, int M,
                                        int N, int K, int block, double tol, int max_iter, float* T, float* P,
                                        double* lambda, int* iters, float* R_out, const gspca_opts* opts) {
    if (!h || !X || !T || !P || !lambda) return GSPCA_ERR_INVALID_ARG;
    if (h->dtype != GSPCA_F32) return GSPCA_ERR_INVALID_ARG;
    if (M < 1 || N < 1 || K < 1 || K > M || K > N) return GSPCA_ERR_INVALID_ARG;
    if (M > h->max_M || N > h->max_N || K > h->max_K) return GSPCA_ERR_INVALID_ARG;
    if (block < 1 || block > kBlkMax || !(tol > 0.0) || max_iter < 1) return GSPCA_ERR_INVALID_ARG;
    if ((layout == GSPCA_COL_MAJOR && ldx < M) || (layout == GSPCA_ROW_MAJOR && ldx < N) ||
        (layout != GSPCA_COL_MAJOR && layout != GSPCA_ROW_MAJOR))
        return GSPCA_ERR_INVALID_ARG;
    const gspca_status ost = check_opts(opts, K);
    if (ost != GSPCA_OK) return ost;
    if (opts && (opts->warm || opts->gs_passes == 2 || opts->coef_trace)) return GSPCA_ERR_NOT_SUPPORTED;
    GS_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->blk_base) {
        const BlockWs probe = carve_block(nullptr, h->max_M, (int)h->max_N, h->max_K);
        void* base = nullptr;
        cudaError_t e = cudaMalloc(&base, probe.bytes);
        if (e != cudaSuccess) {
            cuda_ok(e);
            return e == cudaErrorMemoryAllocation ? GSPCA_ERR_OOM : GSPCA_ERR_CUDA;
        }
        h->blk_base = base;
        cublasHandle_t cb = nullptr;
        if (cublasCreate(&cb) != CUBLAS_STATUS_SUCCESS) {
            block_release(h);
            return GSPCA_ERR_CUDA;
        }
        h->cublas = cb;
        if (!cuda_ok(cudaMallocHost((void**)&h->h_blk, sizeof(int) * 4))) {
            block_release(h);
            return GSPCA_ERR_CUDA;
        }
    }
    const BlockWs w = carve_block(h->blk_base, h->max_M, (int)h->max_N, h->max_K);
    cublasHandle_t cb = (cublasHandle_t)h->cublas;
    BL_CUBLAS(cublasSetStream(cb, s));
    BL_CUBLAS(cublasSetMathMode(cb, CUBLAS_DEFAULT_MATH));  // FP32 products, no TF32
    float* R = h->ws.R;  // the handle's residual buffer, here column-major M x N
    const float one = 1.f, zero = 0.f, mone = -1.f;
    int launches = 0;
    const int center = opts ? opts->center : 0;
    if (center == 1) {
        colmean_kernel<<<(N + 7) / 8, 256, 0, s>>>(X, (int)layout, ldx, M, N, h->ws.cmean);
        ++launches;
    } else if (center == 2) {
        rowmean_kernel<<<(M + 7) / 8, 256, 0, s>>>(X, (int)layout, ldx, M, N, h->ws.rmean);
        ++launches;
    }
    pack_colmajor_kernel<<<1024, 256, 0, s>>>(X, (int)layout, ldx, M, N, center, h->ws.cmean, h->ws.rmean, R);
    ++launches;
    GS_CUDA(cudaGetLastError());
    GS_CUDA(cudaEventRecord(h->ev0, s));

    std::vector<long long> blk_iters;
    int status = GSPCA_OK, found = 0;
    long long total = 0;
    bool not_converged = false;
    for (int k0 = 0; k0 < K; k0 += block) {
        const int bw = (K - k0) < block ? (K - k0) : block;
        GS_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int) * 4, s));
        GS_CUDA(cudaMemsetAsync(w.sp, 0, sizeof(double) * kBlkMax, s));
        // U = R^T R(:, k0 .. k0+bw-1), against U_(k0), orthonormal
        BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_T, CUBLAS_OP_N, N, bw, M, &one, R, M, R + (size_t)k0 * M, M, &zero, w.Z, N));
        if (project_out(cb, P, N, k0, w.Z, bw, w.tmp) != GSPCA_OK) return GSPCA_ERR_CUDA;
        if (cholqr2(cb, s, w.Z, w.U, N, bw, w, false, &launches) != GSPCA_OK) return GSPCA_ERR_CUDA;
        int j = 0, fl = 0;
        for (;;) {
            // Y = R U, against V_(k0), orthonormal -> V
            BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_N, CUBLAS_OP_N, M, bw, N, &one, R, M, w.U, N, &zero, w.Y, M));
            if (project_out(cb, T, M, k0, w.Y, bw, w.tmp) != GSPCA_OK) return GSPCA_ERR_CUDA;
            if (cholqr2(cb, s, w.Y, w.V, M, bw, w, false, &launches) != GSPCA_OK) return GSPCA_ERR_CUDA;
            // Z = R^T V, against U_(k0); Ritz values from Z^T Z
            BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_T, CUBLAS_OP_N, N, bw, M, &one, R, M, w.V, M, &zero, w.Z, N));
            if (project_out(cb, P, N, k0, w.Z, bw, w.tmp) != GSPCA_OK) return GSPCA_ERR_CUDA;
            gram(s, w.Z, N, w.Z, N, N, bw, bw, w, w.G);
            jacobi_eig_kernel<<<1, 256, 0, s>>>(w.G, bw, w.ev, w.evec);
            ritz_test_kernel<<<1, 1, 0, s>>>(w.ev, w.sp, bw, tol, w.flag);
            launches += 6 + (k0 > 0 ? 4 : 0);
            ++j;
            ++total;
            GS_CUDA(cudaMemcpyAsync(h->h_blk, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
            GS_CUDA(cudaStreamSynchronize(s));
            fl = h->h_blk[0];
            if (fl & 1) break;  // dependent columns
            bool stop;
            if (opts && opts->iters_lock) {
                stop = j >= opts->iters_lock[k0];
            } else {
                stop = (fl & 2) != 0;
                if (!stop && j >= max_iter) {
                    stop = true;
                    not_converged = true;
                }
            }
            if (stop) break;
            GS_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int), s));
            // U = qr(Z), the Gram matrix Z^T Z is already in w.G
            if (cholqr2(cb, s, w.Z, w.U, N, bw, w, true, &launches) != GSPCA_OK) return GSPCA_ERR_CUDA;
        }
        if (fl & 1) {
            status = GSPCA_ERR_DEGENERATE;
            break;
        }
        // Rayleigh-Ritz: B = Z^T U (FP64), B^T B = Zh diag(sigma^2) Zh^T, Yh = B Zh / sigma
        gram(s, w.Z, N, w.U, N, N, bw, bw, w, w.Bm);
        btb_kernel<<<1, 1024, 0, s>>>(w.Bm, bw, w.G);
        jacobi_eig_kernel<<<1, 256, 0, s>>>(w.G, bw, w.ev, w.evec);
        ritz_rot_kernel<<<1, 1024, 0, s>>>(w.Bm, w.ev, w.evec, bw, w.sigma, w.Yh, w.Zh, w.flag);
        launches += 5;
        // V <- V Yh (into T's columns), U <- U Zh (into P's columns)
        BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_N, CUBLAS_OP_N, M, bw, bw, &one, w.V, M, w.Yh, bw, &zero,
                              T + (size_t)k0 * M, M));
        BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_N, CUBLAS_OP_N, N, bw, bw, &one, w.U, N, w.Zh, bw, &zero,
                              P + (size_t)k0 * N, N));
        // R -= (V diag(sigma)) U^T
        scale_cols_kernel<<<256, 256, 0, s>>>(T + (size_t)k0 * M, M, w.Y, M, M, bw, w.sigma);
        BL_CUBLAS(cublasSgemm(cb, CUBLAS_OP_N, CUBLAS_OP_T, M, N, bw, &mone, w.Y, M, P + (size_t)k0 * N, N, &one, R, M));
        GS_CUDA(cudaMemcpyAsync(lambda + k0, w.sigma, sizeof(double) * bw, cudaMemcpyDeviceToDevice, s));
        GS_CUDA(cudaMemcpyAsync(h->h_blk, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        GS_CUDA(cudaStreamSynchronize(s));
        if (h->h_blk[0] & 1) {
            status = GSPCA_ERR_DEGENERATE;
            break;
        }
        if (iters) {
            int hi[kBlkMax];
            for (int i = 0; i < bw; ++i) hi[i] = j;
            GS_CUDA(cudaMemcpyAsync(iters + k0, hi, sizeof(int) * bw, cudaMemcpyHostToDevice, s));
            GS_CUDA(cudaStreamSynchronize(s));
        }
        found = k0 + bw;
        blk_iters.push_back(j);
        launches += 2;
    }
    GS_CUDA(cudaEventRecord(h->ev1, s));
    // T = V Lambda (unless the SVD form is asked for); zero past `found`
    if (!(opts && opts->svd_form == 1) && found > 0) {
        scale_cols_kernel<<<256, 256, 0, s>>>(T, M, T, M, M, found, lambda);
        ++launches;
    }
    if (found < K) {
        GS_CUDA(cudaMemsetAsync(T + (size_t)found * M, 0, sizeof(float) * (size_t)M * (K - found), s));
        GS_CUDA(cudaMemsetAsync(P + (size_t)found * N, 0, sizeof(float) * (size_t)N * (K - found), s));
        GS_CUDA(cudaMemsetAsync(lambda + found, 0, sizeof(double) * (K - found), s));
        if (iters) GS_CUDA(cudaMemsetAsync(iters + found, 0, sizeof(int) * (K - found), s));
    }
    if (R_out) GS_CUDA(cudaMemcpyAsync(R_out, R, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToDevice, s));
    GS_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    GS_CUDA(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    h->last.kernel_ms = ms;
    h->last.found = found;
    h->last.total_iters = total;
    h->last.kernel_launches = launches;
    h->last.grid_ctas = kGramCtas;
    h->last.team_ctas = 0;
    h->last.block_threads = 1024;
    h->last.batch_pass = 0;
    // algorithmic bytes: per iteration R read twice (R U, R^T V) and the factors of the earlier
    // blocks twice on each side (projections); per block R read and written once (deflation)
    {
        double bytes = 0.0;
        int k0 = 0;
        for (const long long it : blk_iters) {
            bytes += (double)it * (8.0 * M * N + 16.0 * (double)(M + N) * k0) + 8.0 * M * N;
            k0 += block;
        }
        h->last.alg_bytes = bytes;
    }
    if (status == GSPCA_ERR_DEGENERATE) return GSPCA_ERR_DEGENERATE;
    if (not_converged) return GSPCA_WARN_NOT_CONVERGED;
    return GSPCA_OK;
}
