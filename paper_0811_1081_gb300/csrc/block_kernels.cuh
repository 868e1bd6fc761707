// Small dense kernels of the block power iteration (gspca_fit_block): Gram
// matrices with FP64 accumulation, Cholesky factor inverse (CholQR), a
// symmetric eigensolver for b x b matrices, the convergence test, and the
// output scaling.  The large products (R U, R^T V, projections, the rank-b
// deflation) are plain FP32 GEMMs of cuBLAS.  Every sum runs in a fixed order.
#pragma once

#include <cfloat>

#include "device_common.cuh"

namespace gspca {

constexpr int kBlkMax = 32;          // widest block
constexpr int kGramRows = 64;        // rows per staged chunk of the Gram kernel
constexpr int kGramCtas = 128;       // CTAs of the Gram kernel (partials summed in CTA order)

// part[g] (n x m, FP64, column-major) = sum over the rows of CTA g of A^T B, with
// A (rows x n, lda) and B (rows x m, ldb) FP32 column-major; n, m <= kBlkMax.
// A thread per (i, j); rows staged in shared memory, summed in row order.
__global__ void __launch_bounds__(1024) gram_part_kernel(const float* A, int lda, const float* B, int ldb, int rows,
                                                         int n, int m, double* part) {
    __shared__ float sa[kGramRows][kBlkMax + 1];
    __shared__ float sb[kGramRows][kBlkMax + 1];
    const int t = threadIdx.x, i = t % kBlkMax, j = t / kBlkMax;
    const int G = gridDim.x, g = blockIdx.x;
    const int r0 = (int)(((long long)g * rows) / G), r1 = (int)(((long long)(g + 1) * rows) / G);
    double acc = 0.0;
    for (int rb = r0; rb < r1; rb += kGramRows) {
        const int nr = min(kGramRows, r1 - rb);
        for (int e = t; e < kGramRows * kBlkMax; e += blockDim.x) {
            const int r = e % kGramRows, c = e / kGramRows;
            sa[r][c] = (r < nr && c < n) ? A[(size_t)c * lda + rb + r] : 0.f;
            sb[r][c] = (r < nr && c < m) ? B[(size_t)c * ldb + rb + r] : 0.f;
        }
        __syncthreads();
        if (i < n && j < m)
            for (int r = 0; r < nr; ++r) acc = fma((double)sa[r][i], (double)sb[r][j], acc);
        __syncthreads();
    }
    if (i < n && j < m) part[(size_t)g * n * m + (size_t)j * n + i] = acc;
}

// out (n x m) = sum of the G partials in CTA order.
__global__ void gram_sum_kernel(const double* part, int G, int n, int m, double* out) {
    for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
        double t = 0.0;
        for (int g = 0; g < G; ++g) t += part[(size_t)g * n * m + e];
        out[e] = t;
    }
}

// Cholesky G = S^T S (S upper triangular, positive diagonal) of the n x n FP64
// Gram matrix, and Sinv = S^{-1} written as FP32 (n x n column-major, zero below
// the diagonal).  One CTA.  *flag |= 1 when a pivot is not above 1e-12 of the
// largest diagonal entry of G (numerically dependent columns); Sinv is then the
// identity.
__global__ void chol_inv_kernel(const double* G, int n, float* Sinv, int* flag) {
    __shared__ double a[kBlkMax][kBlkMax + 1];
    __shared__ double x[kBlkMax][kBlkMax + 1];
    __shared__ int bad;
    __shared__ double dmax;
    const int t = threadIdx.x;
    for (int e = t; e < n * n; e += blockDim.x) a[e % n][e / n] = G[e];
    if (t == 0) {
        bad = 0;
        double d = 0.0;
        for (int i = 0; i < n; ++i) d = fmax(d, G[(size_t)i * n + i]);
        dmax = d;
    }
    __syncthreads();
    // right-looking: column k of S^T is row k of S; a holds the trailing matrix
    for (int k = 0; k < n; ++k) {
        if (t == 0) {
            const double p = a[k][k];
            if (!(p > 1e-12 * dmax)) bad = 1;
            a[k][k] = sqrt(p > 0.0 ? p : 1.0);
        }
        __syncthreads();
        const double d = a[k][k];
        for (int j = k + 1 + t; j < n; j += blockDim.x) a[k][j] /= d;  // row k of S
        __syncthreads();
        for (int e = t; e < (n - k - 1) * (n - k - 1); e += blockDim.x) {
            const int i = k + 1 + e % (n - k - 1), j = k + 1 + e / (n - k - 1);
            if (i <= j) a[i][j] -= a[k][i] * a[k][j];
        }
        __syncthreads();
    }
    // S X = I, column j of X by back substitution (a thread per column)
    for (int j = t; j < n; j += blockDim.x) {
        for (int i = n - 1; i >= 0; --i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int l = i + 1; l < n; ++l) s -= a[i][l] * x[l][j];
            x[i][j] = s / a[i][i];
        }
    }
    __syncthreads();
    for (int e = t; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        Sinv[e] = bad ? (i == j ? 1.f : 0.f) : (i <= j ? (float)x[i][j] : 0.f);
    }
    if (t == 0 && bad) atomicOr(flag, 1);
}

// Symmetric eigen-decomposition of the n x n FP64 matrix G (column-major) by
// the cyclic Jacobi method with the parallel (round-robin) pair ordering of
// Golub & Van Loan Sec. 8.5: every step rotates n/2 disjoint pairs at once.
// Sweeps until the off-diagonal norm is at most 1e-15 ||G||_F (at most 40).
// evals: decreasing; evecs (n x n column-major) the matching unit vectors.  One CTA.
__global__ void jacobi_eig_kernel(const double* G, int n, double* evals, double* evecs) {
    __shared__ double A[kBlkMax][kBlkMax + 1];
    __shared__ double W[kBlkMax][kBlkMax + 1];
    __shared__ double cs[kBlkMax / 2][2];
    __shared__ int pr[kBlkMax / 2][2];
    __shared__ int perm[kBlkMax + 1];
    __shared__ double off, tot;
    __shared__ int order[kBlkMax];
    const int t = threadIdx.x;
    const int n2 = (n + 1) / 2 * 2;  // an odd n plays with a dummy index n
    for (int e = t; e < kBlkMax * kBlkMax; e += blockDim.x) {
        const int i = e % kBlkMax, j = e / kBlkMax;
        A[i][j] = (i < n && j < n) ? G[(size_t)j * n + i] : 0.0;
        W[i][j] = (i == j) ? 1.0 : 0.0;
    }
    if (t <= kBlkMax) perm[t] = t;
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (t == 0) {
            double o = 0.0, s = 0.0;
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    s += A[i][j] * A[i][j];
                    if (i != j) o += A[i][j] * A[i][j];
                }
            off = o;
            tot = s;
        }
        __syncthreads();
        if (!(off > 1e-30 * tot)) break;
        for (int step = 0; step < n2 - 1; ++step) {
            // pairs (perm[q], perm[n2 - 1 - q]) (the circle method: over n2 - 1 steps every
            // pair meets once); rotation angles from the current A
            if (t < n2 / 2) {
                int p = perm[t], q = perm[n2 - 1 - t];
                if (p > q) {
                    const int s = p;
                    p = q;
                    q = s;
                }
                double c = 1.0, s = 0.0;
                if (q < n && A[p][q] != 0.0) {
                    const double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                    const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + tt * tt);
                    s = tt * c;
                }
                pr[t][0] = p;
                pr[t][1] = q;
                cs[t][0] = c;
                cs[t][1] = s;
            }
            __syncthreads();
            // A <- A J (columns), W <- W J: a thread per (pair, row)
            for (int e = t; e < (n2 / 2) * n; e += blockDim.x) {
                const int pi = e / n, i = e % n, p = pr[pi][0], q = pr[pi][1];
                if (q < n) {
                    const double c = cs[pi][0], s = cs[pi][1];
                    const double aip = A[i][p], aiq = A[i][q];
                    A[i][p] = c * aip - s * aiq;
                    A[i][q] = s * aip + c * aiq;
                    const double wip = W[i][p], wiq = W[i][q];
                    W[i][p] = c * wip - s * wiq;
                    W[i][q] = s * wip + c * wiq;
                }
            }
            __syncthreads();
            // A <- J^T A (rows)
            for (int e = t; e < (n2 / 2) * n; e += blockDim.x) {
                const int pi = e / n, i = e % n, p = pr[pi][0], q = pr[pi][1];
                if (q < n) {
                    const double c = cs[pi][0], s = cs[pi][1];
                    const double api = A[p][i], aqi = A[q][i];
                    A[p][i] = c * api - s * aqi;
                    A[q][i] = s * api + c * aqi;
                }
            }
            __syncthreads();
            // next arrangement: position 0 fixed, the others rotate by one
            if (t == 0) {
                const int last = perm[n2 - 1];
                for (int i = n2 - 1; i > 1; --i) perm[i] = perm[i - 1];
                perm[1] = last;
            }
            __syncthreads();
        }
    }
    if (t == 0) {  // decreasing eigenvalues (selection order, lowest index on ties)
        for (int i = 0; i < n; ++i) order[i] = i;
        for (int i = 0; i < n; ++i) {
            int best = i;
            for (int j = i + 1; j < n; ++j)
                if (A[order[j]][order[j]] > A[order[best]][order[best]]) best = j;
            const int s = order[i];
            order[i] = order[best];
            order[best] = s;
        }
    }
    __syncthreads();
    for (int e = t; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        evecs[e] = W[i][order[j]];
    }
    if (t < n) evals[t] = A[order[t]][order[t]];
}

// Ritz values s_i = sqrt(max(ev_i, 0)); stop flag (bit 1 of *flag) when every
// |s_i - sp_i| < tol s_i; then sp <- s.  One thread.
__global__ void ritz_test_kernel(const double* ev, double* sp, int n, double tol, int* flag) {
    int stop = 1;
    for (int i = 0; i < n; ++i) {
        const double s = sqrt(ev[i] > 0.0 ? ev[i] : 0.0);
        if (!(fabs(sp[i] - s) < tol * s)) stop = 0;
        sp[i] = s;
    }
    if (stop) atomicOr(flag, 2);
}

// G = B^T B (n x n, FP64, column-major) of the n x n FP64 matrix B.  One CTA.
__global__ void btb_kernel(const double* B, int n, double* G) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        double s = 0.0;
        for (int l = 0; l < n; ++l) s = fma(B[(size_t)i * n + l], B[(size_t)j * n + l], s);
        G[e] = s;
    }
}

// Rayleigh-Ritz rotations from B (n x n, FP64) and the eigenpairs of B^T B:
// sigma_i = sqrt(ev_i); Zh (FP32) = the eigenvectors; Yh (FP32) = B Zh / sigma.
// *flag |= 1 when a sigma is zero.  One CTA.
__global__ void ritz_rot_kernel(const double* B, const double* ev, const double* evec, int n, double* sigma,
                                float* Yh, float* Zh, int* flag) {
    const int t = threadIdx.x;
    for (int e = t; e < n * n; e += blockDim.x) {
        const int i = e % n, j = e / n;
        const double sj = sqrt(ev[j] > 0.0 ? ev[j] : 0.0);
        double s = 0.0;
        for (int l = 0; l < n; ++l) s = fma(B[(size_t)l * n + i], evec[(size_t)j * n + l], s);
        Yh[e] = sj > 0.0 ? (float)(s / sj) : 0.f;
        Zh[e] = (float)evec[e];
    }
    if (t < n) {
        sigma[t] = sqrt(ev[t] > 0.0 ? ev[t] : 0.0);
        if (!(sigma[t] > 0.0)) atomicOr(flag, 1);
    }
}

// D (rows x n, ld) = S (rows x n, lds) with column j scaled by sigma[j].
__global__ void scale_cols_kernel(const float* S, int lds, float* D, int ld, int rows, int n, const double* sigma) {
    const size_t total = (size_t)rows * n, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int r = (int)(e % rows), j = (int)(e / rows);
        D[(size_t)j * ld + r] = (float)((double)S[(size_t)j * lds + r] * sigma[j]);
    }
}

// R (M x N, ld M, column-major FP32) <- X with optional centring (1: column
// means, 2: row means, both FP64), ||R||_F^2 not needed here.
__global__ void pack_colmajor_kernel(const float* X, int layout, long ldx, int M, int N, int center,
                                     const double* cmean, const double* rmean, float* R) {
    const size_t total = (size_t)M * N, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        int r, c;
        if (layout == 0) {
            r = (int)(e % M);
            c = (int)(e / M);
        } else {
            r = (int)(e / N);
            c = (int)(e % N);
        }
        float v = layout == 0 ? X[(size_t)c * ldx + r] : X[(size_t)r * ldx + c];
        if (center == 1) v = (float)((double)v - cmean[c]);
        else if (center == 2) v = (float)((double)v - rmean[r]);
        R[(size_t)c * M + r] = v;
    }
}

}  // namespace gspca
