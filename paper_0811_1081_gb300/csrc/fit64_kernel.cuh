// FP64 storage path: NIPALS-PCA (Sec. 2.2) and GS-PCA (Sec. 2.3) with R, the
// factors and every product in IEEE double, the precision of the paper's
// programs (Sec. 3).  One persistent cooperative launch runs every iteration
// of every component, as the FP32 kernel does, in a simpler form:
//   - R is row-major (M x N, leading dimension N); CTA g owns the rows
//     [r0, r1) and the column slice [n0, n1);
//   - one sweep per iteration: the CTA's rows reach shared memory in chunks of
//     rc rows, v' = R u' is formed per row (a warp per row) and, from the same
//     staged chunk, s' = R^T v' is accumulated per column (a thread per column);
//   - the Gram-Schmidt score correction commutes through R^T: R^T (v' - V b')
//     = s' - W b', with W = R^T V kept by a rank-1 update per deflation, so the
//     loading needs no second read of R;
//   - three grid-wide reductions per GS iteration (after the pass: s', b',
//     ||v'||^2; after the score step: a' = U^T u_pre', ||v' - V b'||^2; after the
//     next loading: its squared norm), every cross-CTA sum in CTA order, so two
//     runs give the same bits;
//   - the deflation of component k-1 (Eq. 3) is applied inside the sweep that
//     takes the start column R(k) of component k.
// GB300 executes FP64 at a small fraction of its FP32 rate, so this path is
// bound by the FP64 pipes, not by memory.
#pragma once

#include <cfloat>

#include "device_common.cuh"

namespace gspca {

constexpr int kBlock64 = 512;
constexpr int kWarps64 = kBlock64 / 32;
constexpr int kMaxRc64 = 16;  // rows per staged chunk (at most one per warp)

struct Fit64Args {
    int M, N, K;
    int algo;                 // 0 = NIPALS, 1 = GS
    int max_iter;
    double tol;
    double eps_thresh;        // degenerate threshold factor: lambda <= eps_thresh * ||X||_F
    const double* xpart;      // partial sums of squares of the packed X
    int nxpart;
    double* R;                // M x N row-major
    double* V;                // M x ldk row-major (GS: unit score directions; NIPALS: scores t)
    double* U;                // N x ldk row-major (loadings)
    double* W;                // N x ldk row-major (R^T V, GS)
    int ldk;
    double* vraw;             // M: v' of the last pass
    double* vcorr;            // M: v' - V b'
    double* ut;               // 2 x N: pass input, double-buffered
    double* upre;             // N: s' - W b' (pass scale)
    double* partS;            // G x LS: s' (or s0, column norms) partials, then the k-vector
    int LS;
    double* partA;            // G x ldk: a' partials
    double* scal;             // G x 4: [0] ||v'||^2 / ||x||^2, [1] ||v' - V b'||^2, [2+b] ||ut[b]||^2
    double* lam;              // K
    int* iters;               // K
    int* info;                // status, found, total iterations (lo, hi)
    unsigned* flags;          // barrier arrival counter, zeroed before the launch
    int* abort;
    const int* iters_lock;    // device, K entries, nullable
    unsigned long long timeout_ns;
    int rc;                   // rows per staged chunk
};

// Shared memory (dynamic): u (N), s accumulators (N), chunk (rc x N), then
// small vectors: row values (kMaxRc64), kb (ldk), ka (ldk), slice (max N / G + 1).
struct Smem64 {
    double* u;
    double* s;
    double* ch;
    double* rowv;
    double* kb;
    double* ka;
    double* sl;
};

__device__ __forceinline__ Smem64 carve64(unsigned char* dyn, const Fit64Args& f, int max_slice) {
    Smem64 m;
    double* p = reinterpret_cast<double*>(dyn);
    m.u = p;
    p += f.N;
    m.s = p;
    p += f.N;
    m.ch = p;
    p += (size_t)f.rc * f.N;
    m.rowv = p;
    p += kMaxRc64;
    m.kb = p;
    p += f.ldk;
    m.ka = p;
    p += f.ldk;
    m.sl = p;
    (void)max_slice;
    return m;
}

// Bytes of dynamic shared memory for N columns, rc rows per chunk, ldk, a slice.
__host__ __device__ inline size_t smem64_bytes(int N, int rc, int ldk, int max_slice) {
    return sizeof(double) * ((size_t)(2 + rc) * N + kMaxRc64 + 2 * (size_t)ldk + max_slice);
}

// CTA-wide sum of one double per thread, in a fixed order (warp butterflies,
// then the warp sums in index order); the result in every thread.
__device__ __forceinline__ double block_sum64(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Sum over the G CTA rows of column c of a G x L partial buffer, in CTA order.
__device__ __forceinline__ double col_sum64(const double* part, int G, int L, int c) {
    double t = 0.0;
#pragma unroll 8
    for (int g = 0; g < G; ++g) t += __ldcg(part + (size_t)g * L + c);
    return t;
}

// One sweep over the CTA's rows [r0, r1).
//   start == false: row value x_r = R_r . u (u in smem), written to vraw;
//   start == true:  with `deflate`, R_r <- R_r - a_r u^T first (a_r = lamf V[r, kprev],
//                   u = the previous loading in smem; the deflated rows are stored),
//                   then x_r = R[r, kcol].
// Both accumulate s[c] += R[r, c] x_r (smem, a thread per column) and return the
// CTA's sum of x_r^2 (every thread).  Sums run in row order within the CTA.
__device__ __forceinline__ double sweep64(const Fit64Args& f, const Smem64& m, double* red, int r0, int r1,
                                          bool start, bool deflate, double lamf, int kprev, int kcol) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = blockDim.x, N = f.N;
    for (int c = tid; c < N; c += T) m.s[c] = 0.0;
    double sq = 0.0;
    for (int rb = r0; rb < r1; rb += f.rc) {
        const int nr = min(f.rc, r1 - rb);
        const double* src = f.R + (size_t)rb * N;
        for (int i = tid; i < nr * N; i += T) m.ch[i] = src[i];
        __syncthreads();
        if (start && deflate) {
            for (int i = tid; i < nr * N; i += T) {
                const int r = rb + i / N, c = i % N;
                const double v = fma(-lamf * f.V[(size_t)r * f.ldk + kprev], m.u[c], m.ch[i]);
                m.ch[i] = v;
                f.R[(size_t)rb * N + i] = v;
            }
            __syncthreads();
        }
        if (start) {
            if (tid < nr) m.rowv[tid] = m.ch[(size_t)tid * N + kcol];
        } else {
            for (int i = warp; i < nr; i += kWarps64) {
                const double* row = m.ch + (size_t)i * N;
                double a = 0.0;
                for (int c = lane; c < N; c += 32) a = fma(row[c], m.u[c], a);
                a = warp_sum(a);
                if (lane == 0) {
                    m.rowv[i] = a;
                    f.vraw[rb + i] = a;
                }
            }
        }
        __syncthreads();
        if (tid < nr) sq = fma(m.rowv[tid], m.rowv[tid], sq);
        for (int c = tid; c < N; c += T) {
            double a = m.s[c];
            for (int i = 0; i < nr; ++i) a = fma(m.ch[(size_t)i * N + c], m.rowv[i], a);
            m.s[c] = a;
        }
        __syncthreads();
    }
    return block_sum64(sq, red);
}

// dst[j] = sum_{r in [a0, a1)} A[r * lda + j] y(r), j < kk: a thread per j, rows in order.
template <class Y>
__device__ __forceinline__ void rows_t64(const double* A, int lda, int a0, int a1, int kk, Y y, double* dst) {
    for (int j = threadIdx.x; j < kk; j += blockDim.x) {
        double t = 0.0;
        for (int r = a0; r < a1; ++r) t = fma(A[(size_t)r * lda + j], y(r), t);
        dst[j] = t;
    }
}

// For every r in [a0, a1): fn(r, sum_j A[r * lda + j] x[j]) with x (kk) in smem; a
// warp per row, lanes over j, fixed butterfly; fn runs in lane 0.
template <class Fn>
__device__ __forceinline__ void rows_dot64(const double* A, int lda, int a0, int a1, int kk, const double* x, Fn fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = a0 + warp; r < a1; r += kWarps64) {
        double t = 0.0;
        for (int j = lane; j < kk; j += 32) t = fma(A[(size_t)r * lda + j], x[j], t);
        t = warp_sum(t);
        if (lane == 0) fn(r, t);
    }
}

// Thread 0 sums slot `slot` of the G x 4 scalar partials in CTA order; the value
// is returned in every thread.
__device__ __forceinline__ double scal_sum64(const Fit64Args& f, int G, int slot, double* bc) {
    if (threadIdx.x == 0) *bc = col_sum64(f.scal, G, 4, slot);
    __syncthreads();
    const double v = *bc;
    __syncthreads();
    return v;
}

// Single problem, whole grid (cooperative launch), FP64 throughout.
__global__ void __launch_bounds__(kBlock64, 1) fit64_kernel(const Fit64Args f) {
    extern __shared__ __align__(16) unsigned char dyn64[];
    __shared__ double red[kWarps64];
    __shared__ double bc;
    __shared__ int s_flag;
    __shared__ double s_best[kWarps64];
    __shared__ int s_bidx[kWarps64];
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int M = f.M, N = f.N, K = f.K;
    const int r0 = (int)(((long long)g * M) / G), r1 = (int)(((long long)(g + 1) * M) / G);
    const int n0 = (int)(((long long)g * N) / G), n1 = (int)(((long long)(g + 1) * N) / G);
    const Smem64 m = carve64(dyn64, f, (N + G - 1) / G + 1);
    const GridBarrier bar{f.flags, f.abort, f.timeout_ns};
    unsigned epoch = 0;
    const bool gs = f.algo == 1;
    double xx = 0.0;  // ||X||_F^2 from the pack kernel's partials, in order
    for (int i = 0; i < f.nxpart; ++i) xx += f.xpart[i];
    const double thresh = f.eps_thresh * sqrt(xx);
    double* pS = f.partS + (size_t)g * f.LS;
    double* pA = f.partA + (size_t)g * f.ldk;
    double* sc = f.scal + (size_t)g * 4;
    int status = kStOK, found = K;
    long long total = 0;
    bool alive = true;
    double lam_prev = 0.0, vinv_prev = 0.0, inv_nu = 0.0;
    int buf = 0;

#define SYNC64()                             \
    do {                                     \
        if (!bar.sync(epoch, &s_flag)) {     \
            alive = false;                   \
            goto leave64;                    \
        }                                    \
    } while (0)

    for (int k = 0; k < K && found == K; ++k) {
        // ------------- start: deflate component k-1 in the sweep that takes R(k)
        const bool defl = k > 0;
        const double lamf = gs ? lam_prev : 1.0;
        // u_{k-1} = the last pass input / its norm: complete behind the barrier before that pass
        // (U(k-1) itself was written slice by slice when the component stopped, with no barrier since)
        if (defl)
            for (int c = tid; c < N; c += T) m.u[c] = __ldcg(f.ut + (size_t)buf * N + c) * inv_nu;
        __syncthreads();
        double xs = sweep64(f, m, red, r0, r1, true, defl, lamf, k - 1, k);
        for (int c = tid; c < N; c += T) pS[c] = m.s[c];
        if (gs && k > 0)  // Gram row v_{k-1} . v_j over this CTA's rows
            rows_t64(f.V, f.ldk, r0, r1, k, [&](int r) { return f.V[(size_t)r * f.ldk + (k - 1)]; }, pS + N);
        if (tid == 0) sc[0] = xs;
        SYNC64();
        double xxs = scal_sum64(f, G, 0, &bc);
        if (xxs == 0.0) {
            // Zero start column: the residual column of largest norm (lowest index on ties);
            // every column zero => rank exhausted.
            for (int c = tid; c < N; c += T) {
                double t = 0.0;
                for (int r = r0; r < r1; ++r) t = fma(f.R[(size_t)r * N + c], f.R[(size_t)r * N + c], t);
                pS[c] = t;
            }
            SYNC64();
            double best = 0.0;
            int bi = N;
            for (int c = tid; c < N; c += T) {
                const double v = col_sum64(f.partS, G, f.LS, c);
                if (v > best) {
                    best = v;
                    bi = c;
                }
            }
            for (int o = 16; o >= 1; o >>= 1) {
                const double ob = __shfl_xor_sync(kFull, best, o);
                const int oi = __shfl_xor_sync(kFull, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (lane == 0) {
                s_best[warp] = best;
                s_bidx[warp] = bi;
            }
            __syncthreads();
            best = 0.0;
            bi = N;
            for (int w = 0; w < kWarps64; ++w)
                if (s_best[w] > best || (s_best[w] == best && s_bidx[w] < bi)) {
                    best = s_best[w];
                    bi = s_bidx[w];
                }
            __syncthreads();
            if (!(best > 0.0)) {
                found = k;
                status = kStDegenerate;
                break;
            }
            xs = sweep64(f, m, red, r0, r1, true, false, 0.0, 0, bi);
            for (int c = tid; c < N; c += T) pS[c] = m.s[c];
            if (tid == 0) sc[0] = xs;
            SYNC64();
            xxs = scal_sum64(f, G, 0, &bc);
        }
        for (int c = n0 + tid; c < n1; c += T) m.sl[c - n0] = col_sum64(f.partS, G, f.LS, c);
        if (gs && k > 0)
            for (int jj = tid; jj < k; jj += T) m.kb[jj] = col_sum64(f.partS, G, f.LS, N + jj);
        __syncthreads();
        if (gs && k > 0) {
            // W <- R_k^T V for the deflation of component k-1: W(:, j) -= lambda u (v_{k-1} . v_j),
            // new column R_{k-1}^T v_{k-1} - lambda u |v_{k-1}|^2 with R_{k-1}^T v_{k-1} = u_pre / ||v' - V b'||
            const int km = k - 1;
            for (int e = tid; e < (n1 - n0) * k; e += T) {
                const int n = n0 + e / k, jj = e % k;
                const double un = f.U[(size_t)n * f.ldk + km];
                double* w = f.W + (size_t)n * f.ldk + jj;
                if (jj < km)
                    *w = fma(-lam_prev * un, m.kb[jj], *w);
                else
                    *w = fma(-lam_prev * un, m.kb[km], f.upre[n] * vinv_prev);
            }
            __syncthreads();
            // a = U_(k)^T s0 over the slice
            rows_t64(f.U, f.ldk, n0, n1, k, [&](int n) { return m.sl[n - n0]; }, pA);
            SYNC64();
            for (int jj = tid; jj < k; jj += T) m.ka[jj] = col_sum64(f.partA, G, f.ldk, jj);
            __syncthreads();
        }
        {
            const double xx_inv = 1.0 / xxs;  // keeps the first loading's norm O(1)
            const int nb = buf ^ 1;
            double nq = 0.0;
            if (gs && k > 0) {
                rows_dot64(f.U, f.ldk, n0, n1, k, m.ka, [&](int n, double s) {
                    const double un = (m.sl[n - n0] - s) * xx_inv;
                    f.ut[(size_t)nb * N + n] = un;
                    nq = fma(un, un, nq);
                });
            } else {
                for (int n = n0 + tid; n < n1; n += T) {
                    const double un = m.sl[n - n0] * xx_inv;
                    f.ut[(size_t)nb * N + n] = un;
                    nq = fma(un, un, nq);
                }
            }
            nq = block_sum64(nq, red);
            if (tid == 0) sc[2 + nb] = nq;
            buf = nb;
        }
        SYNC64();

        // ------------- power iterations
        double mu = 0.0;
        int j = 0;
        for (;;) {
            for (int c = tid; c < N; c += T) m.u[c] = __ldcg(f.ut + (size_t)buf * N + c);
            __syncthreads();
            const double vs = sweep64(f, m, red, r0, r1, false, false, 0.0, 0, 0);
            for (int c = tid; c < N; c += T) pS[c] = m.s[c];
            if (gs && k > 0)  // b' = V_(k)^T v' over this CTA's rows
                rows_t64(f.V, f.ldk, r0, r1, k, [&](int r) { return f.vraw[r]; }, pS + N);
            if (tid == 0) sc[0] = vs;
            SYNC64();
            ++j;
            ++total;
            const double nu2 = scal_sum64(f, G, 2 + buf, &bc);
            const double nvp = scal_sum64(f, G, 0, &bc);
            for (int c = n0 + tid; c < n1; c += T) m.sl[c - n0] = col_sum64(f.partS, G, f.LS, c);
            if (gs && k > 0)
                for (int jj = tid; jj < k; jj += T) m.kb[jj] = col_sum64(f.partS, G, f.LS, N + jj);
            __syncthreads();
            if (!(nu2 > 0.0)) {
                found = k;
                status = kStDegenerate;
                break;
            }
            inv_nu = 1.0 / sqrt(nu2);
            const int nbuf = buf ^ 1;
            double l2;  // ||v' - V b'||^2 (GS) or ||v'||^2, pass scale
            if (!gs || k == 0) {
                l2 = nvp;
                if (gs)
                    for (int n = n0 + tid; n < n1; n += T) f.upre[n] = m.sl[n - n0];
            } else {
                // v_corr = v' - V b' (rows); u_pre = s' - W b' (slice); a' = U^T u_pre (partials)
                double lp = 0.0;
                rows_dot64(f.V, f.ldk, r0, r1, k, m.kb, [&](int r, double s) {
                    const double vc = f.vraw[r] - s;
                    f.vcorr[r] = vc;
                    lp = fma(vc, vc, lp);
                });
                rows_dot64(f.W, f.ldk, n0, n1, k, m.kb, [&](int n, double s) { f.upre[n] = m.sl[n - n0] - s; });
                __syncthreads();
                rows_t64(f.U, f.ldk, n0, n1, k, [&](int n) { return f.upre[n]; }, pA);
                lp = block_sum64(lp, red);
                if (tid == 0) sc[1] = lp;
                SYNC64();
                l2 = scal_sum64(f, G, 1, &bc);
                for (int jj = tid; jj < k; jj += T) m.ka[jj] = col_sum64(f.partA, G, f.ldk, jj);
                __syncthreads();
            }
            // lambda and the relative strict test (Sec. 2.2 / 2.3, as the appendix programs)
            const double lam = sqrt(l2 / nu2);
            int stop;
            if (!(lam > thresh)) {
                stop = 2;
            } else if (f.iters_lock != nullptr) {
                stop = j >= f.iters_lock[k];
            } else {
                stop = fabs(mu - lam) < f.tol * lam;
                if (!stop && j >= f.max_iter) stop = 3;
            }
            if (stop == 2) {
                found = k;
                status = kStDegenerate;
                break;
            }
            if (stop) {
                if (stop == 3 && status == kStOK) status = kStNotConverged;
                const double vinv = 1.0 / sqrt(l2);
                for (int r = r0 + tid; r < r1; r += T)
                    f.V[(size_t)r * f.ldk + k] = gs ? ((k > 0) ? f.vcorr[r] : f.vraw[r]) * vinv : f.vraw[r] * inv_nu;
                for (int n = n0 + tid; n < n1; n += T)
                    f.U[(size_t)n * f.ldk + k] = __ldcg(f.ut + (size_t)buf * N + n) * inv_nu;
                lam_prev = lam;
                vinv_prev = vinv;
                if (g == 0 && tid == 0) {
                    f.lam[k] = lam;
                    f.iters[k] = j;
                }
                break;
            }
            mu = lam;
            const double nscale = sqrt(nu2) / l2;  // keeps ||ut|| ~ 1
            double nq2 = 0.0;
            if (!gs || k == 0) {
                for (int n = n0 + tid; n < n1; n += T) {
                    const double un = m.sl[n - n0] * nscale;
                    f.ut[(size_t)nbuf * N + n] = un;
                    nq2 = fma(un, un, nq2);
                }
            } else {
                rows_dot64(f.U, f.ldk, n0, n1, k, m.ka, [&](int n, double s) {
                    const double un = (f.upre[n] - s) * nscale;
                    f.ut[(size_t)nbuf * N + n] = un;
                    nq2 = fma(un, un, nq2);
                });
            }
            nq2 = block_sum64(nq2, red);
            if (tid == 0) sc[2 + nbuf] = nq2;
            buf = nbuf;
            SYNC64();
        }
    }
#undef SYNC64
leave64:
    if (alive && g == 0 && tid == 0) {
        f.info[0] = status;
        f.info[1] = found;
        f.info[2] = (int)(total & 0x7fffffff);
        f.info[3] = (int)(total >> 31);
    }
}

}  // namespace gspca
