// Persistent single-problem fit kernel: NIPALS-PCA (Sec. 2.2) and GS-PCA
// (Sec. 2.3) with every iteration and every convergence decision on the device.
//
// Work split.  The grid is one cooperative launch of G CTAs.  CTA g owns
//   - a contiguous range of 4-row panels of R (rows [r0, r1)), and with them
//     the same rows of V (score directions), vraw and vcorr;
//   - a contiguous slice [n0, n1) of the N columns, and with it the same rows
//     of U (loadings), W = R^T V, upre.
// Only partial sums, the current loading `ut`, its FP32 copy `ucur` and a few
// norms cross CTAs, always through a bounded grid barrier.
//
// One pass over R per power iteration.  A pass takes the normalised loading
// u, forms v_raw = R u row panel by row panel (FP32 products, warp butterfly,
// cross-warp sum) and, while the panel is still in registers, accumulates
// s = R^T v_raw.  For GS-PCA the score correction v = (v_raw - V b)/lambda,
// b = V^T v_raw, commutes through R^T: R^T v = (s - W b)/lambda with W = R^T V
// kept up to date by a rank-1 update per component, so the paper's second
// matrix-vector product (u = R^T v) needs no second read of R.  The rank-1
// deflation of component k-1 (Eq. 3) is applied inside the first pass of
// component k, which also extracts the start column R(k).
//
// Precision: R and every O(M k), O(N k) product are FP32 with FP32 sums
// inside a CTA; sums across CTAs, the Gram-Schmidt coefficients' use against
// FP64 vectors, every norm, lambda and the convergence test are FP64.
#pragma once

#include "device_common.cuh"

namespace gspca {

constexpr int kBlock = 512;
constexpr int kMaxWarps = kBlock / 32;

enum : int { kInfoStatus = 0, kInfoFound = 1, kInfoItersLo = 2, kInfoItersHi = 3, kInfoWords = 8 };

struct FitArgs {
    int M, N, K, np;          // np = number of 4-row panels (Mp / 4)
    int algo;                 // 0 = NIPALS, 1 = GS
    int max_iter;
    double tol;
    double eps_thresh;        // degenerate threshold factor: lambda <= eps_thresh * ||X||_F
    const double* xpart;      // partial sums of squares of the packed X
    int nxpart;
    float* R;                 // [np][N][4] panel layout (row 4p+q, column c) at ((p*N + c)*4 + q)
    float* V;                 // Mp x ldv row-major: V[r*ldv + k]
    int ldv;
    float* U;                 // N x ldu row-major
    int ldu;
    float* W;                 // N x ldw row-major (R^T V)
    int ldw;
    float* vraw;              // Mp
    float* vcorr;             // Mp
    float* ut;                // N, unnormalised current loading
    double* upre;             // N
    float* ucur;              // N, FP32 normalised loading used by the last pass
    float* part;              // G x L vector partials
    int L;
    double* spart;            // G x 4 scalar partials
    double* red;              // L reduced vectors
    double* reds;             // 4 reduced scalars
    double* normpart;         // G partial squared norms of ut
    double* lam;              // K
    int* iters;               // K
    int* info;                // kInfoWords
    unsigned* bar;            // [count, generation]
    int* abort;
    const int* iters_lock;    // device, K entries, nullable
    unsigned long long timeout_ns;
};

struct __align__(16) SmemFit {
    float wsum[kMaxWarps][32];
    float vrow[2][32];
    float tmpf[kMaxWarps][128];
    double dtmp[kMaxWarps * 4];
    double bcast[4];
    int flag;
    int sel;
};

enum : int { kPassDot = 0, kPassCol = 1, kPassSq = 2 };

template <int CPT>
struct PassShape {
    static constexpr int PPR = (CPT >= 8) ? 1 : 8 / CPT;  // panels per round
    static constexpr int RPR = 4 * PPR;                   // rows per round
};

// One streaming pass over the CTA's panels [p0, p1).
//   kPassDot: rows = R u (u in uc[]), written to vraw; sacc = R^T rows; sc = sum rows^2.
//   kPassCol: rows = R(:, kcol) after the optional deflation
//             R <- R - (lamf * V(:, kprev)) ucur^T (uc[] holds ucur); sacc = R^T rows;
//             sc = ||R(:, kcol)||^2 over the CTA's rows.
//   kPassSq : sacc = column sums of squares (start-column fallback).
template <int CPT, int MODE>
__device__ __forceinline__ void row_pass(const FitArgs& f, SmemFit& sm, int p0, int p1,
                                         const float (&uc)[CPT], int kcol, bool deflate, float lamf,
                                         int kprev, float (&sacc)[CPT], double& sc) {
    constexpr int PPR = PassShape<CPT>::PPR;
    constexpr int RPR = PassShape<CPT>::RPR;
    constexpr int SH = 5 - Log2<RPR>::value;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int T = blockDim.x, N = f.N;
    int owner = -1;
    if (MODE == kPassCol && (kcol % T) == tid) owner = kcol / T;
#pragma unroll
    for (int i = 0; i < CPT; ++i) sacc[i] = 0.f;
    double my = 0.0;
    int buf = 0;
    for (int pb = p0; pb < p1; pb += PPR, buf ^= 1) {
        float4 d[PPR][CPT];
#pragma unroll
        for (int pp = 0; pp < PPR; ++pp) {
            const int p = pb + pp;
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T;
                d[pp][i] = (p < p1 && c < N) ? ld_stream4(f.R + ((size_t)p * N + c) * 4)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (MODE == kPassCol && deflate) {
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                const int p = pb + pp;
                float cf[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int row = 4 * p + q;
                    cf[q] = (p < p1 && row < f.M) ? lamf * f.V[(size_t)row * f.ldv + kprev] : 0.f;
                }
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int c = tid + i * T;
                    float4 v = d[pp][i];
                    v.x = fmaf(-cf[0], uc[i], v.x);
                    v.y = fmaf(-cf[1], uc[i], v.y);
                    v.z = fmaf(-cf[2], uc[i], v.z);
                    v.w = fmaf(-cf[3], uc[i], v.w);
                    d[pp][i] = v;
                    if (p < p1 && c < N) st_stream4(f.R + ((size_t)p * N + c) * 4, v);
                }
            }
        }
        float rowv[RPR];
        if (MODE == kPassDot) {
            float acc[RPR];
#pragma unroll
            for (int r = 0; r < RPR; ++r) acc[r] = 0.f;
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
#pragma unroll
                for (int pp = 0; pp < PPR; ++pp) {
                    acc[pp * 4 + 0] = fmaf(d[pp][i].x, uc[i], acc[pp * 4 + 0]);
                    acc[pp * 4 + 1] = fmaf(d[pp][i].y, uc[i], acc[pp * 4 + 1]);
                    acc[pp * 4 + 2] = fmaf(d[pp][i].z, uc[i], acc[pp * 4 + 2]);
                    acc[pp * 4 + 3] = fmaf(d[pp][i].w, uc[i], acc[pp * 4 + 3]);
                }
            }
            const float r = warp_multi_reduce<RPR>(acc, lane);
            if ((lane & ((1 << SH) - 1)) == 0) sm.wsum[warp][lane >> SH] = r;
            __syncthreads();
            if (tid < RPR) {
                float s = 0.f;
                for (int w = 0; w < nw; ++w) s += sm.wsum[w][tid];
                if (pb + (tid >> 2) < p1) {
                    f.vraw[(size_t)pb * 4 + tid] = s;
                    my += (double)s * (double)s;
                }
                sm.vrow[buf][tid] = s;
            }
            __syncthreads();
#pragma unroll
            for (int r2 = 0; r2 < RPR; ++r2) rowv[r2] = sm.vrow[buf][r2];
        } else if (MODE == kPassCol) {
            if (owner >= 0) {
#pragma unroll
                for (int pp = 0; pp < PPR; ++pp) {
                    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int i = 0; i < CPT; ++i)
                        if (i == owner) x = d[pp][i];
                    sm.vrow[buf][pp * 4 + 0] = x.x;
                    sm.vrow[buf][pp * 4 + 1] = x.y;
                    sm.vrow[buf][pp * 4 + 2] = x.z;
                    sm.vrow[buf][pp * 4 + 3] = x.w;
                    my += (double)x.x * x.x + (double)x.y * x.y + (double)x.z * x.z + (double)x.w * x.w;
                }
            }
            __syncthreads();
#pragma unroll
            for (int r2 = 0; r2 < RPR; ++r2) rowv[r2] = sm.vrow[buf][r2];
        }
        if (MODE == kPassSq) {
#pragma unroll
            for (int i = 0; i < CPT; ++i)
#pragma unroll
                for (int pp = 0; pp < PPR; ++pp) {
                    const float4 v = d[pp][i];
                    sacc[i] = fmaf(v.x, v.x, sacc[i]);
                    sacc[i] = fmaf(v.y, v.y, sacc[i]);
                    sacc[i] = fmaf(v.z, v.z, sacc[i]);
                    sacc[i] = fmaf(v.w, v.w, sacc[i]);
                }
        } else {
#pragma unroll
            for (int i = 0; i < CPT; ++i)
#pragma unroll
                for (int pp = 0; pp < PPR; ++pp) {
                    const float4 v = d[pp][i];
                    sacc[i] = fmaf(v.x, rowv[pp * 4 + 0], sacc[i]);
                    sacc[i] = fmaf(v.y, rowv[pp * 4 + 1], sacc[i]);
                    sacc[i] = fmaf(v.z, rowv[pp * 4 + 2], sacc[i]);
                    sacc[i] = fmaf(v.w, rowv[pp * 4 + 3], sacc[i]);
                }
        }
    }
    // CTA total of `my` (nonzero only in warp 0 for kPassDot, in the owner for kPassCol).
    if (MODE == kPassDot) {
        if (warp == 0) {
            const double t = warp_sum(my);
            if (lane == 0) sm.bcast[0] = t;
        }
    } else if (MODE == kPassCol) {
        if (owner >= 0) sm.bcast[0] = my;
    } else {
        if (tid == 0) sm.bcast[0] = 0.0;
    }
    __syncthreads();
    sc = sm.bcast[0];
    __syncthreads();
}

// dst[j] = sum_{r in [r0, r1)} A[r*lda + j] * y(r) for j < kk, FP32 within the CTA.
template <class Y>
__device__ __forceinline__ void rows_times_matrix(const float* A, int lda, int r0, int r1, int kk, Y y,
                                                  float* dst, SmemFit& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int j0 = 0; j0 < kk; j0 += 128) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int r = r0 + warp; r < r1; r += nw) {
            const float yr = y(r);
            const float* a = A + (size_t)r * lda + j0 + lane;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + lane + 32 * q < kk) acc[q] = fmaf(ldcg(a + 32 * q), yr, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) sm.tmpf[warp][lane + 32 * q] = acc[q];
        __syncthreads();
        for (int t = tid; t < 128 && j0 + t < kk; t += blockDim.x) {
            float s = 0.f;
            for (int w = 0; w < nw; ++w) s += sm.tmpf[w][t];
            dst[j0 + t] = s;
        }
        __syncthreads();
    }
}

// For r in [r0, r1): fn(r, sum_j A[r*lda + j] * x[j]) with x (kk floats) in shared memory.
template <class Fn>
__device__ __forceinline__ void matrix_times_vector(const float* A, int lda, int r0, int r1, int kk,
                                                    const float* x, Fn fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = r0 + warp; r < r1; r += nw) {
        float s = 0.f;
        const float* a = A + (size_t)r * lda;
        for (int j = lane; j < kk; j += 32) s = fmaf(ldcg(a + j), x[j], s);
        s = warp_sum(s);
        fn(r, s, lane);
    }
}

// CTA-wide FP64 sum of per-thread values in a fixed order (deterministic).
__device__ __forceinline__ double block_sum(double v, SmemFit& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sm.dtmp[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sm.dtmp[w];
        sm.bcast[1] = s;
    }
    __syncthreads();
    const double r = sm.bcast[1];
    __syncthreads();
    return r;
}

// Reduce the vector partials part[0..G)[0..Lc) into red[0..Lc): columns are
// dealt out in groups of 4 to the warps of all CTAs in a fixed pattern; a
// lane sums every 8th CTA row in FP32 and the 8 lanes of a column combine
// in FP64 through a fixed butterfly.  If outv != nullptr, columns c < sq_n
// are also stored to outv (FP32) and their squares summed into normpart[g].
// CTA G-1 also reduces the nsc scalar partials spart[.][0..nsc) in FP64.
__device__ __forceinline__ void slice_reduce(const FitArgs& f, int Lc, float* outv, int sq_n, int nsc,
                                             SmemFit& sm) {
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int ng = (Lc + 3) >> 2;
    const int g0 = (int)(((long long)g * ng) / G), g1 = (int)(((long long)(g + 1) * ng) / G);
    double sq = 0.0;
    for (int grp = g0 + warp; grp < g1; grp += nw) {
        const int c = grp * 4 + (lane & 3);
        float s = 0.f;
        if (c < Lc)
            for (int r = lane >> 2; r < G; r += 8) s += ldcg(f.part + (size_t)r * f.L + c);
        double d = (double)s;
        d += __shfl_xor_sync(kFull, d, 4);
        d += __shfl_xor_sync(kFull, d, 8);
        d += __shfl_xor_sync(kFull, d, 16);
        if (lane < 4 && c < Lc) {
            f.red[c] = d;
            if (outv != nullptr && c < sq_n) {
                outv[c] = (float)d;
                sq += d * d;
            }
        }
    }
    if (outv != nullptr) {
        if (lane < 4) sm.dtmp[warp * 4 + lane] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int i = 0; i < nw * 4; ++i) t += sm.dtmp[i];
            f.normpart[g] = t;
        }
        __syncthreads();
    }
    if (nsc > 0 && g == G - 1 && warp == nw - 1) {
        for (int s = 0; s < nsc; ++s) {
            double t = 0.0;
            for (int r = lane; r < G; r += 32) t += ldcg(f.spart + (size_t)r * 4 + s);
            t = warp_sum(t);
            if (lane == 0) f.reds[s] = t;
        }
    }
}

// Sum of the G norm partials, same order in every CTA.
__device__ __forceinline__ double sum_normparts(const FitArgs& f, SmemFit& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        double t = 0.0;
        for (int r = lane; r < (int)gridDim.x; r += 32) t += ldcg(f.normpart + r);
        t = warp_sum(t);
        if (lane == 0) sm.bcast[2] = t;
    }
    __syncthreads();
    const double r = sm.bcast[2];
    __syncthreads();
    return r;
}

template <int CPT>
__global__ void __launch_bounds__(kBlock, 1) fit_kernel(const FitArgs f) {
    __shared__ SmemFit sm;
    extern __shared__ float dyn_smem[];
    float* bs = dyn_smem;           // b (or a) as FP32, up to max(ldv, ldu) entries
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int p0 = (int)(((long long)g * f.np) / G), p1 = (int)(((long long)(g + 1) * f.np) / G);
    const int r0 = min(p0 * 4, f.M), r1 = min(p1 * 4, f.M);
    const int n0 = (int)(((long long)g * f.N) / G), n1 = (int)(((long long)(g + 1) * f.N) / G);
    const GridBarrier bar{f.bar, f.bar + 1, f.abort, f.timeout_ns};
    const bool gs = (f.algo == 1);
    const int N = f.N, K = f.K;
    float* part_g = f.part + (size_t)g * f.L;

    // ||X||_F^2 from the pack kernel's partials (fixed order, every CTA).
    if (warp == 0) {
        double t = 0.0;
        for (int i = lane; i < f.nxpart; i += 32) t += f.xpart[i];
        t = warp_sum(t);
        if (lane == 0) sm.bcast[3] = t;
    }
    __syncthreads();
    const double thresh = f.eps_thresh * sqrt(sm.bcast[3]);

    int status = kStOK, found = K;
    long long total = 0;
    double lam_prev = 0.0;
    float uc[CPT], sacc[CPT];
    double sc = 0.0;

    for (int k = 0; k < K && found == K; ++k) {
        // ---------------- start pass: deflate component k-1, take column k
        __syncthreads();  // finalize of k-1 (V, U rows of this CTA) before they are read
        const bool defl = k > 0;
        const float lamf = gs ? (float)lam_prev : 1.f;
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int c = tid + i * T;
            uc[i] = (defl && c < N) ? ldcg(f.ucur + c) : 0.f;
        }
        row_pass<CPT, kPassCol>(f, sm, p0, p1, uc, k, defl, lamf, k - 1, sacc, sc);
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int c = tid + i * T;
            if (c < N) part_g[c] = sacc[i];
        }
        if (tid == 0) f.spart[(size_t)g * 4] = sc;
        if (gs && k > 0)  // Gram row G[k-1][j] = V(k-1)^T V(j), j <= k-1
            rows_times_matrix(f.V, f.ldv, r0, r1, k, [&](int r) { return f.V[(size_t)r * f.ldv + (k - 1)]; },
                              part_g + N, sm);
        if (!bar.sync(&sm.flag)) return;
        slice_reduce(f, N + (gs ? k : 0), gs ? nullptr : f.ut, gs ? 0 : N, 1, sm);
        if (!bar.sync(&sm.flag)) return;

        if (ldcg(f.reds) == 0.0) {
            // Zero start column: restart from the residual column of largest norm
            // (lowest index on ties); every column zero => rank exhausted.
            row_pass<CPT, kPassSq>(f, sm, p0, p1, uc, 0, false, 0.f, 0, sacc, sc);
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T;
                if (c < N) part_g[c] = sacc[i];
            }
            if (!bar.sync(&sm.flag)) return;
            slice_reduce(f, N, nullptr, 0, 0, sm);
            if (!bar.sync(&sm.flag)) return;
            if (warp == 0) {
                double best = 0.0;
                int bi = N;
                for (int c = lane; c < N; c += 32) {
                    const double v = ldcg(f.red + c);
                    if (v > best) { best = v; bi = c; }
                }
                for (int o = 16; o >= 1; o >>= 1) {
                    const double ob = __shfl_xor_sync(kFull, best, o);
                    const int oi = __shfl_xor_sync(kFull, bi, o);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (lane == 0) sm.sel = (best > 0.0) ? bi : -1;
            }
            __syncthreads();
            const int kcol = sm.sel;
            __syncthreads();
            if (kcol < 0) {
                found = k;
                status = kStDegenerate;
                break;
            }
            row_pass<CPT, kPassCol>(f, sm, p0, p1, uc, kcol, false, 0.f, 0, sacc, sc);
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T;
                if (c < N) part_g[c] = sacc[i];
            }
            if (!bar.sync(&sm.flag)) return;
            slice_reduce(f, N, gs ? nullptr : f.ut, gs ? 0 : N, 0, sm);
            if (!bar.sync(&sm.flag)) return;
        }

        if (gs) {
            // W <- R_k^T V: rank-1 update for the deflation of component k-1 plus
            // the new column R_k^T v_{k-1} = upre/lambda - lambda u_{k-1} (v^T v).
            if (k > 0) {
                const double lp = lam_prev;
                for (int e = tid; e < (n1 - n0) * k; e += T) {
                    const int n = n0 + e / k, jj = e % k;
                    const double un = (double)f.U[(size_t)n * f.ldu + (k - 1)];
                    const double gj = ldcg(f.red + N + jj);
                    float* w = f.W + (size_t)n * f.ldw + jj;
                    if (jj < k - 1)
                        *w = (float)((double)*w - lp * un * gj);
                    else
                        *w = (float)(f.upre[n] / lp - lp * un * gj);
                }
                __syncthreads();
            }
            for (int n = n0 + tid; n < n1; n += T) f.upre[n] = ldcg(f.red + n);
            __syncthreads();
            if (k > 0) {
                rows_times_matrix(f.U, f.ldu, n0, n1, k, [&](int n) { return (float)f.upre[n]; }, part_g, sm);
                if (!bar.sync(&sm.flag)) return;
                slice_reduce(f, k, nullptr, 0, 0, sm);
                if (!bar.sync(&sm.flag)) return;
                for (int j = tid; j < k; j += T) bs[j] = (float)ldcg(f.red + j);
                __syncthreads();
            }
            double nq = 0.0;
            if (k > 0) {
                matrix_times_vector(f.U, f.ldu, n0, n1, k, bs, [&](int n, float s, int ln) {
                    if (ln == 0) {
                        const double un = f.upre[n] - (double)s;
                        f.ut[n] = (float)un;
                        nq += un * un;
                    }
                });
            } else {
                for (int n = n0 + tid; n < n1; n += T) {
                    const double un = f.upre[n];
                    f.ut[n] = (float)un;
                    nq += un * un;
                }
            }
            nq = block_sum(nq, sm);
            if (tid == 0) f.normpart[g] = nq;
            if (!bar.sync(&sm.flag)) return;
        }

        // ---------------- power iterations
        double mu = 0.0, lam = 0.0;
        int j = 0;
        for (;;) {
            const double nrm2 = sum_normparts(f, sm);
            if (!(nrm2 > 0.0)) {
                found = k;
                status = kStDegenerate;
                break;
            }
            const float inv = (float)(1.0 / sqrt(nrm2));
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T;
                uc[i] = (c < N) ? ldcg(f.ut + c) * inv : 0.f;
                if (g == 0 && c < N) f.ucur[c] = uc[i];
            }
            row_pass<CPT, kPassDot>(f, sm, p0, p1, uc, 0, false, 0.f, 0, sacc, sc);
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T;
                if (c < N) part_g[c] = sacc[i];
            }
            if (tid == 0) f.spart[(size_t)g * 4] = sc;
            if (gs && k > 0)  // b = V_(k)^T v_raw over the CTA's rows
                rows_times_matrix(f.V, f.ldv, r0, r1, k, [&](int r) { return f.vraw[r]; }, part_g + N, sm);
            if (!bar.sync(&sm.flag)) return;
            slice_reduce(f, N + (gs ? k : 0), gs ? nullptr : f.ut, gs ? 0 : N, 1, sm);
            if (!bar.sync(&sm.flag)) return;
            ++j;
            ++total;
            if (!gs) {
                lam = sqrt(ldcg(f.reds));
            } else if (k == 0) {
                lam = sqrt(ldcg(f.reds));
                for (int r = r0 + tid; r < r1; r += T) f.vcorr[r] = f.vraw[r];
                for (int n = n0 + tid; n < n1; n += T) f.upre[n] = ldcg(f.red + n);
            } else {
                // v = v_raw - V b (rows), upre = s - W b (slice), a = U^T upre (partials)
                for (int jj = tid; jj < k; jj += T) bs[jj] = (float)ldcg(f.red + N + jj);
                __syncthreads();
                double l2 = 0.0;
                matrix_times_vector(f.V, f.ldv, r0, r1, k, bs, [&](int r, float s, int ln) {
                    if (ln == 0) {
                        const double vc = (double)f.vraw[r] - (double)s;
                        f.vcorr[r] = (float)vc;
                        l2 += vc * vc;
                    }
                });
                matrix_times_vector(f.W, f.ldw, n0, n1, k, bs, [&](int n, float s, int ln) {
                    if (ln == 0) f.upre[n] = ldcg(f.red + n) - (double)s;
                });
                __syncthreads();
                rows_times_matrix(f.U, f.ldu, n0, n1, k, [&](int n) { return (float)f.upre[n]; }, part_g, sm);
                l2 = block_sum(l2, sm);
                if (tid == 0) f.spart[(size_t)g * 4] = l2;
                if (!bar.sync(&sm.flag)) return;
                slice_reduce(f, k, nullptr, 0, 1, sm);
                if (!bar.sync(&sm.flag)) return;
                lam = sqrt(ldcg(f.reds));
            }
            if (!(lam > thresh)) {
                found = k;
                status = kStDegenerate;
                break;
            }
            bool stop;
            if (f.iters_lock != nullptr) {
                stop = j >= f.iters_lock[k];
            } else {
                stop = fabs(mu - lam) < f.tol * lam;
                if (!stop && j >= f.max_iter) {
                    stop = true;
                    if (status == kStOK) status = kStNotConverged;
                }
            }
            if (stop) {
                // Finalize component k: V(k), U(k), lambda_k, iters_k.
                if (gs) {
                    const double il = 1.0 / lam;
                    for (int r = r0 + tid; r < r1; r += T)
                        f.V[(size_t)r * f.ldv + k] = (float)((double)f.vcorr[r] * il);
                } else {
                    for (int r = r0 + tid; r < r1; r += T) f.V[(size_t)r * f.ldv + k] = f.vraw[r];
                }
                for (int n = n0 + tid; n < n1; n += T) f.U[(size_t)n * f.ldu + k] = ldcg(f.ucur + n);
                if (g == 0 && tid == 0) {
                    f.lam[k] = lam;
                    f.iters[k] = j;
                }
                lam_prev = lam;
                break;
            }
            mu = lam;
            if (gs) {
                double nq = 0.0;
                if (k > 0) {
                    for (int jj = tid; jj < k; jj += T) bs[jj] = (float)ldcg(f.red + jj);
                    __syncthreads();
                    matrix_times_vector(f.U, f.ldu, n0, n1, k, bs, [&](int n, float s, int ln) {
                        if (ln == 0) {
                            const double un = f.upre[n] - (double)s;
                            f.ut[n] = (float)un;
                            nq += un * un;
                        }
                    });
                } else {
                    for (int n = n0 + tid; n < n1; n += T) {
                        const double un = f.upre[n];
                        f.ut[n] = (float)un;
                        nq += un * un;
                    }
                }
                nq = block_sum(nq, sm);
                if (tid == 0) f.normpart[g] = nq;
                if (!bar.sync(&sm.flag)) return;
            }
        }
    }
    if (g == 0 && tid == 0) {
        f.info[kInfoStatus] = status;
        f.info[kInfoFound] = found;
        f.info[kInfoItersLo] = (int)(total & 0x7fffffff);
        f.info[kInfoItersHi] = (int)(total >> 31);
    }
}

}  // namespace gspca
