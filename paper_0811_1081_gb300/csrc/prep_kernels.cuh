// Kernels around the persistent fit: optional centring (Sec. 2.1, Eq. 1),
// packing X into the 4-row panel layout of R, and writing the caller's
// column-major outputs (T = V Lambda or T = t, P = U, lambda, iters, R).
#pragma once

#include "device_common.cuh"

namespace gspca {

constexpr int kPackThreads = 256;

__device__ __forceinline__ float load_x(const float* X, int layout, long ldx, int r, int c) {
    return layout == 0 ? X[(size_t)c * ldx + r] : X[(size_t)r * ldx + c];
}

// mean over rows of every column (warp per column), FP64 sums.
static __global__ void colmean_kernel(const float* X, int layout, long ldx, int M, int N, double* mean) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= N) return;
    double s = 0.0;
    for (int r = lane; r < M; r += 32) s += (double)load_x(X, layout, ldx, r, c);
    s = warp_sum(s);
    if (lane == 0) mean[c] = s / (double)M;
}

// Eq. 1 as printed: the average column, i.e. the mean over columns of every row.
static __global__ void rowmean_kernel(const float* X, int layout, long ldx, int M, int N, double* mean) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= M) return;
    double s = 0.0;
    for (int c = lane; c < N; c += 32) s += (double)load_x(X, layout, ldx, r, c);
    s = warp_sum(s);
    if (lane == 0) mean[r] = s / (double)N;
}

// Pack X (M x N, either layout) into R (4-row panels of ldp cells, padded rows
// zero, Cell<E> storage), with optional subtraction of column means (center 1)
// or row means (center 2).  Each block writes the FP64 sum of squares of its
// tile (of the stored values) to xpart.  Block
// (0,0) also clears the fit kernel's barrier words (one every 32), the four
// abort words (the flag and the testing hook's stall word) and the info words:
// everything the fit needs to start at zero.
// Tile: 32 columns x 32 panels (128 rows); 256 threads.
template <class E>
__global__ void __launch_bounds__(kPackThreads) pack_kernel(const float* __restrict__ X, int layout, long ldx,
                                                            int M, int N, int np, int ldp, int center,
                                                            const double* __restrict__ cmean,
                                                            const double* __restrict__ rmean, void* R,
                                                            double* xpart, unsigned* flags, int nflags, int* abort,
                                                            int* info, int ninfo) {
    __shared__ float tile[32][129];
    __shared__ double wsum[kPackThreads / 32];
    const int t = threadIdx.x;
    const int c0 = blockIdx.x * 32, p0 = blockIdx.y * 32, rbase = p0 * 4;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        for (int i = t; i < nflags; i += kPackThreads) flags[(size_t)i * 32] = 0u;
        if (t < 4) abort[t] = 0;  // the abort flag and the spare words after it
        if (t < ninfo) info[t] = 0;
    }
    float sq = 0.f;
    if (layout == 0) {
        // column-major: coalesced reads down each column
        const int tx = t & 127, ty = t >> 7;
        for (int cc = ty; cc < 32; cc += 2) {
            const int c = c0 + cc, r = rbase + tx;
            float v = 0.f;
            if (c < N && r < M) {
                v = X[(size_t)c * ldx + r];
                if (center == 1) v = (float)((double)v - cmean[c]);
                else if (center == 2) v = (float)((double)v - rmean[r]);
            }
            tile[cc][tx] = v;
        }
    } else {
        const int cc = t & 31;
        for (int rr = t >> 5; rr < 128; rr += kPackThreads / 32) {
            const int c = c0 + cc, r = rbase + rr;
            float v = 0.f;
            if (c < N && r < M) {
                v = X[(size_t)r * ldx + c];
                if (center == 1) v = (float)((double)v - cmean[c]);
                else if (center == 2) v = (float)((double)v - rmean[r]);
            }
            tile[cc][rr] = v;
        }
    }
    __syncthreads();
    {
        const int cc = t & 31;
        for (int pp = t >> 5; pp < 32; pp += kPackThreads / 32) {
            const int p = p0 + pp, c = c0 + cc;
            if (p < np && c < N) {
                float4 v = Cell<E>::quant(make_float4(tile[cc][pp * 4 + 0], tile[cc][pp * 4 + 1],
                                                      tile[cc][pp * 4 + 2], tile[cc][pp * 4 + 3]));
                sq = fmaf(v.x, v.x, sq);
                sq = fmaf(v.y, v.y, sq);
                sq = fmaf(v.z, v.z, sq);
                sq = fmaf(v.w, v.w, sq);
                Cell<E>::stg_plain(R, (size_t)p * ldp + c, v);
            }
        }
    }
    double d = warp_sum((double)sq);
    if ((t & 31) == 0) wsum[t >> 5] = d;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kPackThreads / 32; ++w) s += wsum[w];
        xpart[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// T (M x K, ld M), P (N x K, ld N), lambda, iters from the row-major
// workspace factors.  Components >= found are zero.  T = V lambda_k (GS) or the
// unnormalised scores t_k that the NIPALS workspace V holds; with svd set, the
// unit score directions instead (the SVD form of Eq. 5): V (GS), t_k / lambda_k
// (NIPALS).
static __global__ void epilogue_kernel(const float* __restrict__ V, int ldv, const float* __restrict__ U, int ldu,
                                const double* __restrict__ lam_ws, const int* __restrict__ iters_ws,
                                const int* __restrict__ info, int M, int N, int K, int gs, int svd, float* T,
                                float* P, double* lambda, int* iters) {
    __shared__ float tile[32][33];
    const int found = info[1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: 32 x 8
    const int k0 = blockIdx.y * 32;
    const int rows_T = M;
    // blocks with blockIdx.x < ceil(M/32) do T, the rest do P
    const int bT = (rows_T + 31) / 32;
    const bool doT = blockIdx.x < bT;
    const int r0 = (doT ? blockIdx.x : blockIdx.x - bT) * 32;
    const int R = doT ? M : N;
    const float* S = doT ? V : U;
    const int ld = doT ? ldv : ldu;
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, k = k0 + tx;
        float v = 0.f;
        if (r < R && k < K && k < found) {
            v = S[(size_t)r * ld + k];
            if (doT && gs && !svd) v = (float)((double)v * lam_ws[k]);        // T = V Lambda
            else if (doT && !gs && svd) v = (float)((double)v / lam_ws[k]);  // t_k / lambda_k
        }
        tile[i][tx] = v;
    }
    __syncthreads();
    float* D = doT ? T : P;
    for (int i = ty; i < 32; i += 8) {
        const int k = k0 + i, r = r0 + tx;
        if (k < K && r < R) D[(size_t)k * R + r] = tile[tx][i];
    }
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            lambda[k] = k < found ? lam_ws[k] : 0.0;
            if (iters) iters[k] = k < found ? iters_ws[k] : 0;
        }
    }
}

// R_out (M x N, ld M) from the panels; when every component was found the
// deflation of the last one, R <- R - mult * V(K-1) U(K-1)^T (Eq. 3), is
// applied here (inside the fit it happens in the next component's first pass)
// and rounded as the storage of R rounds it.
template <class E>
__global__ void __launch_bounds__(kPackThreads) unpack_kernel(const void* __restrict__ R, int M, int N, int np, int ldp,
                                                              const float* __restrict__ V, int ldv,
                                                              const float* __restrict__ U, int ldu,
                                                              const double* __restrict__ lam_ws,
                                                              const int* __restrict__ info, int K, int gs,
                                                              float* Rout) {
    __shared__ float tile[32][129];
    const int t = threadIdx.x;
    const int c0 = blockIdx.x * 32, p0 = blockIdx.y * 32, rbase = p0 * 4;
    const bool defl = info[1] == K;
    const int kl = K - 1;
    const float lamf = gs ? (float)lam_ws[kl] : 1.f;
    {
        const int cc = t & 31;
        const int c = c0 + cc;
        const float uk = (defl && c < N) ? U[(size_t)c * ldu + kl] : 0.f;
        for (int pp = t >> 5; pp < 32; pp += kPackThreads / 32) {
            const int p = p0 + pp;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (p < np && c < N) {
                v = Cell<E>::ldg_plain(R, (size_t)p * ldp + c);
                if (defl) {
                    float cf[4];
                    for (int q = 0; q < 4; ++q) {
                        const int row = 4 * p + q;
                        cf[q] = row < M ? lamf * V[(size_t)row * ldv + kl] : 0.f;
                    }
                    v.x = fmaf(-cf[0], uk, v.x);
                    v.y = fmaf(-cf[1], uk, v.y);
                    v.z = fmaf(-cf[2], uk, v.z);
                    v.w = fmaf(-cf[3], uk, v.w);
                    v = Cell<E>::quant(v);
                }
            }
            tile[cc][pp * 4 + 0] = v.x;
            tile[cc][pp * 4 + 1] = v.y;
            tile[cc][pp * 4 + 2] = v.z;
            tile[cc][pp * 4 + 3] = v.w;
        }
    }
    __syncthreads();
    const int tx = t & 127, ty = t >> 7;
    for (int cc = ty; cc < 32; cc += 2) {
        const int c = c0 + cc, r = rbase + tx;
        if (c < N && r < M) Rout[(size_t)c * M + r] = tile[cc][tx];
    }
}

}  // namespace gspca
