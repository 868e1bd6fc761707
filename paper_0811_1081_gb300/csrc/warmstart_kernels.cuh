// Standalone kernels of the learned warm start: features of a residual from a
// finished fit, the network over many rows, and one training step (forward,
// loss, backward, gradient reduction, Adam).  Definitions of the features,
// network and loss: warmstart.cuh.
#pragma once

#include "warmstart.cuh"

namespace gspca {

// ------------------------------------------------------------------ features

// Raw features of the columns of R_k = X - T(:, :k) P(:, :k)^T: one warp per
// column, feat[n*17] = c_n^2, feat[n*17 + 1 + j] = s_nj.  X column-major (ldx),
// T (M x >=k, ld M), P (N x >=k, ld N) column-major, G row-major (16 per row).
static __global__ void ws_raw_features_kernel(const float* __restrict__ X, long ldx, int M, int N,
                                              const float* __restrict__ T, const float* __restrict__ P, int k,
                                              const float* __restrict__ G, float* __restrict__ feat) {
    const int lane = threadIdx.x & 31;
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (n >= N) return;
    float c2 = 0.f, s[kWsSketch];
#pragma unroll
    for (int j = 0; j < kWsSketch; ++j) s[j] = 0.f;
    for (int r = lane; r < M; r += 32) {
        float x = X[(size_t)n * ldx + r];
        for (int j = 0; j < k; ++j) x = fmaf(-T[(size_t)j * M + r], P[(size_t)j * N + n], x);
        c2 = fmaf(x, x, c2);
        const float4* g4 = reinterpret_cast<const float4*>(G + (size_t)r * kWsSketch);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 g = __ldg(g4 + q);
            s[4 * q + 0] = fmaf(g.x, x, s[4 * q + 0]);
            s[4 * q + 1] = fmaf(g.y, x, s[4 * q + 1]);
            s[4 * q + 2] = fmaf(g.z, x, s[4 * q + 2]);
            s[4 * q + 3] = fmaf(g.w, x, s[4 * q + 3]);
        }
    }
    c2 = warp_sum(c2);
#pragma unroll
    for (int j = 0; j < kWsSketch; ++j) s[j] = warp_sum(s[j]);
    if (lane == 0) {
        feat[(size_t)n * kWsIn] = c2;
#pragma unroll
        for (int j = 0; j < kWsSketch; ++j) feat[(size_t)n * kWsIn + 1 + j] = s[j];
    }
}

// One block: rho from the raw c_n^2 (fixed-order sum), then every feature
// row scaled by 1/rho (c_n^2 replaced by c_n / rho).
static __global__ void ws_normalize_kernel(float* __restrict__ feat, int N) {
    __shared__ double part[32];
    __shared__ float s_inv;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double acc = 0.0;
    for (int n = t; n < N; n += blockDim.x) acc += (double)feat[(size_t)n * kWsIn];
    acc = warp_sum(acc);
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (t == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
        const double rho = sqrt(tot / N);
        s_inv = rho > 0.0 ? (float)(1.0 / rho) : 0.f;
    }
    __syncthreads();
    const float inv = s_inv;
    for (int n = t; n < N; n += blockDim.x) {
        float* f = feat + (size_t)n * kWsIn;
        f[0] = sqrtf(fmaxf(f[0], 0.f)) * inv;
        for (int j = 1; j < kWsIn; ++j) f[j] *= inv;
    }
}

// w[n] = network(feat[n]) for n < count (one warp per row).
static __global__ void ws_forward_kernel(const float* __restrict__ net, const float* __restrict__ feat, long count,
                                         float* __restrict__ w) {
    const int lane = threadIdx.x & 31;
    const long n = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (n >= count) return;
    float x[kWsIn];
#pragma unroll
    for (int f = 0; f < kWsIn; ++f) x[f] = feat[(size_t)n * kWsIn + f];
    const float out = ws_forward_warp(net, x, lane);
    if (lane == 0) w[n] = out;
}

// ------------------------------------------------------------------ training

// Scratch layout of one training step over ncols feature rows: activations and
// deltas unit-major ([64][ncols], so consecutive columns are consecutive words).
struct WsTrainScratch {
    float *Z1, *Z2, *D1, *D2, *w, *g;
    float* part;       // [nblk][kWsParams] per-block gradient sums
    float* inst;       // [ninst] per-instance losses
    int nblk;
};

// Forward with stored pre-activations: one thread per column.
static __global__ void ws_train_fwd_kernel(const float* __restrict__ net, const float* __restrict__ feat, long ncols,
                                           WsTrainScratch s) {
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= ncols) return;
    float x[kWsIn], h1[kWsH];
#pragma unroll
    for (int f = 0; f < kWsIn; ++f) x[f] = feat[(size_t)n * kWsIn + f];
#pragma unroll
    for (int i = 0; i < kWsH; ++i) {
        float a = __ldg(net + kWsB1 + i);
#pragma unroll
        for (int f = 0; f < kWsIn; ++f) a = fmaf(__ldg(net + kWsW1 + i * kWsIn + f), x[f], a);
        s.Z1[(size_t)i * ncols + n] = a;
        h1[i] = ws_gelu(a);
    }
    float out = __ldg(net + kWsB3);
    for (int i = 0; i < kWsH; ++i) {
        float a = __ldg(net + kWsB2 + i);
#pragma unroll
        for (int j = 0; j < kWsH; ++j) a = fmaf(__ldg(net + kWsW2 + i * kWsH + j), h1[j], a);
        s.Z2[(size_t)i * ncols + n] = a;
        out = fmaf(__ldg(net + kWsW3 + i), ws_gelu(a), out);
    }
    s.w[n] = out;
}

// One block per instance: a = w.p*, b = w.w (fixed-order block sums), the loss
// and dL/dw for its columns (already divided by ninst).
static __global__ void ws_loss_kernel(const float* __restrict__ target, const int* __restrict__ offsets, int ninst,
                                      WsTrainScratch s) {
    __shared__ double sa[32], sb[32];
    const int i = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const int c0 = offsets[i], c1 = offsets[i + 1];
    double a = 0.0, b = 0.0;
    for (int c = c0 + t; c < c1; c += blockDim.x) {
        const double w = s.w[c];
        a += w * (double)target[c];
        b += w * w;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (t == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < nw; ++w) {
            A += sa[w];
            B += sb[w];
        }
        sa[0] = A;
        sb[0] = B;
        s.inst[i] = B > 0.0 ? (float)(1.0 - A * A / B) : 1.f;
    }
    __syncthreads();
    const double A = sa[0], B = sb[0];
    for (int c = c0 + t; c < c1; c += blockDim.x)
        s.g[c] = B > 0.0 ? (float)((-2.0 * A * (double)target[c] / B + 2.0 * A * A * (double)s.w[c] / (B * B)) / ninst)
                         : 0.f;
}

// Deltas: D2 = g W3 * gelu'(Z2), D1 = (W2^T D2) * gelu'(Z1); one thread per column.
static __global__ void ws_train_bwd_kernel(const float* __restrict__ net, long ncols, WsTrainScratch s) {
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= ncols) return;
    const float g = s.g[n];
    float d2[kWsH];
#pragma unroll
    for (int i = 0; i < kWsH; ++i) {
        d2[i] = g * __ldg(net + kWsW3 + i) * ws_gelu_d(s.Z2[(size_t)i * ncols + n]);
        s.D2[(size_t)i * ncols + n] = d2[i];
    }
    for (int j = 0; j < kWsH; ++j) {
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < kWsH; ++i) a = fmaf(__ldg(net + kWsW2 + i * kWsH + j), d2[i], a);
        s.D1[(size_t)j * ncols + n] = a * ws_gelu_d(s.Z1[(size_t)j * ncols + n]);
    }
}

// Per-block parameter gradients over a range of columns: 256 threads, tiles of
// 32 columns staged in shared memory.  Every output entry is owned by one
// thread, which sums its tile contributions in column order.
constexpr int kWsGradThreads = 256;
constexpr int kWsGradTile = 32;

static __global__ void __launch_bounds__(kWsGradThreads) ws_wgrad_kernel(const float* __restrict__ feat, long ncols,
                                                                          long cols_per_blk, WsTrainScratch s) {
    __shared__ float sD1[kWsH][kWsGradTile + 1], sD2[kWsH][kWsGradTile + 1];
    __shared__ float sH1[kWsH][kWsGradTile + 1], sH2[kWsH][kWsGradTile + 1];
    __shared__ float sX[kWsIn][kWsGradTile + 1], sG[kWsGradTile];
    const int t = threadIdx.x;
    const long c_begin = (long)blockIdx.x * cols_per_blk;
    const long c_end = c_begin + cols_per_blk < ncols ? c_begin + cols_per_blk : ncols;
    // owned outputs: W2 entries t + 256 q (q < 16), W1 entries t + 256 q (q < 5, < 1088), and for
    // t < 64: b1[t], b2[t], W3[t]; t == 64: b3
    float aW2[16], aW1[5], ab1 = 0.f, ab2 = 0.f, aW3 = 0.f, ab3 = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) aW2[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 5; ++q) aW1[q] = 0.f;
    for (long cb = c_begin; cb < c_end; cb += kWsGradTile) {
        const int nc = (int)(c_end - cb < kWsGradTile ? c_end - cb : kWsGradTile);
        for (int e = t; e < kWsH * kWsGradTile; e += kWsGradThreads) {
            const int i = e / kWsGradTile, c = e % kWsGradTile;
            const bool ok = c < nc;
            const size_t idx = (size_t)i * ncols + cb + c;
            sD1[i][c] = ok ? s.D1[idx] : 0.f;
            sD2[i][c] = ok ? s.D2[idx] : 0.f;
            sH1[i][c] = ok ? ws_gelu(s.Z1[idx]) : 0.f;
            sH2[i][c] = ok ? ws_gelu(s.Z2[idx]) : 0.f;
        }
        for (int e = t; e < kWsIn * kWsGradTile; e += kWsGradThreads) {
            const int f = e / kWsGradTile, c = e % kWsGradTile;
            sX[f][c] = c < nc ? feat[(size_t)(cb + c) * kWsIn + f] : 0.f;
        }
        if (t < kWsGradTile) sG[t] = t < nc ? s.g[cb + t] : 0.f;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = t + kWsGradThreads * q, i = e >> 6, j = e & 63;  // dW2[i][j] = sum D2_i H1_j
            float a = aW2[q];
            for (int c = 0; c < kWsGradTile; ++c) a = fmaf(sD2[i][c], sH1[j][c], a);
            aW2[q] = a;
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int e = t + kWsGradThreads * q;
            if (e < kWsH * kWsIn) {
                const int j = e / kWsIn, f = e % kWsIn;  // dW1[j][f] = sum D1_j x_f
                float a = aW1[q];
                for (int c = 0; c < kWsGradTile; ++c) a = fmaf(sD1[j][c], sX[f][c], a);
                aW1[q] = a;
            }
        }
        if (t < kWsH) {
            for (int c = 0; c < kWsGradTile; ++c) {
                ab1 += sD1[t][c];
                ab2 += sD2[t][c];
                aW3 = fmaf(sG[c], sH2[t][c], aW3);
            }
        } else if (t == kWsH) {
            for (int c = 0; c < kWsGradTile; ++c) ab3 += sG[c];
        }
        __syncthreads();
    }
    float* out = s.part + (size_t)blockIdx.x * kWsParams;
#pragma unroll
    for (int q = 0; q < 16; ++q) out[kWsW2 + t + kWsGradThreads * q] = aW2[q];
#pragma unroll
    for (int q = 0; q < 5; ++q)
        if (t + kWsGradThreads * q < kWsH * kWsIn) out[kWsW1 + t + kWsGradThreads * q] = aW1[q];
    if (t < kWsH) {
        out[kWsB1 + t] = ab1;
        out[kWsB2 + t] = ab2;
        out[kWsW3 + t] = aW3;
    } else if (t == kWsH) {
        out[kWsB3] = ab3;
    }
}

// Sum of the block gradients (fixed order), optional copy out, Adam step
// (t >= 1, bias-corrected), and the minibatch loss (thread 0 of block 0).
static __global__ void ws_adam_kernel(float* __restrict__ net, float* __restrict__ m, float* __restrict__ v,
                                      WsTrainScratch s, int ninst, int step, float lr, float b1, float b2, float eps,
                                      float* __restrict__ grad_out, float* __restrict__ loss_out, int update) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss_out) {
        double L = 0.0;
        for (int i = 0; i < ninst; ++i) L += (double)s.inst[i];
        *loss_out = (float)(L / ninst);
    }
    if (p >= kWsParams) return;
    float g = 0.f;
    for (int b = 0; b < s.nblk; ++b) g += s.part[(size_t)b * kWsParams + p];
    if (grad_out) grad_out[p] = g;
    if (!update) return;
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    net[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

}  // namespace gspca
