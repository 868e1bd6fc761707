// Learned warm start of GS-PCA (not in the paper): the Gaussian sketch of the
// residual's columns, the per-column network 17 -> 64 -> 64 -> 1 (erf GELU),
// and the kernels that train it (forward, loss, backward, Adam).
//
// Definitions shared with the fit kernel (fit_kernel.cuh):
//   features of column n of a residual R (M x N):
//     c_n = ||R(n)||, s_n = G^T R(n) (G: M x 16, row-major, given by the caller),
//     rho = sqrt(sum_n c_n^2 / N), x_n = [c_n, s_n] / rho (zero when rho = 0);
//   network parameters, one FP32 array of kWsParams values: W1 (64 x 17,
//   row-major), b1 (64), W2 (64 x 64, row-major), b2 (64), W3 (64), b3;
//   output w_n, start loading p0 = w / ||w||;
//   training loss of an instance (the columns of one residual, target loading
//   p*): L = 1 - (w . p*)^2 / (w . w), 1 with zero gradient when w = 0; the loss
//   of a minibatch is the mean over its instances.
#pragma once

#include "device_common.cuh"

namespace gspca {

constexpr int kWsSketch = 16;
constexpr int kWsIn = 17;
constexpr int kWsH = 64;
constexpr int kWsW1 = 0;
constexpr int kWsB1 = kWsW1 + kWsH * kWsIn;
constexpr int kWsW2 = kWsB1 + kWsH;
constexpr int kWsB2 = kWsW2 + kWsH * kWsH;
constexpr int kWsW3 = kWsB2 + kWsH;
constexpr int kWsB3 = kWsW3 + kWsH;
constexpr int kWsParams = kWsB3 + 1;  // 5377

__device__ __forceinline__ float ws_gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

// d/dz [z Phi(z)] = Phi(z) + z phi(z)
__device__ __forceinline__ float ws_gelu_d(float z) {
    const float Phi = 0.5f * (1.f + erff(z * 0.70710678118654752f));
    return Phi + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Network output for one column, computed by a whole warp: lane l owns hidden
// units l and l + 32.  x (17 values) must be identical in every lane.  The
// second layer forms, per lane, the 64 partial products of its two input
// units and reduces them across the warp with two 32-value butterflies.
// Result (w) in every lane.  `net` may point to global or shared memory
// (generic loads; the access pattern is bank-conflict free in shared memory).
__device__ __forceinline__ float ws_forward_warp(const float* __restrict__ net, const float (&x)[kWsIn], int lane) {
    float h1[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int i = lane + 32 * q;
        float a = net[kWsB1 + i];
#pragma unroll
        for (int f = 0; f < kWsIn; ++f) a = fmaf(net[kWsW1 + i * kWsIn + f], x[f], a);
        h1[q] = ws_gelu(a);
    }
    float out = 0.f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float part[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int i = 32 * half + t;  // output unit
            part[t] = fmaf(net[kWsW2 + i * kWsH + lane], h1[0], net[kWsW2 + i * kWsH + lane + 32] * h1[1]);
        }
        const float z = warp_multi_reduce<32>(part, lane) + net[kWsB2 + 32 * half + lane];  // unit 32 half + lane
        out = fmaf(net[kWsW3 + 32 * half + lane], ws_gelu(z), out);
    }
    return warp_sum(out) + net[kWsB3];
}

}  // namespace gspca
