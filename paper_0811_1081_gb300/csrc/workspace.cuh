// Device workspace of one fit: the layout of the buffers the persistent loop
// works on, carved from one allocation (host code; shared by every entry point).
#pragma once

#include <cstddef>

#include "fit_kernel.cuh"

namespace gspca {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Dimensions the workspace is laid out for (maximum sizes for a handle, the
// exact problem for the no-allocation entry point).
struct WsDims {
    long Mp;   // rows rounded up to a multiple of 4
    int N, K;
    int G;     // CTAs the partial buffers hold
    bool warm = false;  // with the buffers of the learned warm start
};

// Leading dimension of the k-column factors: a power of two up to 128 (the
// float4 row-chunk products), a multiple of 4 beyond.
inline int ws_ld(int K) {
    if (K > 128) return (int)align_up((size_t)K, 4);
    int ld = 4;
    while (ld < K) ld *= 2;
    return ld;
}
// Pass partials: s' (N), b' and c' (K each), 4 spare.
inline int ws_LA(int N, int K) { return (int)align_up((size_t)N + 2 * (size_t)K + 4, 4); }
inline int ws_xcap(long Mp, int N) { return (int)(((N + 31) / 32) * ((Mp / 4 + 31) / 32)); }

struct Workspace {
    float *R, *V, *U, *W, *vraw, *vcorr, *ut, *upre, *partA, *partB;
    float *wsF, *wsP0, *pC, *wsPart, *wsInit;  // learned warm start (null unless WsDims::warm)
    float2* spart;
    double *red, *lam, *xpart, *cmean, *rmean;
    int *iters, *info, *abort, *lock;
    unsigned* flags;
    long long* facc;  // 2 x ld fixed-point accumulators (kernels for more than 128 components)
    int ld, LA, LB, G, xcap;
    size_t bytes;
};

// Lay the workspace out from `base` (nullptr: only compute the size).
inline Workspace carve(void* base, const WsDims& d) {
    Workspace w{};
    w.ld = ws_ld(d.K);
    w.LA = ws_LA(d.N, d.K);
    w.LB = 3 * w.ld;  // a' (GS step), or a, U^T u, W^T u and u.u_pre (component start)
    w.G = d.G;
    w.xcap = ws_xcap(d.Mp, d.N);
    char* b = static_cast<char*>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = align_up(off, 256);
        void* p = b ? b + off : nullptr;
        off += align_up(bytes > 0 ? bytes : 1, 256);
        return p;
    };
    w.R = (float*)take(sizeof(float) * (size_t)d.Mp * d.N);
    w.V = (float*)take(sizeof(float) * (size_t)d.Mp * w.ld);
    w.U = (float*)take(sizeof(float) * (size_t)d.N * w.ld);
    w.W = (float*)take(sizeof(float) * (size_t)d.N * w.ld);
    w.vraw = (float*)take(sizeof(float) * (size_t)d.Mp);
    w.vcorr = (float*)take(sizeof(float) * (size_t)d.Mp);
    w.ut = (float*)take(sizeof(float) * 2 * (size_t)d.N);
    w.upre = (float*)take(sizeof(float) * (size_t)d.N);
    w.partA = (float*)take(sizeof(float) * (size_t)d.G * w.LA);
    w.partB = (float*)take(sizeof(float) * (size_t)d.G * w.LB);
    w.spart = (float2*)take(sizeof(float2) * 4 * (size_t)d.G);
    w.red = (double*)take(sizeof(double) * (size_t)w.LA);
    w.lam = (double*)take(sizeof(double) * (size_t)d.K);
    w.xpart = (double*)take(sizeof(double) * (size_t)w.xcap);
    w.cmean = (double*)take(sizeof(double) * (size_t)d.N);
    w.rmean = (double*)take(sizeof(double) * (size_t)d.Mp);
    w.iters = (int*)take(sizeof(int) * (size_t)d.K);
    w.info = (int*)take(sizeof(int) * kInfoWords);
    w.abort = (int*)take(sizeof(int) * 4);
    w.lock = (int*)take(sizeof(int) * (size_t)d.K);
    w.flags = (unsigned*)take(sizeof(unsigned) * 32);
    w.facc = (long long*)take(sizeof(long long) * 2 * (size_t)w.ld);
    if (d.warm) {
        w.wsF = (float*)take(sizeof(float) * 17 * (size_t)d.N);
        w.wsP0 = (float*)take(sizeof(float) * (size_t)d.N);
        w.pC = (float*)take(sizeof(float) * (size_t)d.G * d.N);
        w.wsPart = (float*)take(sizeof(float) * 32 * (size_t)d.G);
        w.wsInit = (float*)take(sizeof(float) * 17 * (size_t)d.G * d.N);
    }
    w.bytes = off;
    return w;
}

}  // namespace gspca
