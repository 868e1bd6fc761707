// Device workspace of the FP64 storage path (host code): the buffers the
// persistent FP64 loop works on, carved from one allocation owned by a
// GSPCA_F64 handle.
#pragma once

#include <cstddef>

namespace gspca {

constexpr int kPack64Blocks = 2048;  // pack kernel grid: one ||X||_F^2 partial per block

struct Workspace64 {
    double *R, *V, *U, *W, *vraw, *vcorr, *ut, *upre, *partS, *partA, *scal, *lam, *xpart, *cmean, *rmean;
    int *iters, *info, *abort, *lock;
    unsigned* flags;
    int ld, LS, G;
    size_t bytes;
};

// Leading dimension of the FP64 factors: K rounded up to 2 (16-byte rows).
inline int ws64_ld(int K) { return (K + 1) / 2 * 2; }

inline Workspace64 carve64_ws(void* base, long M, int N, int K, int G) {
    Workspace64 w{};
    w.ld = ws64_ld(K);
    w.LS = N + w.ld;
    w.G = G;
    char* b = static_cast<char*>(base);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = (off + 255) / 256 * 256;
        void* p = b ? b + off : nullptr;
        off += (bytes > 0 ? bytes : 1);
        return p;
    };
    w.R = (double*)take(sizeof(double) * (size_t)M * N);
    w.V = (double*)take(sizeof(double) * (size_t)M * w.ld);
    w.U = (double*)take(sizeof(double) * (size_t)N * w.ld);
    w.W = (double*)take(sizeof(double) * (size_t)N * w.ld);
    w.vraw = (double*)take(sizeof(double) * (size_t)M);
    w.vcorr = (double*)take(sizeof(double) * (size_t)M);
    w.ut = (double*)take(sizeof(double) * 2 * (size_t)N);
    w.upre = (double*)take(sizeof(double) * (size_t)N);
    w.partS = (double*)take(sizeof(double) * (size_t)G * w.LS);
    w.partA = (double*)take(sizeof(double) * (size_t)G * w.ld);
    w.scal = (double*)take(sizeof(double) * 4 * (size_t)G);
    w.lam = (double*)take(sizeof(double) * (size_t)K);
    w.xpart = (double*)take(sizeof(double) * kPack64Blocks);
    w.cmean = (double*)take(sizeof(double) * (size_t)N);
    w.rmean = (double*)take(sizeof(double) * (size_t)M);
    w.iters = (int*)take(sizeof(int) * (size_t)K);
    w.info = (int*)take(sizeof(int) * 8);
    w.abort = (int*)take(sizeof(int) * 4);
    w.lock = (int*)take(sizeof(int) * (size_t)K);
    w.flags = (unsigned*)take(sizeof(unsigned) * 32);
    w.bytes = (off + 255) / 256 * 256;
    return w;
}

}  // namespace gspca
