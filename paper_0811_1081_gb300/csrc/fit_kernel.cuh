// Persistent single-problem fit kernel: NIPALS-PCA (Sec. 2.2) and GS-PCA
// (Sec. 2.3) with every iteration and every convergence decision on the device.
//
// Work split.  The grid is one cooperative launch of G CTAs.  CTA g owns
//   - a contiguous range of 4-row panels of R (rows [r0, r1)), and with them
//     the same rows of V (score directions), vraw and vcorr;
//   - a contiguous slice [n0, n1) of the N columns, and with it the same rows
//     of U (loadings), W = R^T V and upre.
// Partial sums, the pass input `ut` and a few scalars cross CTAs, always
// through a bounded grid barrier (device_common.cuh).
//
// One pass over R per power iteration.  A pass takes the current loading up to
// a positive factor nu (known exactly from the squared-norm partials of its
// input), forms v' = R u' panel by panel (FP32 products, warp butterfly,
// cross-warp sum) and, while the panel is still on chip, accumulates
// s' = R^T v'.  For GS-PCA the score correction v' - V b', b' = V^T v',
// commutes through R^T: R^T (v' - V b') = s' - W b' with W = R^T V kept up to
// date by a rank-1 update per component, so the paper's second matrix-vector
// product needs no second read of R.  The rank-1 deflation of component k-1
// (Eq. 3) is applied inside the first pass of component k, which also takes
// the start column R(k).  Panels reach shared memory through a ring of 1-D
// TMA bulk copies; the first stages of every pass are issued before the
// barrier that precedes it.
//
// Barriers per iteration: NIPALS and GS component 0 need two (after the
// pass; after the new loading); GS components k > 0 need three in the form of
// Sec. 2.3 (one more after u_pre' = s' - W b' and its coefficients
// a' = U^T u_pre').  Up to 64 components and 4096 columns per CTA the middle
// one goes: Q = R_k U and Z = U^T W are kept up to date per component like W
// (with bfloat16 storage Q's rows are recomputed from the stored residual), so
// a' = Q^T v' - Z b' (Q^T v' reduced with b' after the
// pass) and ||v' - V b'||^2 = ||v'||^2 - 2 b'.b' + b'^T V^T V b' come from
// reduced values, where that is numerically safe (see the guards at the step).
// The k-vectors are reduced by every CTA from the CTA partials when G*k is
// small, otherwise once across the grid with one more barrier each.
//
// Precision: R and every O(M N), O(M k), O(N k) product are FP32 with FP32
// sums inside a CTA; cross-CTA vector sums are FP32 over the CTA partials of
// one lane combined in float-float across lanes; every norm and scalar sum
// is float-float; lambda and the convergence test are FP64.
#pragma once

#include <cfloat>

#include "device_common.cuh"
#include "warmstart.cuh"

namespace gspca {

constexpr int kBlock = 512;
constexpr int kMaxWarps = kBlock / 32;
constexpr int kMaxStages = 8;

enum : int { kInfoStatus = 0, kInfoFound = 1, kInfoItersLo = 2, kInfoItersHi = 3, kInfoWords = 8 };

struct FitArgs {
    int M, N, K, np;          // np = number of 4-row panels (Mp / 4)
    int algo;                 // 0 = NIPALS, 1 = GS
    int max_iter;
    double tol;
    double eps_thresh;        // degenerate threshold factor: lambda <= eps_thresh * ||X||_F
    const double* xpart;      // partial sums of squares of the packed X
    int nxpart;
    void* R;                  // [np][ldp] cells (Cell<E>): row 4p+q, column c in cell p*ldp + c
    int ldp;                  // cells per panel (panel_cells(N, Cell<E>::kBytes))
    float* V;                 // Mp x ldv row-major: V[r*ldv + k]
    int ldv;
    float* U;                 // N x ldu row-major
    int ldu;
    float* W;                 // N x ldw row-major (R^T V)
    int ldw;
    float* vraw;              // Mp: v' of the last pass
    float* vcorr;             // Mp: v' - V b'
    float* ut;                // 2 x N: pass input, double-buffered
    float* upre;              // N: s' - W b' (pass scale)
    float* partA;             // G x LA vector partials of the pass (s' | b' or Gram row)
    int LA;
    float* partB;             // G x LB vector partials of the GS step (a')
    int LB;
    float2* spart;            // G x 4 float-float scalars: [0] pass, [1] lambda'^2, [2+b] ||ut[b]||^2
    double* red;              // LA doubles: grid-wide reductions (large k, start-column fallback)
    double* lam;              // K
    int* iters;               // K
    int* info;                // kInfoWords
    unsigned* flags;          // barrier arrival counter (flags[0]), zeroed before the launch
    int* abort;
    long long* facc;          // WIDE kernels: 2 x ldk 64-bit fixed-point accumulators of b' and a'
                              // (zeroed by the kernel itself)
    float* coef_trace;        // testing aid, nullable: per component k >= 1, at k (2K + M + N), the
                              // last iteration's b' (K slots), a' (K slots), v' (M) and u_pre' (N)
    const int* iters_lock;    // device, K entries, nullable
    unsigned long long timeout_ns;
    unsigned long long* timing;  // phase-time accumulators (instrumented builds only), nullable
    int tma_stages;           // TMA ring stages (0 = panels loaded straight into registers)
    int ring_bytes;           // shared-memory bytes reserved for the ring (vectors follow)
    int dot_groups;           // 2: the loading pass runs as two independent 256-thread groups
    int ldk;                  // shared-memory length of the k-vectors (>= K)
    int max_slice;            // shared-memory length of the N slice (>= n1 - n0)
    int redundant_max;        // reduce k-vectors in every CTA when k <= this
    int narrow;               // 1: the loading pass is pass_lds (N <= 1024, no CTA ring)
    int res_rows;             // > 0: this CTA's rows of V (res_rows) and its slices of U and W
                              // (max_slice each) live in shared memory at byte res_off
    int res_off;
    int gs2;                  // 1 (single-problem GS-PCA, resident, K <= 64, up to 4096 columns
                              // per CTA; bfloat16 storage recomputes Q's rows per component): the
                              // resident block also holds this CTA's rows of Q = R_k U_(k) and the
                              // matrices Z = U^T W and V^T V (ldk x ldk), kept up to date per component, and an
                              // iteration may form a' and ||v' - V b'||^2 from them (two grid-wide
                              // reductions per iteration instead of three)
    // learned warm start (GS-PCA; all null when off)
    const float* ws_net;      // kWsParams network parameters
    const float* ws_G;        // sketch, M x 16 row-major
    float* wsF;               // N x 17: squared norm and sketch of every column of the current residual
    float* wsP0;              // N: network output for the current component
    float* pC;                // G x N: CTA partials of R^T v_b (the learned candidate)
    float* wsPart;            // G x 32: CTA partials of the per-component feature update
    float* wsInit;            // G x 17 x N: CTA partials of the initial sketch
    int* ws_choice;           // K, nullable: 1 where the learned start was used
    const int* stall_word;    // testing, nullable: a word nothing sets; the first ring wait of
                              // every pass first waits for it (bounded) and so runs out
};

struct __align__(16) SmemFit {
    float wsum[2][kMaxWarps][32];
    float wsum2[2][2][kMaxWarps / 2][4];
    ff ffg[2];
    float vrow[2][32];
    float tmpf[kMaxWarps][128];
    ff ffw[kMaxWarps];
    ff ffq[kMaxWarps][4];
    ff sff[4];
    ff lamff;
    ff lam2s;
    double dsc[4];
    double wsv[24];
    unsigned long long mbar[kMaxStages];
    int flag;
    int sel;
    int stop;
    int step2;
    int mbar_live;
#ifdef GSPCA_PHASE_TIMING
    unsigned long long tacc[16];
    unsigned long long tlast;
    int tcur;
    int tmark;  // this CTA records phase times
#endif
};

// Instrumented builds (-DGSPCA_PHASE_TIMING) accumulate, in CTA 0, the
// %globaltimer time spent in each phase of the loop; product builds compile
// the marks away.
#ifdef GSPCA_PHASE_TIMING
#define PHASE_MARK(id)                                      \
    do {                                                    \
        if (threadIdx.x == 0 && sm.tmark) {                 \
            const unsigned long long t_ = globaltimer_ns(); \
            sm.tacc[sm.tcur] += t_ - sm.tlast;              \
            sm.tlast = t_;                                  \
            sm.tcur = (id);                                 \
        }                                                   \
    } while (0)
#else
#define PHASE_MARK(id) \
    do {               \
    } while (0)
#endif

template <int CPT>
struct PassShape {
    static constexpr int PPR = (CPT >= 8) ? 1 : 8 / CPT;  // panels per round
    static constexpr int RPR = 4 * PPR;                   // rows per round
};

// ------------------------------------------------------------------ TMA ring

// Per-CTA ring of S shared-memory stages, each holding PPR consecutive panels
// of this CTA's rows.  Sequence numbers run across passes: sequence q lives in
// stage q % S and completes phase (q / S) & 1 of that stage's mbarrier.  Only
// thread 0 issues copies; every thread keeps the counters identically.
struct Ring {
    unsigned char* base;
    unsigned long long* mbar;
    int S;
    int stage_bytes;
    unsigned issued;  // sequences issued so far
    unsigned used;    // sequences consumed so far

    __device__ __forceinline__ unsigned char* stage(unsigned q) const { return base + (size_t)(q % S) * stage_bytes; }
    __device__ __forceinline__ uint64_t* bar(unsigned q) const { return reinterpret_cast<uint64_t*>(&mbar[q % S]); }
};

// Issue round i (sequence rg.issued) of a pass over panels [p0, p1).
template <class E>
__device__ __forceinline__ void ring_issue(const FitArgs& f, Ring& rg, int p0, int p1, int ppr, int i) {
    constexpr int CB = Cell<E>::kBytes;
    const unsigned q = rg.issued;
    const int pa = p0 + i * ppr;
    const int npan = min(ppr, p1 - pa);
    if (threadIdx.x == 0)
        tma_load_1d(rg.stage(q), static_cast<const unsigned char*>(f.R) + (size_t)pa * f.ldp * CB,
                    (uint32_t)npan * (uint32_t)f.ldp * (uint32_t)CB, rg.bar(q));
    rg.issued = q + 1;
}

// Issue the first rounds of the next pass (e.g. before the barrier preceding it).
template <class E>
__device__ __forceinline__ void ring_prefetch(const FitArgs& f, Ring& rg, int p0, int p1, int ppr) {
    if (rg.S == 0) return;
    const int nrounds = (p1 - p0 + ppr - 1) / ppr;
    for (int i = (int)(rg.issued - rg.used); i < rg.S && i < nrounds; ++i) ring_issue<E>(f, rg, p0, p1, ppr, i);
}

// A ring wait that gave up after the caller's limit is reported as a timeout,
// but the copy it waited for was issued and normally lands a little later: the
// stage is awaited again, for at most this long, before it is read, refilled
// or abandoned, so that no copy is still in flight when its stage (or the
// CTA's shared memory) is reused.
constexpr unsigned long long kSettleNs = 1000000000ull;

// Testing hook: wait, bounded by the caller's limit, for a word that nothing
// sets; returns false when the limit runs out.
__device__ __forceinline__ bool stall_wait(const FitArgs& f) {
    const uint64_t t0 = globaltimer_ns();
    while (ld_relaxed_s32(f.stall_word) == 0)
        if (globaltimer_ns() - t0 > f.timeout_ns) return false;
    return true;
}

// Wait (bounded) for the copies still in flight (before leaving, or before the
// ring is set up again).
__device__ __forceinline__ void ring_drain(const FitArgs& f, const Ring& rg) {
    const unsigned long long bound = f.timeout_ns > kSettleNs ? f.timeout_ns : kSettleNs;
    if (threadIdx.x == 0)
        for (unsigned q = rg.used; q < rg.issued; ++q)
            if (!mbar_wait(rg.bar(q), (q / rg.S) & 1u, bound)) break;
    __syncthreads();
}

// ------------------------------------------------------------------ passes

enum : int { kPassDot = 0, kPassCol = 1, kPassSq = 2 };

// One streaming pass over the CTA's panels [p0, p1).
//   kPassDot: rows = R u' (u' in uc[]), written to vraw; sacc = R^T rows;
//             sc = sum rows^2.  Panels come through the TMA ring when S > 0.
//   kPassCol: rows = R(:, kcol) after the optional deflation
//             R <- R - (lamf * V(:, kprev)) uc^T; sacc = R^T rows;
//             sc = ||R(:, kcol)||^2 over the CTA's rows.  Register path.
//   kPassSq : sacc = column sums of squares (start-column fallback).
// Returns false (in every thread) if a bounded wait on the ring timed out.
template <int CPT, int MODE, class E>
__device__ __forceinline__ bool row_pass(const FitArgs& f, SmemFit& sm, Ring& rg, int p0, int p1,
                                         const float (&uc)[CPT], int kcol, bool deflate, float lamf, int kprev,
                                         float (&sacc)[CPT], ff& sc) {
    constexpr int PPR = PassShape<CPT>::PPR;
    constexpr int RPR = PassShape<CPT>::RPR;
    constexpr int SH = 5 - Log2<RPR>::value;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int T = blockDim.x, N = f.N;
    const size_t ldp = (size_t)f.ldp;
    const bool tma = (MODE == kPassDot) && rg.S > 0;
    int owner = -1;
    if (MODE == kPassCol && (kcol % T) == tid) owner = kcol / T;
#pragma unroll
    for (int i = 0; i < CPT; ++i) sacc[i] = 0.f;
    ff my = ff_zero();
    int ok = 1;
    if (tma) ring_prefetch<E>(f, rg, p0, p1, PPR);
    const unsigned base = rg.used;
    int buf = 0;
    int round = 0;
    for (int pb = p0; pb < p1; pb += PPR, buf ^= 1, ++round) {
        float4 d[PPR][CPT];
        if (tma) {
            const unsigned q = base + (unsigned)round;
            if (f.stall_word && round == 0 && !stall_wait(f)) ok = 0;
            if (!mbar_wait(rg.bar(q), (q / rg.S) & 1u, f.timeout_ns)) {
                ok = 0;  // reported; the stage is still awaited before it is read or refilled
                mbar_wait(rg.bar(q), (q / rg.S) & 1u, kSettleNs);
            }
            const unsigned char* st = rg.stage(q);
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int c = tid + i * T;
                    d[pp][i] = (pb + pp < p1 && c < N) ? Cell<E>::lds(st, (size_t)pp * ldp + c)
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        } else {
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                const int p = pb + pp;
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int c = tid + i * T;
                    d[pp][i] = (p < p1 && c < N) ? Cell<E>::ldg(f.R, (size_t)p * ldp + c)
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                }
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
                    v = Cell<E>::quant(v);  // the stored residual, as later passes read it
                    d[pp][i] = v;
                    if (p < p1 && c < N) Cell<E>::stg(f.R, (size_t)p * ldp + c, v);
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
            if ((lane & ((1 << SH) - 1)) == 0) sm.wsum[buf][warp][lane >> SH] = r;
            // One CTA barrier per round: the warp partials are double-buffered by
            // round parity, and every warp finishes the row sums itself.
            __syncthreads();
            // every thread has its panel data in registers: refill this stage
            if (tma) {
                const int ahead = round + rg.S;
                if (pb + rg.S * PPR < p1 && (int)(rg.issued - base) == ahead) ring_issue<E>(f, rg, p0, p1, PPR, ahead);
            }
            float rs = 0.f;
            if (lane < RPR)
                for (int w = 0; w < nw; ++w) rs += sm.wsum[buf][w][lane];
            if (warp == 0 && lane < RPR && pb + (lane >> 2) < p1) {
                f.vraw[(size_t)pb * 4 + lane] = rs;
                my = ff_add(my, ff_sqr(rs));
            }
#pragma unroll
            for (int r2 = 0; r2 < RPR; ++r2) rowv[r2] = __shfl_sync(kFull, rs, r2);
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
                    my = ff_add(my, ff_sqr(x.x));
                    my = ff_add(my, ff_sqr(x.y));
                    my = ff_add(my, ff_sqr(x.z));
                    my = ff_add(my, ff_sqr(x.w));
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
    if (tma) rg.used = base + (unsigned)round;
    // CTA total of `my` (nonzero only in warp 0 for kPassDot, in the owner for kPassCol).
    if (MODE == kPassDot) {
        if (warp == 0) {
            const ff t = warp_sum_ff(my);
            if (lane == 0) sm.sff[3] = t;
        }
    } else if (MODE == kPassCol) {
        if (owner >= 0) sm.sff[3] = my;
    } else {
        if (tid == 0) sm.sff[3] = ff_zero();
    }
    const int all_ok = __syncthreads_and(ok);
    sc = sm.sff[3];
    __syncthreads();
    return all_ok != 0;
}

// bf_unpack through opaque instructions, so the compiler re-derives the values
// instead of keeping an earlier unpacking of the same words alive.
__device__ __forceinline__ float4 bf_unpack_again(uint2 w) {
    uint32_t a, b, c, d;
    asm volatile("shl.b32 %0, %1, 16;" : "=r"(a) : "r"(w.x));
    asm volatile("and.b32 %0, %1, 0xffff0000;" : "=r"(b) : "r"(w.x));
    asm volatile("shl.b32 %0, %1, 16;" : "=r"(c) : "r"(w.y));
    asm volatile("and.b32 %0, %1, 0xffff0000;" : "=r"(d) : "r"(w.y));
    return make_float4(__uint_as_float(a), __uint_as_float(b), __uint_as_float(c), __uint_as_float(d));
}

// Loading pass (kPassDot) for bfloat16 storage read straight into registers (up
// to 4096 columns per CTA; wider rows would not fit the registers):
// a cell stays packed (two 32-bit words) until it is used and is unpacked twice
// (for R u' and for R^T v'), and the packed cells of the next round are loaded
// before the current one is used, so two rounds of R are in flight in the
// registers a FP32 round occupies.  Same arithmetic as row_pass<kPassDot>.
// Input u' from u_in (N values), output: the CTA's s' partials in pA[0..N).
template <int CPT>
__device__ __noinline__ void pass_dot_reg_bf16(const FitArgs& f, SmemFit& sm, int p0, int p1, const float* u_in,
                                               float* pA, ff* sc_out) {
    constexpr int PPR = PassShape<CPT>::PPR;
    constexpr int RPR = PassShape<CPT>::RPR;
    constexpr int SH = 5 - Log2<RPR>::value;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int T = blockDim.x, N = f.N;
    const size_t ldp = (size_t)f.ldp;
    const uint2* Rw = static_cast<const uint2*>(f.R);
    float uc[CPT], sacc[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = tid + i * T;
        uc[i] = c < N ? ldcg(u_in + c) : 0.f;
        sacc[i] = 0.f;
    }
    ff my = ff_zero();
    uint2 nxt[PPR][CPT];
    auto load = [&](int pb) {
#pragma unroll
        for (int pp = 0; pp < PPR; ++pp)
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T, p = pb + pp;
                uint2 w = make_uint2(0u, 0u);
                if (p < p1 && c < N)
                    asm volatile("ld.global.cg.v2.u32 {%0,%1}, [%2];" : "=r"(w.x), "=r"(w.y) : "l"(Rw + (size_t)p * ldp + c));
                nxt[pp][i] = w;
            }
    };
    if (p0 < p1) load(p0);
    int buf = 0;
    for (int pb = p0; pb < p1; pb += PPR, buf ^= 1) {
        uint2 cur[PPR][CPT];
#pragma unroll
        for (int pp = 0; pp < PPR; ++pp)
#pragma unroll
            for (int i = 0; i < CPT; ++i) cur[pp][i] = nxt[pp][i];
        if (pb + PPR < p1) load(pb + PPR);
        float acc[RPR];
#pragma unroll
        for (int r = 0; r < RPR; ++r) acc[r] = 0.f;
#pragma unroll
        for (int i = 0; i < CPT; ++i)
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                const float4 d = bf_unpack(cur[pp][i]);
                acc[pp * 4 + 0] = fmaf(d.x, uc[i], acc[pp * 4 + 0]);
                acc[pp * 4 + 1] = fmaf(d.y, uc[i], acc[pp * 4 + 1]);
                acc[pp * 4 + 2] = fmaf(d.z, uc[i], acc[pp * 4 + 2]);
                acc[pp * 4 + 3] = fmaf(d.w, uc[i], acc[pp * 4 + 3]);
            }
        const float r = warp_multi_reduce<RPR>(acc, lane);
        if ((lane & ((1 << SH) - 1)) == 0) sm.wsum[buf][warp][lane >> SH] = r;
        __syncthreads();
        float rs = 0.f;
        if (lane < RPR)
            for (int w = 0; w < nw; ++w) rs += sm.wsum[buf][w][lane];
        if (warp == 0 && lane < RPR && pb + (lane >> 2) < p1) {
            f.vraw[(size_t)pb * 4 + lane] = rs;
            my = ff_add(my, ff_sqr(rs));
        }
        float rowv[RPR];
#pragma unroll
        for (int r2 = 0; r2 < RPR; ++r2) rowv[r2] = __shfl_sync(kFull, rs, r2);
#pragma unroll
        for (int i = 0; i < CPT; ++i)
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                // unpacked again rather than kept from the first use: the unpacked round
                // would need twice the registers across the row reduction
                const float4 d = bf_unpack_again(cur[pp][i]);
                sacc[i] = fmaf(d.x, rowv[pp * 4 + 0], sacc[i]);
                sacc[i] = fmaf(d.y, rowv[pp * 4 + 1], sacc[i]);
                sacc[i] = fmaf(d.z, rowv[pp * 4 + 2], sacc[i]);
                sacc[i] = fmaf(d.w, rowv[pp * 4 + 3], sacc[i]);
            }
    }
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = tid + i * T;
        if (c < N) pA[c] = sacc[i];
    }
    if (warp == 0) {
        const ff t = warp_sum_ff(my);
        if (lane == 0) sm.sff[3] = t;
    }
    __syncthreads();
    *sc_out = sm.sff[3];
    __syncthreads();
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Loading pass (kPassDot) as two independent groups of 256 threads.  Group g
// takes rounds g, g+2, ... of one 4-row panel each; its barriers are named
// barriers of 256 threads, so while one group waits in its barrier or its
// shuffle chain the other one computes.  Thread t of a group holds columns
// t + 256 i (i < 2 CPT) of u' (uc2) and of its s' accumulators (sacc2).  The
// ring holds one panel per stage and has an even number of stages, so round
// r + S belongs to the same group as round r and that group refills its own
// stages.  On return group 0 holds the CTA's s' partials and sc = sum v'^2.
// Returns false (in every thread) if a bounded wait on the ring timed out.
template <int CPT, class E>
__device__ __forceinline__ bool pass_dot2(const FitArgs& f, SmemFit& sm, Ring& rg, int p0, int p1,
                                          const float (&uc2)[2 * CPT], float (&sacc2)[2 * CPT], ff& sc) {
    constexpr int C2 = 2 * CPT;
    const int tid = threadIdx.x, grp = tid >> 8, lt = tid & 255, lane = tid & 31, lw = (tid >> 5) & 7;
    constexpr int CB = Cell<E>::kBytes;
    const int N = f.N, ldp = f.ldp;
#pragma unroll
    for (int i = 0; i < C2; ++i) sacc2[i] = 0.f;
    ff my = ff_zero();
    int ok = 1;
    ring_prefetch<E>(f, rg, p0, p1, 1);
    const unsigned base = rg.used;
    const int nrounds = p1 - p0;
    // stage and mbarrier phase of the group's first round; each later round of the group is
    // two sequences on (S is even: the group keeps to the stages of one parity)
    int sidx = (int)((base + (unsigned)grp) % (unsigned)rg.S);
    unsigned ph = ((base + (unsigned)grp) / (unsigned)rg.S) & 1u;
    for (int round = grp; round < nrounds; round += 2) {
        const int p = p0 + round;
        uint64_t* mb = reinterpret_cast<uint64_t*>(&rg.mbar[sidx]);
        if (f.stall_word && round == grp && !stall_wait(f)) ok = 0;
        if (!mbar_wait(mb, ph, f.timeout_ns)) {
            ok = 0;  // reported; the stage is still awaited before it is read or refilled
            mbar_wait(mb, ph, kSettleNs);
        }
        unsigned char* st = rg.base + (size_t)sidx * rg.stage_bytes;
        float4 d[C2];
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            const int c = lt + i * 256;
            d[i] = c < N ? Cell<E>::lds(st, (size_t)c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            acc[0] = fmaf(d[i].x, uc2[i], acc[0]);
            acc[1] = fmaf(d[i].y, uc2[i], acc[1]);
            acc[2] = fmaf(d[i].z, uc2[i], acc[2]);
            acc[3] = fmaf(d[i].w, uc2[i], acc[3]);
        }
        const float r = warp_multi_reduce<4>(acc, lane);  // lane l: row l >> 3
        const int par = (round >> 1) & 1;
        if ((lane & 7) == 0) sm.wsum2[grp][par][lw][lane >> 3] = r;
        named_barrier(1 + grp, 256);
        // this group has read the stage: refill it with round + S (same group)
        if (lt == 0 && round + rg.S < nrounds)
            tma_load_1d(st, static_cast<const unsigned char*>(f.R) + (size_t)(p + rg.S) * ldp * CB,
                        (uint32_t)ldp * (uint32_t)CB, mb);
        float rs = 0.f;
        if (lane < 4)
#pragma unroll
            for (int w = 0; w < 8; ++w) rs += sm.wsum2[grp][par][w][lane];
        if (lw == 0 && lane < 4 && 4 * p + lane < 4 * p1) {
            f.vraw[(size_t)p * 4 + lane] = rs;
            my = ff_add(my, ff_sqr(rs));
        }
        float rowv[4];
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) rowv[r2] = __shfl_sync(kFull, rs, r2);
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            sacc2[i] = fmaf(d[i].x, rowv[0], sacc2[i]);
            sacc2[i] = fmaf(d[i].y, rowv[1], sacc2[i]);
            sacc2[i] = fmaf(d[i].z, rowv[2], sacc2[i]);
            sacc2[i] = fmaf(d[i].w, rowv[3], sacc2[i]);
        }
        sidx += 2;
        if (sidx >= rg.S) {
            sidx -= rg.S;
            ph ^= 1u;
        }
    }
    rg.used = base + (unsigned)nrounds;
    rg.issued = rg.used;
    if (lw == 0) {
        const ff t = warp_sum_ff(my);
        if (lane == 0) sm.ffg[grp] = t;
    }
    // group 1 hands its s' partials to group 0 through the (now idle) ring memory
    const int all_ok = __syncthreads_and(ok);
    float* xch = reinterpret_cast<float*>(rg.base);
    if (grp == 1)
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            const int c = lt + i * 256;
            if (c < N) xch[c] = sacc2[i];
        }
    __syncthreads();
    if (grp == 0)
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            const int c = lt + i * 256;
            if (c < N) sacc2[i] += xch[c];
        }
    sc = ff_add(sm.ffg[0], sm.ffg[1]);
    // the exchange area is ring memory: order these generic accesses before the
    // next TMA writes into it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    return all_ok != 0;
}

// Loading pass (kPassDot) for narrow problems, N <= 256 * TW, with no
// CTA-wide barrier inside the pass.  The 16 warps form 16 / TW groups of TW
// warps; group g takes rounds g, g + 16/TW, ... of PP consecutive panels.
// Warp wi of a group owns the column chunk [256 wi, 256 wi + cw) (TW > 1) or
// all N columns (TW == 1); lane l holds columns chunk + l + 32 j (j < NJW) of
// u' and of the group's s' partials.
//
// Every lane streams its own 16-byte pieces of R (4 rows x 1 column) through
// a private ring of kLdsStages shared-memory stages with asynchronous copies
// (cp.async, one commit group per round), issued kLdsStages rounds ahead, so
// no register holds data in flight and no lane waits for another lane's copy.
// Per round: v' for the 4 PP rows (one multi-value butterfly per warp, then,
// for TW > 1, the TW warp partials summed through shared memory behind a named
// barrier of the group), then s' += R_round^T v' from the same stage.
//
// Shared memory (dyn): 16 warps x kLdsStages stages of 4 KB; at the end of the
// pass the same bytes hold the groups' s' partials (16 / TW x N floats), summed
// in a fixed order into pA[0..N).  sc = sum v'^2 over the CTA's rows.  Returns
// false (in every thread) if the testing stall hook ran out.
constexpr int kLdsStages = 3;
constexpr int kLdsStageBytes = 4096;
constexpr int kLdsBytes = kMaxWarps * kLdsStages * kLdsStageBytes;

template <int NJW, int TW>
struct LdsTraits {
    static constexpr int PP = (NJW == 8) ? 1 : 8 / NJW;  // panels per round (PP * NJW = 8 pieces per lane)
    static constexpr int CW = 32 * NJW;                  // column chunk of a warp
    static constexpr int NG = kMaxWarps / TW;            // groups
    static constexpr int GT = 32 * TW;                   // threads per group
    static constexpr int V = 4 * PP;                     // row values per round
    static_assert(PP * CW * 16 == kLdsStageBytes, "one stage holds a round");
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int NJW, int TW, class E>
__device__ __forceinline__ bool pass_lds(const FitArgs& f, SmemFit& sm, int p0, int p1, const float* __restrict__ u_in,
                                         float* pA, ff& sc, unsigned char* dyn) {
    using B = LdsTraits<NJW, TW>;
    constexpr int PP = B::PP, CW = B::CW, NG = B::NG, GT = B::GT, V = B::V, SW = kLdsStages;
    constexpr int CB = Cell<E>::kBytes;
    const size_t ldp = (size_t)f.ldp;
    constexpr int SHIFT = 5 - Log2<V>::value;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int grp = warp / TW, wi = warp % TW;
    const int N = f.N;
    const int c0 = (TW == 1) ? 0 : wi * CW;  // first column of the warp's chunk
    // its width; 0 for the last warps of a group when N <= 256 (TW - 1): those
    // warps copy and read nothing but still take part in the group's barriers
    const int cw = (TW == 1) ? N : max(0, min(CW, N - c0));
    unsigned char* stages = dyn + (size_t)warp * SW * kLdsStageBytes;
    int ok = 1;
    if (f.stall_word && !stall_wait(f)) ok = 0;
    float u[NJW], s[NJW];
#pragma unroll
    for (int j = 0; j < NJW; ++j) {
        const int c = lane + 32 * j;
        u[j] = c < cw ? ldcg(u_in + c0 + c) : 0.f;
        s[j] = 0.f;
    }
    ff my = ff_zero();
    const int npan = p1 - p0;
    const int nrounds = (npan + PP - 1) / PP;
    const int nr = nrounds > grp ? (nrounds - grp + NG - 1) / NG : 0;  // this group's rounds
    // piece (pp, j) of a round: panel pb + pp, column c0 + lane + 32 j, at
    // stage cell (pp * NJW + j) * 32 + lane (a warp's copies of one piece index
    // are 32 contiguous cells on both sides)
    auto issue = [&](int i) {
        if (i < nr) {
            unsigned char* st = stages + (size_t)(i % SW) * kLdsStageBytes;
            const int pb = p0 + (grp + NG * i) * PP;
#pragma unroll
            for (int pp = 0; pp < PP; ++pp)
#pragma unroll
                for (int j = 0; j < NJW; ++j) {
                    const int c = lane + 32 * j;
                    if (pb + pp < p1 && c < cw)
                        Cell<E>::cp_async(st + ((pp * NJW + j) * 32 + lane) * CB,
                                          static_cast<const unsigned char*>(f.R) +
                                              ((size_t)(pb + pp) * ldp + c0 + c) * CB);
                }
        }
        cp_async_commit();  // one group per round (possibly empty) keeps the counts uniform
    };
#pragma unroll
    for (int i = 0; i < SW; ++i) issue(i);
    for (int i = 0; i < nr; ++i) {
        const int pb = p0 + (grp + NG * i) * PP;
        cp_async_wait<SW - 1>();  // this lane's pieces of round i have landed
        const unsigned char* sb = stages + (size_t)(i % SW) * kLdsStageBytes;
        float4 d[PP][NJW];
#pragma unroll
        for (int pp = 0; pp < PP; ++pp)
#pragma unroll
            for (int j = 0; j < NJW; ++j) {
                const int c = lane + 32 * j;
                d[pp][j] = (pb + pp < p1 && c < cw) ? Cell<E>::lds(sb, (size_t)((pp * NJW + j) * 32 + lane))
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        float acc[V];
#pragma unroll
        for (int pp = 0; pp < PP; ++pp) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
            for (int j = 0; j < NJW; ++j) {
                a0 = fmaf(d[pp][j].x, u[j], a0);
                a1 = fmaf(d[pp][j].y, u[j], a1);
                a2 = fmaf(d[pp][j].z, u[j], a2);
                a3 = fmaf(d[pp][j].w, u[j], a3);
            }
            acc[pp * 4 + 0] = a0;
            acc[pp * 4 + 1] = a1;
            acc[pp * 4 + 2] = a2;
            acc[pp * 4 + 3] = a3;
        }
        // every piece of the stage has been used (so read): refill it with round i + SW
        issue(i + SW);
        const float wsum = warp_multi_reduce<V>(acc, lane);  // value lane >> SHIFT
        const int par = i & 1;
        if ((lane & ((1 << SHIFT) - 1)) == 0) sm.tmpf[warp][par * 32 + (lane >> SHIFT)] = wsum;
        if (TW == 1)
            __syncwarp();
        else
            named_barrier(1 + grp, GT);
        float v[V];
#pragma unroll
        for (int k4 = 0; k4 < V; k4 += 4) {
            float4 t = *reinterpret_cast<const float4*>(&sm.tmpf[grp * TW][par * 32 + k4]);
#pragma unroll
            for (int w = 1; w < TW; ++w) {
                const float4 o = *reinterpret_cast<const float4*>(&sm.tmpf[grp * TW + w][par * 32 + k4]);
                t.x += o.x;
                t.y += o.y;
                t.z += o.z;
                t.w += o.w;
            }
            v[k4] = t.x;
            v[k4 + 1] = t.y;
            v[k4 + 2] = t.z;
            v[k4 + 3] = t.w;
        }
        if (wi == 0 && lane < V) {
            float mine = v[0];
#pragma unroll
            for (int k2 = 1; k2 < V; ++k2)
                if (k2 == lane) mine = v[k2];
            const int p = pb + lane / 4;
            if (p < p1) {
                f.vraw[(size_t)p * 4 + (lane & 3)] = mine;
                my = ff_add(my, ff_sqr(mine));
            }
        }
#pragma unroll
        for (int pp = 0; pp < PP; ++pp)
#pragma unroll
            for (int j = 0; j < NJW; ++j) {
                s[j] = fmaf(d[pp][j].x, v[pp * 4 + 0], s[j]);
                s[j] = fmaf(d[pp][j].y, v[pp * 4 + 1], s[j]);
                s[j] = fmaf(d[pp][j].z, v[pp * 4 + 2], s[j]);
                s[j] = fmaf(d[pp][j].w, v[pp * 4 + 3], s[j]);
            }
    }
    cp_async_wait<0>();  // only empty groups remain; nothing may land after this
    // groups' s' partials -> pA (fixed order); sum v'^2 over the CTA
    __syncthreads();  // every stage consumed: the stage memory becomes the exchange area
    float* xch = reinterpret_cast<float*>(dyn);
#pragma unroll
    for (int j = 0; j < NJW; ++j) {
        const int c = lane + 32 * j;
        if (c < cw) xch[(size_t)grp * N + c0 + c] = s[j];
    }
    my = warp_sum_ff(my);
    if (lane == 0) sm.ffw[warp] = my;
    const int all_ok = __syncthreads_and(ok);
    for (int c = tid; c < N; c += blockDim.x) {
        float t = xch[c];
        for (int g2 = 1; g2 < NG; ++g2) t += xch[(size_t)g2 * N + c];
        pA[c] = t;
    }
    if (warp == 0) {
        ff t = lane < kMaxWarps ? sm.ffw[lane] : ff_zero();
#pragma unroll
        for (int o = 8; o >= 1; o >>= 1) t = ff_add(t, ff_shfl_xor(t, o));
        if (lane == 0) sm.sff[3] = t;
    }
    __syncthreads();
    sc = sm.sff[3];
    __syncthreads();
    return all_ok != 0;
}

// pass_lds for the column count of f (N <= 512 when CPT == 1, N <= 1024 when
// CPT == 2).
template <int CPT, class E>
__device__ __forceinline__ bool pass_narrow(const FitArgs& f, SmemFit& sm, int p0, int p1, const float* u_in,
                                            float* pA, ff& sc, unsigned char* dyn) {
    const int nj = (f.N + 31) / 32;
    if constexpr (CPT == 1) {
        if (nj <= 1) return pass_lds<1, 1, E>(f, sm, p0, p1, u_in, pA, sc, dyn);
        if (nj <= 2) return pass_lds<2, 1, E>(f, sm, p0, p1, u_in, pA, sc, dyn);
        if (nj <= 4) return pass_lds<4, 1, E>(f, sm, p0, p1, u_in, pA, sc, dyn);
        if (nj <= 8) return pass_lds<8, 1, E>(f, sm, p0, p1, u_in, pA, sc, dyn);
        return pass_lds<8, 2, E>(f, sm, p0, p1, u_in, pA, sc, dyn);
    } else {
        return pass_lds<8, 4, E>(f, sm, p0, p1, u_in, pA, sc, dyn);
    }
}

// ------------------------------------------------------------------ small products

// The factor products below read A with generic loads: A is this CTA's own
// rows of V or slice of U / W (written only by this CTA, in shared memory when
// resident) or the read-only sketch.
//
// Row-major k-column factors (V, U, W) with a power-of-two leading dimension
// lda in [4, 128] are read as float4 chunks: lda / 4 lanes cover one row, a
// warp load covers 32 / (lda / 4) consecutive rows (512 contiguous bytes), and
// a lane issues kVecRows such loads before using any of them.
constexpr int kVecRows = 8;

// Used for long row ranges only: with few rows per CTA, spreading rows over
// all warps (the general path) finishes sooner than packing them into few.
constexpr int kVecMinRows = 512;

__device__ __forceinline__ bool vec_rows(int lda, int rows) {
    return rows >= kVecMinRows && lda >= 4 && lda <= 128 && (lda & (lda - 1)) == 0;
}

template <class Y>
__device__ __forceinline__ void rows_times_matrix_vec(const float* A, int lda, int r0, int r1, int kk, Y y,
                                                      float* dst, SmemFit& sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int L4 = lda >> 2, rpw = 32 / L4, sub = lane / L4, cq = lane % L4;
    const bool live = 4 * cq < kk;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int rb = r0 + warp * rpw * kVecRows; rb < r1; rb += nw * rpw * kVecRows) {
        float4 a[kVecRows];
        float yr[kVecRows];
#pragma unroll
        for (int u = 0; u < kVecRows; ++u) {
            const int r = rb + u * rpw + sub;
            const bool ok = r < r1;
            yr[u] = ok ? y(r) : 0.f;
            a[u] = (ok && live) ? reinterpret_cast<const float4*>(A + (size_t)r * lda)[cq]
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kVecRows; ++u) {
            acc.x = fmaf(a[u].x, yr[u], acc.x);
            acc.y = fmaf(a[u].y, yr[u], acc.y);
            acc.z = fmaf(a[u].z, yr[u], acc.z);
            acc.w = fmaf(a[u].w, yr[u], acc.w);
        }
    }
    for (int o = 16; o >= L4; o >>= 1) {
        acc.x += __shfl_xor_sync(kFull, acc.x, o);
        acc.y += __shfl_xor_sync(kFull, acc.y, o);
        acc.z += __shfl_xor_sync(kFull, acc.z, o);
        acc.w += __shfl_xor_sync(kFull, acc.w, o);
    }
    if (lane < L4) *reinterpret_cast<float4*>(&sm.tmpf[warp][4 * lane]) = acc;
    __syncthreads();
    for (int t = tid; t < kk; t += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < nw; ++w) s += sm.tmpf[w][t];
        dst[t] = s;
    }
    __syncthreads();
}

template <class Pre, class Fn>
__device__ __forceinline__ void matrix_times_vector_vec(const float* A, int lda, int r0, int r1, int kk,
                                                        const float* x, Pre pre, Fn fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int L4 = lda >> 2, rpw = 32 / L4, sub = lane / L4, cq = lane % L4;
    const int j = 4 * cq;
    const float4 xv = make_float4(j < kk ? x[j] : 0.f, j + 1 < kk ? x[j + 1] : 0.f, j + 2 < kk ? x[j + 2] : 0.f,
                                  j + 3 < kk ? x[j + 3] : 0.f);
    const bool live = j < kk;
    for (int rb = r0 + warp * rpw * kVecRows; rb < r1; rb += nw * rpw * kVecRows) {
        float4 a[kVecRows];
        float pv[kVecRows];
#pragma unroll
        for (int u = 0; u < kVecRows; ++u) {
            const int r = rb + u * rpw + sub;
            const bool ok = r < r1;
            pv[u] = (ok && cq == 0) ? pre(r) : 0.f;
            a[u] = (ok && live) ? reinterpret_cast<const float4*>(A + (size_t)r * lda)[cq]
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kVecRows; ++u) {
            // columns at or past kk hold data of other components: weight 0 and masked value
            float d = (j < kk ? a[u].x * xv.x : 0.f);
            d = (j + 1 < kk) ? fmaf(a[u].y, xv.y, d) : d;
            d = (j + 2 < kk) ? fmaf(a[u].z, xv.z, d) : d;
            d = (j + 3 < kk) ? fmaf(a[u].w, xv.w, d) : d;
            for (int o = 1; o < L4; o <<= 1) d += __shfl_xor_sync(kFull, d, o);
            const int r = rb + u * rpw + sub;
            if (cq == 0 && r < r1) fn(r, d, pv[u]);
        }
    }
}

// dst[j] = sum_{r in [r0, r1)} A[r*lda + j] * y(r) for j < kk, FP32 within the CTA.
// A warp takes rows r0 + warp + 16 i (i < 8 per block) and issues every load
// of the block (A and y) before using any of them.
// rows_times_matrix of two matrices with the same rows and weights (kk <= 64):
// dstA = A^T y and dstB = B^T y over rows [r0, r1) in one sweep and one
// cross-warp sum; dstA's arithmetic is the general path's of rows_times_matrix.
template <class Y>
__device__ __forceinline__ void rows_times_two(const float* A, const float* B, int lda, int r0, int r1, int kk, Y y,
                                               float* dstA, float* dstB, SmemFit& sm) {
    constexpr int MAXR = 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    float accA[2] = {0.f, 0.f}, accB[2] = {0.f, 0.f};
    for (int rb = r0 + warp; rb < r1; rb += nw * MAXR) {
        float a[MAXR][2], b[MAXR][2], yr[MAXR];
#pragma unroll
        for (int i = 0; i < MAXR; ++i) {
            const int r = rb + nw * i;
            const bool ok = r < r1;
            yr[i] = ok ? y(r) : 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = lane + 32 * q;
                a[i][q] = (ok && j < kk) ? A[(size_t)r * lda + j] : 0.f;
                b[i][q] = (ok && j < kk) ? B[(size_t)r * lda + j] : 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < MAXR; ++i)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                accA[q] = fmaf(a[i][q], yr[i], accA[q]);
                accB[q] = fmaf(b[i][q], yr[i], accB[q]);
            }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        sm.tmpf[warp][lane + 32 * q] = accA[q];
        sm.tmpf[warp][64 + lane + 32 * q] = accB[q];
    }
    __syncthreads();
    for (int t = tid; t < 2 * kk; t += blockDim.x) {
        const int c = t < kk ? t : 64 + (t - kk);
        float s = 0.f;
        for (int w = 0; w < nw; ++w) s += sm.tmpf[w][c];
        if (t < kk)
            dstA[t] = s;
        else
            dstB[t - kk] = s;
    }
    __syncthreads();
}

// Past 128 columns (the leading dimension is then a multiple of 4, rows 16-byte
// aligned) the products below take these forms: a thread owns columns and
// sums its rows in index order (no cross-warp reduction), and a warp owns a
// row and loads up to 1024 of its columns before using any, so a product
// costs one or two L2 round trips instead of one per 64 or 128 columns.  They
// are compiled into the WIDE kernel variants only (chosen for K > 128), so the
// kernels for fewer components keep their code and register allocation.
template <class Y, class Out>
__device__ __forceinline__ void rows_times_matrix_wide_out(const float* A, int lda, int r0, int r1, int kk, Y y,
                                                           Out out) {
    constexpr int RB = 16;
    const int tid = threadIdx.x, T = blockDim.x;
    for (int j0 = 0; j0 < kk; j0 += 2 * T) {
        const int ja = j0 + tid, jb = ja + T;
        float sa = 0.f, sb = 0.f;
        for (int rb = r0; rb < r1; rb += RB) {
            float a[RB], b[RB], yr[RB];
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int r = rb + i;
                const bool ok = r < r1;
                yr[i] = ok ? y(r) : 0.f;
                a[i] = (ok && ja < kk) ? A[(size_t)r * lda + ja] : 0.f;
                b[i] = (ok && jb < kk) ? A[(size_t)r * lda + jb] : 0.f;
            }
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                sa = fmaf(a[i], yr[i], sa);
                sb = fmaf(b[i], yr[i], sb);
            }
        }
        if (ja < kk) out(ja, sa);
        if (jb < kk) out(jb, sb);
    }
    __syncthreads();
}

template <class Y>
__device__ __forceinline__ void rows_times_matrix_wide(const float* A, int lda, int r0, int r1, int kk, Y y,
                                                       float* dst) {
    rows_times_matrix_wide_out(A, lda, r0, r1, kk, y, [&](int j, float s) { dst[j] = s; });
}

// Grid-wide sums of k-vectors without a second barrier (WIDE kernels): every
// CTA adds its FP32 partials, scaled by 2^S and rounded to integers, into 64-bit
// accumulators with integer atomics before the barrier that precedes their use,
// and every CTA reads the sums after it.  Integer addition is exact and
// independent of order, so the sums are deterministic.  S is chosen, alike in
// every CTA, from a bound on every partial: G * bound * 2^S <= 2^61, so no sum
// can overflow; the unit 2^-S is about 2^-52 of the bound (far below the FP32
// rounding of the partials themselves).
// S from two factors of the bound, a and b (G a b < 2^e), in integer and FP32
// arithmetic only (GB300 runs FP64 at a small fraction of the FP32 rate).
__device__ __forceinline__ int fx_shift(float a, float b, int G) {
    const int e = (32 - __clz(G)) + ilogbf(fmaxf(a, FLT_MIN)) + 1 + ilogbf(fmaxf(b, FLT_MIN)) + 1;
    return 61 - e;
}

__device__ __forceinline__ void fx_add(long long* acc, float x, int S, int G) {
    const float lim = ldexpf(1.f, 61 - (32 - __clz(G)));  // 2^61 / G or less
    float y = ldexpf(x, S);  // exact: a power-of-two scaling within the FP32 range
    if (!(y == y)) y = 0.f;  // NaN (a failed pass): the degenerate test catches it
    y = fminf(fmaxf(y, -lim), lim);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)__float2ll_rn(y));
}

__device__ __forceinline__ float fx_get(const long long* acc, int S) {
    return ldexpf(__ll2float_rn(__ldcg(acc)), -S);
}

template <class Pre, class Fn>
__device__ __forceinline__ void matrix_times_vector_wide(const float* A, int lda, int r0, int r1, int kk,
                                                         const float* x, Pre pre, Fn fn) {
    constexpr int Q = 8;  // float4 per lane: 1024 columns per round trip
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = r0 + warp; r < r1; r += nw) {
        const float pv = lane == 0 ? pre(r) : 0.f;
        const float* ar = A + (size_t)r * lda;
        float acc = 0.f;
        for (int j0 = 0; j0 < kk; j0 += 128 * Q) {
            float4 a[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int j = j0 + 4 * lane + 128 * q;
                a[q] = j < kk ? *reinterpret_cast<const float4*>(ar + j) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int j = j0 + 4 * lane + 128 * q;
                // columns at or past kk hold data of other components: not used
                if (j < kk) acc = fmaf(a[q].x, x[j], acc);
                if (j + 1 < kk) acc = fmaf(a[q].y, x[j + 1], acc);
                if (j + 2 < kk) acc = fmaf(a[q].z, x[j + 2], acc);
                if (j + 3 < kk) acc = fmaf(a[q].w, x[j + 3], acc);
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) fn(r, acc, pv);
    }
}

// WIDE: the wide forms are compiled in (the WIDE single-problem kernels).
template <bool WIDE = false, class Y>
__device__ __forceinline__ void rows_times_matrix(const float* A, int lda, int r0, int r1, int kk, Y y, float* dst,
                                                  SmemFit& sm) {
    if (WIDE && kk > 128) {
        rows_times_matrix_wide(A, lda, r0, r1, kk, y, dst);
        return;
    }
    if (vec_rows(lda, r1 - r0)) {
        rows_times_matrix_vec(A, lda, r0, r1, kk, y, dst, sm);
        return;
    }
    constexpr int MAXR = 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int j0 = 0; j0 < kk; j0 += 128) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int rb = r0 + warp; rb < r1; rb += nw * MAXR) {
            float a[MAXR][4], yr[MAXR];
#pragma unroll
            for (int i = 0; i < MAXR; ++i) {
                const int r = rb + nw * i;
                const bool ok = r < r1;
                yr[i] = ok ? y(r) : 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = j0 + lane + 32 * q;
                    a[i][q] = (ok && j < kk) ? A[(size_t)r * lda + j] : 0.f;
                }
            }
#pragma unroll
            for (int i = 0; i < MAXR; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(a[i][q], yr[i], acc[q]);
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

// For every row r in [r0, r1): fn(r, sum_j A[r*lda + j] * x[j], pre(r)) with x
// (kk floats) in shared memory; fn runs in one lane per row.  A warp takes rows
// r0 + warp + 16 i (i < 8 per block), issues all their loads (and pre(r))
// first, and reduces the 8 row sums across lanes with one multi-value
// butterfly.
template <bool WIDE = false, class Pre, class Fn>
__device__ __forceinline__ void matrix_times_vector(const float* A, int lda, int r0, int r1, int kk, const float* x,
                                                    Pre pre, Fn fn) {
    if (WIDE && kk > 128) {
        matrix_times_vector_wide(A, lda, r0, r1, kk, x, pre, fn);
        return;
    }
    if (vec_rows(lda, r1 - r0)) {
        matrix_times_vector_vec(A, lda, r0, r1, kk, x, pre, fn);
        return;
    }
    constexpr int MAXR = 8, MAXJ = 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int rb = r0 + warp; rb < r1; rb += nw * MAXR) {
        float acc[MAXR], pv[MAXR];
#pragma unroll
        for (int i = 0; i < MAXR; ++i) {
            acc[i] = 0.f;
            const int r = rb + nw * i;
            pv[i] = (r < r1) ? pre(r) : 0.f;
        }
        for (int j0 = 0; j0 < kk; j0 += 32 * MAXJ) {
            float a[MAXR][MAXJ];
#pragma unroll
            for (int i = 0; i < MAXR; ++i)
#pragma unroll
                for (int q = 0; q < MAXJ; ++q) {
                    const int r = rb + nw * i, j = j0 + lane + 32 * q;
                    a[i][q] = (r < r1 && j < kk) ? A[(size_t)r * lda + j] : 0.f;
                }
#pragma unroll
            for (int q = 0; q < MAXJ; ++q) {
                const int j = j0 + lane + 32 * q;
                const float xj = j < kk ? x[j] : 0.f;
#pragma unroll
                for (int i = 0; i < MAXR; ++i) acc[i] = fmaf(a[i][q], xj, acc[i]);
            }
        }
        const float sum = warp_multi_reduce<MAXR>(acc, lane);  // lane l: row index l >> 2
        const int i = lane >> 2;
        float p = pv[0];
#pragma unroll
        for (int t = 1; t < MAXR; ++t)
            if (t == i) p = pv[t];
        const int r = rb + nw * i;
        if ((lane & 3) == 0 && r < r1) fn(r, sum, p);
    }
}

// For every row r in [r0, r1): fn(r, A_r . x, B_r . y, pre(r)) with kk <= 64
// columns and x, y in shared memory; each product in the order of the general
// path of matrix_times_vector.
// A warp takes rows r0 + warp, r0 + warp + 16, ... one at a time: the rows are a
// CTA's slice of the N columns (a few dozen), so a wider unrolled block would mostly
// carry masked rows through its shuffles.
template <class Pre, class Fn>
__device__ __forceinline__ void matrix_times_two(const float* A, const float* B, int lda, int r0, int r1, int kk,
                                                 const float* x, const float* y, Pre pre, Fn fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool c0 = lane < kk, c1 = lane + 32 < kk;
    const float x0 = c0 ? x[lane] : 0.f, x1 = c1 ? x[lane + 32] : 0.f;
    const float y0 = c0 ? y[lane] : 0.f, y1 = c1 ? y[lane + 32] : 0.f;
    for (int r = r0 + warp; r < r1; r += nw) {
        const float pv = pre(r);
        const float* ar = A + (size_t)r * lda;
        const float* br = B + (size_t)r * lda;
        const float a0 = c0 ? ar[lane] : 0.f, a1 = c1 ? ar[lane + 32] : 0.f;
        const float b0 = c0 ? br[lane] : 0.f, b1 = c1 ? br[lane + 32] : 0.f;
        const float sA = warp_sum(fmaf(a1, x1, fmaf(a0, x0, 0.f)));
        const float sB = warp_sum(fmaf(b1, y1, fmaf(b0, y0, 0.f)));
        if (lane == 0) fn(r, sA, sB, pv);
    }
}

// CTA-wide float-float sum (deterministic: warp butterflies, then a 16-lane
// butterfly over the warp sums), result in every thread.
__device__ __forceinline__ ff block_sum_ff(ff v, SmemFit& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_ff(v);
    if (lane == 0) sm.ffw[warp] = v;
    __syncthreads();
    if (warp == 0) {
        ff t = lane < nw ? sm.ffw[lane] : ff_zero();
#pragma unroll
        for (int o = 8; o >= 1; o >>= 1) t = ff_add(t, ff_shfl_xor(t, o));
        if (lane == 0) sm.sff[2] = t;
    }
    __syncthreads();
    const ff r = sm.sff[2];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ reductions

// Every CTA reduces, over the G CTA rows,
//   - nq <= 2 float-float scalar slots s0, s1 into sm.sff[0..nq), and
//   - nv virtual columns col(v) of a FP32 partial buffer into out[0..nv)
//     (shared memory, FP32 rounded from float-float).
// All loads of the scalars and of the first block of 64 columns are issued
// before any of them is used (one L2 round trip).  Warp w loads rows w, w+16,
// ...; lane l loads columns l and l+32 of a block; a thread sums its rows in
// FP32, the 16 warp sums of a column combine in a fixed float-float butterfly.
template <int MAXJ = 2, class Col>
__device__ __forceinline__ void gather_reduce(const FitArgs& f, SmemFit& sm, int G, int nq, int s0, int s1,
                                              const float* part, int L, int nv, Col col, float* out) {
    static_assert(MAXJ == 2 || MAXJ == 4, "32 MAXJ values per round trip");
    constexpr int MAXI = 10, NW = kMaxWarps;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float2 q0 = make_float2(0.f, 0.f), q1 = make_float2(0.f, 0.f);
    if (t < G) {
        if (nq > 0) q0 = ldcg(f.spart + (size_t)t * 4 + s0);
        if (nq > 1) q1 = ldcg(f.spart + (size_t)t * 4 + s1);
    }
    for (int vb = 0; vb < nv || vb == 0; vb += 32 * MAXJ) {
        float s[MAXJ];
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) s[j] = 0.f;
        for (int rb = 0; rb < G && vb < nv; rb += NW * MAXI) {
            float x[MAXI][MAXJ];
#pragma unroll
            for (int i = 0; i < MAXI; ++i)
#pragma unroll
                for (int j = 0; j < MAXJ; ++j) {
                    const int r = rb + warp + NW * i, v = vb + lane + 32 * j;
                    x[i][j] = (r < G && v < nv) ? ldcg(part + (size_t)r * L + col(v)) : 0.f;
                }
#pragma unroll
            for (int j = 0; j < MAXJ; ++j)
#pragma unroll
                for (int i = 0; i < MAXI; ++i) s[j] += x[i][j];
        }
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) sm.tmpf[warp][lane + 32 * j] = s[j];
        if (vb == 0 && nq > 0) {
            const ff a0 = warp_sum_ff(ff{q0.x, q0.y});
            const ff a1 = warp_sum_ff(ff{q1.x, q1.y});
            if (lane == 0) {
                sm.ffq[warp][0] = a0;
                sm.ffq[warp][1] = a1;
            }
        }
        __syncthreads();
        for (int cb = 0; cb < 32 * MAXJ && vb + cb < nv; cb += 64) {
            // warp w combines columns cb + 4w .. cb + 4w + 3 of the block: lane = 8*c + h
            const int c = cb + 4 * warp + (lane >> 3), h = lane & 7;
            ff a = ff_add(ff{sm.tmpf[h][c], 0.f}, ff{sm.tmpf[h + 8][c], 0.f});
            a = ff_add(a, ff_shfl_xor(a, 1));
            a = ff_add(a, ff_shfl_xor(a, 2));
            a = ff_add(a, ff_shfl_xor(a, 4));
            if (h == 0 && vb + c < nv) out[vb + c] = __fadd_rn(a.hi, a.lo);
        }
        if (vb == 0 && nq > 0 && warp == NW - 1) {  // lane = 16*q + w
            const int q = lane >> 4, w = lane & 15;
            ff a = (q < nq) ? sm.ffq[w][q] : ff_zero();
#pragma unroll
            for (int o = 8; o >= 1; o >>= 1) a = ff_add(a, ff_shfl_xor(a, o));
            if (w == 0 && q < nq) sm.sff[q] = a;
        }
        __syncthreads();
    }
}

// Sum of column c of a G x L FP32 partial buffer: lane l adds CTA rows
// l, l+32, ... in FP32 (loads issued together), then a fixed float-float
// butterfly across the 32 lanes.  Result in every lane.
__device__ __forceinline__ ff column_sum(const float* part, int G, int L, int c) {
    const int lane = threadIdx.x & 31;
    float s = 0.f;
#pragma unroll 8
    for (int r = lane; r < G; r += 32) s += ldcg(part + (size_t)r * L + c);
    return warp_sum_ff(ff{s, 0.f});
}

// Columns [c0, c0+nc) reduced once across the whole grid into red[0..nc)
// (FP64): columns are dealt to the warps of all CTAs in a fixed pattern.
__device__ __forceinline__ void reduce_cols_distributed(const float* part, int G, int g, int L, int c0, int nc,
                                                        double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int gw = g * nw + warp, nwt = G * nw;
    for (int c = gw; c < nc; c += nwt) {
        const ff t = column_sum(part, G, L, c0 + c);
        if (lane == 0) red[c] = ff_to_double(t);
    }
}

__device__ __forceinline__ void write_scalar(const FitArgs& f, int g, int slot, ff v) {
    if (threadIdx.x == 0) f.spart[(size_t)g * 4 + slot] = make_float2(v.hi, v.lo);
}

// ------------------------------------------------------------------ teams

// The CTAs that fit one problem together.  TeamGrid: every CTA of a
// cooperative launch, synchronised by the bounded counter barrier (a failed
// wait means "leave the kernel").  TeamCluster: the CTAs of one thread-block
// cluster, synchronised by the hardware cluster barrier (release/acquire at
// cluster scope orders their global-memory partials).
//
// A pass whose bounded ring wait gave up calls fail(): the grid team raises
// the kernel-wide abort word and leaves at once (the other CTAs see the word
// inside their barrier waits); the cluster team cannot leave a hardware
// barrier early, so it records the failure in a per-team word and carries on
// with a NaN pass scalar, which every CTA of the team reduces to the same
// "degenerate" exit at the next test.
struct TeamGrid {
    int G, g;
    GridBarrier bar;
    __device__ __forceinline__ bool sync(unsigned& epoch, int* flag) const { return bar.sync(epoch, flag); }
    __device__ __forceinline__ bool fail(const FitArgs& f) const {
        if (threadIdx.x == 0) atomicCAS(f.abort, 0, kStTimeout);
        return true;
    }
};

struct TeamCluster {
    int G, g;
    int* failed;  // per-team word, read by the caller after the team's last barrier
    __device__ __forceinline__ bool sync(unsigned& epoch, int*) const {
        ++epoch;
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        return true;
    }
    __device__ __forceinline__ bool fail(const FitArgs&) const {
        if (threadIdx.x == 0) atomicExch(failed, 1);
        return false;
    }
};

struct FitOutcome {
    int status, found;
    long long total;
    bool alive;  // false: a bounded wait gave up, the kernel must leave
};

// ------------------------------------------------------------------ learned warm start

// Sums over the team's CTAs of nv values: value j = sum_g part[g * stride + j],
// in double, into out[j] (shared memory).  A warp per value; its lanes load the
// CTA rows lane, lane + 32, ... together (one L2 round trip) and combine them
// with a fixed butterfly, so the result is deterministic.
__device__ __forceinline__ void team_sum(const float* part, int stride, int G, int nv, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < nv; j += nw) {
        double t = 0.0;
        for (int g2 = lane; g2 < G; g2 += 32) t += (double)ldcg(part + (size_t)g2 * stride + j);
        t = warp_sum(t);
        if (lane == 0) out[j] = t;
    }
    __syncthreads();
}

// Sketch of the initial residual.  Every CTA accumulates, for every column, the
// squared norm and the 16 sketch sums G^T R(n) over its own panels (a thread
// per column, rows in order), writes them to wsInit[g][j][n]; after the team
// barrier each CTA sums its column slice over the team in CTA order into wsF.
// Returns false if the barrier failed.
template <class E, class Team>
__device__ __noinline__ bool ws_sketch_init(const FitArgs& f, const Team& tm, SmemFit& sm, unsigned& epoch, int p0,
                                            int p1, int n0, int n1) {
    const int tid = threadIdx.x, T = blockDim.x, N = f.N;
    for (int c = tid; c < N; c += T) {
        float acc[kWsIn];
#pragma unroll
        for (int j = 0; j < kWsIn; ++j) acc[j] = 0.f;
        for (int p = p0; p < p1; ++p) {
            const float4 d = Cell<E>::ldg(f.R, (size_t)p * f.ldp + c);
            const float v4[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = 4 * p + q;
                if (row >= f.M) break;
                const float v = v4[q];
                acc[0] = fmaf(v, v, acc[0]);
                const float4* g4 = reinterpret_cast<const float4*>(f.ws_G + (size_t)row * kWsSketch);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float4 gg = __ldg(g4 + h);
                    acc[1 + 4 * h] = fmaf(gg.x, v, acc[1 + 4 * h]);
                    acc[2 + 4 * h] = fmaf(gg.y, v, acc[2 + 4 * h]);
                    acc[3 + 4 * h] = fmaf(gg.z, v, acc[3 + 4 * h]);
                    acc[4 + 4 * h] = fmaf(gg.w, v, acc[4 + 4 * h]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kWsIn; ++j) f.wsInit[((size_t)tm.g * kWsIn + j) * N + c] = acc[j];
    }
    if (!tm.sync(epoch, &sm.flag)) return false;
    // a warp per (column, value) of this CTA's slice, CTA partials in order
    const int nc = n1 - n0, lane = tid & 31;
    for (int e = tid >> 5; e < nc * kWsIn; e += T >> 5) {
        const int n = n0 + e / kWsIn, j = e % kWsIn;
        double t = 0.0;
        for (int g2 = lane; g2 < tm.G; g2 += 32) t += (double)ldcg(f.wsInit + ((size_t)g2 * kWsIn + j) * N + n);
        t = warp_sum(t);
        if (lane == 0) f.wsF[(size_t)n * kWsIn + j] = (float)t;
    }
    return true;
}

// Features and network output for component k (GS-PCA).  For k > 0 the
// features first follow the deflation of component k-1, R_k = R_{k-1} -
// lambda v u^T (Eq. 3), exactly:
//   s_n <- s_n - lambda (G^T v) u_n,
//   c_n^2 <- c_n^2 - 2 lambda u_n (R_{k-1}^T v)_n + lambda^2 u_n^2,
// with (R_{k-1}^T v)_n = upre_n / ||v' - V b'|| from the last pass of k-1 and
// G^T v summed over the team.  rho^2 = sum c_n^2 / N follows the same update.
// Then a warp per column of this CTA's slice evaluates the network on
// x_n = [c_n, s_n] / rho and writes wsP0; *ww receives ||w||^2 over the team.
// Two team barriers.  Returns false if one failed.
// The network parameters are staged in `stage` (shared memory of at least
// kWsParams floats, idle at this point) when it is non-null.
template <class Team>
__device__ __noinline__ bool ws_prepare(const FitArgs& f, const Team& tm, SmemFit& sm, unsigned& epoch, int k,
                                        int r0, int r1, int n0, int n1, double lam_prev, float vinv_prev,
                                        float* stage, double* ww) {
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    float* wp = f.wsPart + (size_t)tm.g * 32;
    if (k > 0)  // G^T v_{k-1} over this CTA's rows
        rows_times_matrix(f.ws_G, kWsSketch, r0, r1, kWsSketch,
                          [&](int r) { return f.V[(size_t)r * f.ldv + (k - 1)]; }, wp, sm);
    ff a0 = ff_zero(), a1 = ff_zero(), a2 = ff_zero();
    for (int n = n0 + tid; n < n1; n += T) {
        a0 = ff_add(a0, ff{f.wsF[(size_t)n * kWsIn], 0.f});
        if (k > 0) {
            const float u = f.U[(size_t)n * f.ldu + (k - 1)];
            a1 = ff_add(a1, ff_mul_ff(u, f.upre[n] * vinv_prev));
            a2 = ff_add(a2, ff_sqr(u));
        }
    }
    a0 = block_sum_ff(a0, sm);
    a1 = block_sum_ff(a1, sm);
    a2 = block_sum_ff(a2, sm);
    if (tid == 0) {
        wp[16] = a0.hi;
        wp[17] = a0.lo;
        wp[18] = a1.hi;
        wp[19] = a1.lo;
        wp[20] = a2.hi;
        wp[21] = a2.lo;
    }
    const float* net = f.ws_net;
    if (stage) {
        for (int i = tid; i < kWsParams; i += T) stage[i] = __ldg(f.ws_net + i);
        net = stage;  // visible to every thread after the barrier below
    }
    if (!tm.sync(epoch, &sm.flag)) return false;
    team_sum(f.wsPart, 32, tm.G, 22, sm.wsv);
    const double lam = lam_prev;
    double rho2 = sm.wsv[16] + sm.wsv[17];
    if (k > 0) {
        rho2 += -2.0 * lam * (sm.wsv[18] + sm.wsv[19]) + lam * lam * (sm.wsv[20] + sm.wsv[21]);
        const float lamf = (float)lam;
        for (int n = n0 + tid; n < n1; n += T) {
            const float u = f.U[(size_t)n * f.ldu + (k - 1)];
            float* x = f.wsF + (size_t)n * kWsIn;
            const float rv = f.upre[n] * vinv_prev;
            x[0] = fmaf(lamf * u, fmaf(lamf, u, -2.f * rv), x[0]);
#pragma unroll
            for (int j = 0; j < kWsSketch; ++j) x[1 + j] = fmaf(-lamf * (float)sm.wsv[j], u, x[1 + j]);
        }
        __syncthreads();
    }
    rho2 /= (double)f.N;
    const float invrho = rho2 > 0.0 ? (float)(1.0 / sqrt(rho2)) : 0.f;
    ff my = ff_zero();
    for (int n = n0 + warp; n < n1; n += nw) {
        const float* xr = f.wsF + (size_t)n * kWsIn;
        float x[kWsIn];
        x[0] = sqrtf(fmaxf(xr[0], 0.f)) * invrho;
#pragma unroll
        for (int j = 1; j < kWsIn; ++j) x[j] = xr[j] * invrho;
        const float w = ws_forward_warp(net, x, lane);
        if (lane == 0) {
            f.wsP0[n] = w;
            my = ff_add(my, ff_sqr(w));
        }
    }
    my = block_sum_ff(my, sm);
    if (tid == 0) {
        wp[22] = my.hi;
        wp[23] = my.lo;
    }
    // the staged parameters live in ring memory that TMA copies refill later
    if (stage) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!tm.sync(epoch, &sm.flag)) return false;
    team_sum(f.wsPart + 22, 32, tm.G, 2, sm.wsv + 22);
    *ww = sm.wsv[22] + sm.wsv[23];
    return true;
}

// The first pass of component k with both starts (learned candidate on):
// deflation of component k-1 as in row_pass<kPassCol>, the paper's start
// v_a = R(kcol) and the candidate v_b = R p0 (p0 = wsP0 / sqrt(ww)) row by row,
// and s_a = R^T v_a (-> pA), s_b = R^T v_b (-> pC) while the panel is in
// registers.  *sa / *sb receive ||v_a||^2 / ||v_b||^2 over the CTA's rows.
template <int CPT, class E>
__device__ __noinline__ void ws_start_pass(const FitArgs& f, SmemFit& sm, int g, int p0, int p1, int kcol,
                                           bool deflate, float lamf, int kprev, int buf, float inv_nu, double ww,
                                           float* pA, ff* sa, ff* sb) {
    // half the panels per round of the other passes where the loads are
    // software-pipelined (two rounds of cells in registers)
    constexpr bool PIPE = CPT <= 4;
    constexpr int PPR = PIPE ? (PassShape<CPT>::PPR > 1 ? PassShape<CPT>::PPR / 2 : 1) : PassShape<CPT>::PPR;
    constexpr int RPR = 4 * PPR;
    constexpr int SH = 5 - Log2<RPR>::value;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int T = blockDim.x, N = f.N;
    const size_t ldp = (size_t)f.ldp;
    const float pscale = (float)(1.0 / sqrt(ww));
    float uc[CPT], pc[CPT], acc_a[CPT], acc_b[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = tid + i * T;
        uc[i] = (deflate && c < N) ? ldcg(f.ut + (size_t)buf * N + c) * inv_nu : 0.f;
        pc[i] = c < N ? ldcg(f.wsP0 + c) * pscale : 0.f;
        acc_a[i] = acc_b[i] = 0.f;
    }
    int owner = -1;
    if ((kcol % T) == tid) owner = kcol / T;
    ff my_a = ff_zero(), my_b = ff_zero();
    int bsel = 0;
    // software pipeline (up to 2048 columns, where the registers allow it): the next
    // round's cells are loaded before this round is used
    float4 dn[PPR][CPT];
    auto load_round = [&](int pb, float4 (&dst)[PPR][CPT]) {
#pragma unroll
        for (int pp = 0; pp < PPR; ++pp) {
            const int p = pb + pp;
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T;
                dst[pp][i] = (p < p1 && c < N) ? Cell<E>::ldg(f.R, (size_t)p * ldp + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    if (PIPE && p0 < p1) load_round(p0, dn);
    for (int pb = p0; pb < p1; pb += PPR, bsel ^= 1) {
        float4 d[PPR][CPT];
        if constexpr (PIPE) {
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp)
#pragma unroll
                for (int i = 0; i < CPT; ++i) d[pp][i] = dn[pp][i];
            if (pb + PPR < p1) load_round(pb + PPR, dn);
        } else {
            load_round(pb, d);
        }
        if (deflate) {
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
                    v = Cell<E>::quant(v);
                    d[pp][i] = v;
                    if (p < p1 && c < N) Cell<E>::stg(f.R, (size_t)p * ldp + c, v);
                }
            }
        }
        // v_b rows: warp butterflies, then the warp partials through shared memory
        float acc[RPR];
#pragma unroll
        for (int r = 0; r < RPR; ++r) acc[r] = 0.f;
#pragma unroll
        for (int i = 0; i < CPT; ++i)
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                acc[pp * 4 + 0] = fmaf(d[pp][i].x, pc[i], acc[pp * 4 + 0]);
                acc[pp * 4 + 1] = fmaf(d[pp][i].y, pc[i], acc[pp * 4 + 1]);
                acc[pp * 4 + 2] = fmaf(d[pp][i].z, pc[i], acc[pp * 4 + 2]);
                acc[pp * 4 + 3] = fmaf(d[pp][i].w, pc[i], acc[pp * 4 + 3]);
            }
        const float r = warp_multi_reduce<RPR>(acc, lane);
        if ((lane & ((1 << SH) - 1)) == 0) sm.wsum[bsel][warp][lane >> SH] = r;
        // v_a rows: the owner of column kcol publishes them
        if (owner >= 0) {
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int i = 0; i < CPT; ++i)
                    if (i == owner) x = d[pp][i];
                sm.vrow[bsel][pp * 4 + 0] = x.x;
                sm.vrow[bsel][pp * 4 + 1] = x.y;
                sm.vrow[bsel][pp * 4 + 2] = x.z;
                sm.vrow[bsel][pp * 4 + 3] = x.w;
                my_a = ff_add(my_a, ff_sqr(x.x));
                my_a = ff_add(my_a, ff_sqr(x.y));
                my_a = ff_add(my_a, ff_sqr(x.z));
                my_a = ff_add(my_a, ff_sqr(x.w));
            }
        }
        __syncthreads();
        float rs = 0.f;
        if (lane < RPR)
            for (int w = 0; w < nw; ++w) rs += sm.wsum[bsel][w][lane];
        if (warp == 0 && lane < RPR && pb + (lane >> 2) < p1) my_b = ff_add(my_b, ff_sqr(rs));
        float ra[RPR], rb[RPR];
#pragma unroll
        for (int r2 = 0; r2 < RPR; ++r2) {
            rb[r2] = __shfl_sync(kFull, rs, r2);
            ra[r2] = sm.vrow[bsel][r2];
        }
#pragma unroll
        for (int i = 0; i < CPT; ++i)
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                const float4 v = d[pp][i];
                acc_a[i] = fmaf(v.x, ra[pp * 4 + 0], acc_a[i]);
                acc_a[i] = fmaf(v.y, ra[pp * 4 + 1], acc_a[i]);
                acc_a[i] = fmaf(v.z, ra[pp * 4 + 2], acc_a[i]);
                acc_a[i] = fmaf(v.w, ra[pp * 4 + 3], acc_a[i]);
                acc_b[i] = fmaf(v.x, rb[pp * 4 + 0], acc_b[i]);
                acc_b[i] = fmaf(v.y, rb[pp * 4 + 1], acc_b[i]);
                acc_b[i] = fmaf(v.z, rb[pp * 4 + 2], acc_b[i]);
                acc_b[i] = fmaf(v.w, rb[pp * 4 + 3], acc_b[i]);
            }
    }
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = tid + i * T;
        if (c < N) {
            pA[c] = acc_a[i];
            f.pC[(size_t)g * N + c] = acc_b[i];
        }
    }
    if (warp == 0) {
        const ff t = warp_sum_ff(my_b);
        if (lane == 0) sm.sff[3] = t;
    }
    if (owner >= 0) sm.ffg[0] = my_a;  // kcol < N: exactly one thread owns it
    __syncthreads();
    *sa = sm.ffg[0];
    *sb = sm.sff[3];
    __syncthreads();
}

// After the first pass with both starts (sm.sff[0] = ||v_a||^2, sm.sff[1] =
// ||v_b||^2 reduced; sv = this CTA's slice of s_a = R^T v_a): reduce this CTA's
// slice of s_b into sbv, form ||s_a||^2 and ||s_b||^2 over the team, and keep
// the start with the larger Rayleigh quotient ||s||^2 / ||v||^2: on return sv
// and sm.sff[0] describe the chosen start.  One team barrier; false if it failed.
template <class Team>
__device__ __noinline__ bool ws_select(const FitArgs& f, const Team& tm, SmemFit& sm, unsigned& epoch, int k,
                                       int n0, int nc1, float* sv, float* sbv) {
    const int tid = threadIdx.x, T = blockDim.x;
    const ff va2 = sm.sff[0], vb2 = sm.sff[1];
    gather_reduce(f, sm, tm.G, 0, 0, 0, f.pC, f.N, nc1, [&](int v) { return n0 + v; }, sbv);
    ff qa = ff_zero(), qb = ff_zero();
    for (int v = tid; v < nc1; v += T) {
        qa = ff_add(qa, ff_sqr(sv[v]));
        qb = ff_add(qb, ff_sqr(sbv[v]));
    }
    qa = block_sum_ff(qa, sm);
    qb = block_sum_ff(qb, sm);
    if (tid == 0) {
        float* wp = f.wsPart + (size_t)tm.g * 32;
        wp[24] = qa.hi;
        wp[25] = qa.lo;
        wp[26] = qb.hi;
        wp[27] = qb.lo;
    }
    if (!tm.sync(epoch, &sm.flag)) return false;
    team_sum(f.wsPart + 24, 32, tm.G, 4, sm.wsv);
    if (tid == 0) {
        const double Sa = sm.wsv[0] + sm.wsv[1], Sb = sm.wsv[2] + sm.wsv[3];
        const double na = ff_to_double(va2), nb = ff_to_double(vb2);
        sm.sel = (na > 0.0 && nb > 0.0 && Sb / nb > Sa / na) ? 1 : 0;
    }
    __syncthreads();
    const int use = sm.sel;
    if (use)
        for (int v = tid; v < nc1; v += T) sv[v] = sbv[v];
    if (tid == 0) sm.sff[0] = use ? vb2 : va2;
    if (tm.g == 0 && tid == 0 && f.ws_choice) f.ws_choice[k] = use;
    __syncthreads();
    return true;
}

// The first pass of a component (and of the zero-column restart): the optional
// deflation of component kprev (Eq. 3), R <- R - (lamf V(:, kprev)) u^T with u =
// u_in * inv_nu, stored as it goes; the start column R(:, kcol) after it, row by
// row; s = R^T R(:, kcol) (-> pA) while each panel is in registers, and *sc =
// ||R(:, kcol)||^2 over this CTA's rows.  No CTA barrier per round: every
// thread reads the start column's cells itself (the same address in every lane)
// and deflates them exactly as their owner does, and the owner stores column
// kcol only after the last round, so no thread ever reads an already deflated
// cell of it.  Register loads; warps stream their panels independently.
template <int CPT, class E>
__device__ __forceinline__ void pass_start_col(const FitArgs& f, SmemFit& sm, int p0, int p1, int kcol, bool deflate,
                                            float lamf, int kprev, const float* u_in, float inv_nu, float* pA,
                                            ff* sc) {
    constexpr int PPR = PassShape<CPT>::PPR;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = blockDim.x, N = f.N;
    const size_t ldp = (size_t)f.ldp;
    float uc[CPT], sacc[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = tid + i * T;
        uc[i] = (deflate && c < N) ? ldcg(u_in + c) * inv_nu : 0.f;
        sacc[i] = 0.f;
    }
    const float uk = deflate ? ldcg(u_in + kcol) * inv_nu : 0.f;
    ff my = ff_zero();
    for (int pb = p0; pb < p1; pb += PPR) {
        float4 d[PPR][CPT], dk[PPR];
#pragma unroll
        for (int pp = 0; pp < PPR; ++pp) {
            const int p = pb + pp;
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T;
                d[pp][i] = (p < p1 && c < N) ? Cell<E>::ldg(f.R, (size_t)p * ldp + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            dk[pp] = p < p1 ? Cell<E>::ldg(f.R, (size_t)p * ldp + kcol) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (deflate) {
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
                    v = Cell<E>::quant(v);
                    d[pp][i] = v;
                    if (p < p1 && c < N && c != kcol) Cell<E>::stg(f.R, (size_t)p * ldp + c, v);
                }
                float4 v = dk[pp];
                v.x = fmaf(-cf[0], uk, v.x);
                v.y = fmaf(-cf[1], uk, v.y);
                v.z = fmaf(-cf[2], uk, v.z);
                v.w = fmaf(-cf[3], uk, v.w);
                dk[pp] = Cell<E>::quant(v);
            }
        }
        if (tid == 0)
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                my = ff_add(my, ff_sqr(dk[pp].x));
                my = ff_add(my, ff_sqr(dk[pp].y));
                my = ff_add(my, ff_sqr(dk[pp].z));
                my = ff_add(my, ff_sqr(dk[pp].w));
            }
#pragma unroll
        for (int i = 0; i < CPT; ++i)
#pragma unroll
            for (int pp = 0; pp < PPR; ++pp) {
                const float4 v = d[pp][i];
                sacc[i] = fmaf(v.x, dk[pp].x, sacc[i]);
                sacc[i] = fmaf(v.y, dk[pp].y, sacc[i]);
                sacc[i] = fmaf(v.z, dk[pp].z, sacc[i]);
                sacc[i] = fmaf(v.w, dk[pp].w, sacc[i]);
            }
    }
    if (tid == 0) sm.sff[3] = my;
    __syncthreads();  // every thread has read column kcol's cells
    if (deflate && warp == 0) {
        // column kcol, deflated as every thread deflated it above
        for (int p = p0 + lane; p < p1; p += 32) {
            float4 v = Cell<E>::ldg(f.R, (size_t)p * ldp + kcol);
            float cf[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = 4 * p + q;
                cf[q] = row < f.M ? lamf * f.V[(size_t)row * f.ldv + kprev] : 0.f;
            }
            v.x = fmaf(-cf[0], uk, v.x);
            v.y = fmaf(-cf[1], uk, v.y);
            v.z = fmaf(-cf[2], uk, v.z);
            v.w = fmaf(-cf[3], uk, v.w);
            Cell<E>::stg(f.R, (size_t)p * ldp + kcol, Cell<E>::quant(v));
        }
    }
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = tid + i * T;
        if (c < N) pA[c] = sacc[i];
    }
    *sc = sm.sff[3];
    __syncthreads();
}

// (Re)initialise this CTA's ring: S stages of ppr panels of panel_bytes each.
// Must be called with no copy in flight.
__device__ __forceinline__ void ring_setup(Ring& rg, SmemFit& sm, unsigned char* dyn_smem, int S, int ppr,
                                          int panel_bytes) {
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < sm.mbar_live; ++s)
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&sm.mbar[s])) : "memory");
        for (int s = 0; s < S; ++s) mbar_init(reinterpret_cast<uint64_t*>(&sm.mbar[s]), 1);
        sm.mbar_live = S;
        fence_mbar_init();
    }
    __syncthreads();
    rg.S = S;
    rg.stage_bytes = ppr * panel_bytes;
    rg.base = dyn_smem;
    rg.mbar = sm.mbar;
    rg.issued = rg.used = 0;
}

// Second classical Gram-Schmidt pass (the CG2 kernel instantiations) of the
// vector x (global memory, entries a0 .. a1-1 owned by this CTA) against the
// k factor columns A (this CTA's rows a0 .. a1-1, leading dimension lda):
// partials A^T x -> partB[g][off, off + k), a team barrier, the reduced
// coefficients -> kx (shared memory), then x <- x - A kx.  Returns in *sq the
// CTA's sum of the new x^2 (every thread), false if a barrier failed.
template <class Team>
__device__ __noinline__ bool cgs_second_pass(const FitArgs& f, const Team& tm, SmemFit& sm, unsigned& epoch,
                                             const float* A, int lda, int a0, int a1, int k, float* x, int off,
                                             bool small_k, float* kx, ff* sq) {
    const int tid = threadIdx.x, T = blockDim.x;
    __syncthreads();
    rows_times_matrix<true>(A, lda, a0, a1, k, [&](int r) { return ldcg(x + r); }, f.partB + (size_t)tm.g * f.LB + off, sm);
    if (!tm.sync(epoch, &sm.flag)) return false;
    if (small_k) {
        gather_reduce(f, sm, tm.G, 0, 0, 0, f.partB + off, f.LB, k, [](int v) { return v; }, kx);
    } else {
        reduce_cols_distributed(f.partB, tm.G, tm.g, f.LB, off, k, f.red);
        if (!tm.sync(epoch, &sm.flag)) return false;
        for (int j = tid; j < k; j += T) kx[j] = (float)ldcg(f.red + j);
        __syncthreads();
    }
    ff q = ff_zero();
    matrix_times_vector<true>(
        A, lda, a0, a1, k, kx, [&](int r) { return ldcg(x + r); },
        [&](int r, float s, float p) {
            const float v = p - s;
            x[r] = v;
            q = ff_add(q, ff_sqr(v));
        });
    *sq = block_sum_ff(q, sm);
    return true;
}

// Which first pass a team uses: the barrier-free one (pass_start_col) in the
// single-problem kernel; the batched kernel keeps row_pass<kPassCol>, whose
// register needs fit its larger state without spills.
template <class Team>
constexpr bool kStartColPass = false;
template <>
constexpr bool kStartColPass<TeamGrid> = true;

// The two-reduction GS step (FitArgs::gs2) exists in the single-problem kernel,
// up to 4096 columns per CTA, without the learned warm start.
template <int CPT, class E, bool WARM, class Team>
constexpr bool kGs2Step = kStartColPass<Team> && !WARM && CPT <= 8;

// Fit one problem (f) with a team of CTAs.  The caller provides the
// degenerate threshold and this CTA's shared memory; the ring must be set up
// for f.N.  Writes V, U, W and lambda/iters for k < found; returns the
// outcome (identical in every CTA of the team).
// CG2 (single-problem kernels only): GS-PCA takes two classical Gram-Schmidt
// passes per half-iteration (CGS2, the iterated form Sec. 2.3 mentions), the
// second pass's coefficients from the vector the first pass left, with one
// more grid-wide reduction per half-iteration; the two-reduction step is off.
// A compile-time variant, so the one-pass kernels carry none of its code.
// WIDE: the factor products take their wide forms past 128 components (the
// kernel variant chosen for K > 128).
// bfloat16 storage, two-reduction GS step: this CTA's rows of Q = R_k U_(k)
// recomputed from the stored residual after each deflation (the rank-1 update
// the FP32 path uses does not see the bfloat16 rounding of the deflation, and
// c' = Q^T v' multiplies that error by the whole v').  Panels go in rounds of up
// to 32; in a round thread t takes panel t / np2 and the columns 2 (t % np2), +1
// (np2 = ceil(k / 2), k <= 64) and sums n = 0 .. N-1 in order in FP32.  U (16
// rows x 64) and the round's cells of R (16 columns per panel) reach shared
// memory (sm.tmpf) chunk by chunk, the next chunk held in registers meanwhile,
// so no thread waits on L2 inside a chunk.
template <class E>
__device__ __forceinline__ void q_rows_from_residual(const FitArgs& f, SmemFit& sm, float* Ql, int p0, int p1,
                                                     int k) {
    constexpr int NC = 16, PRMAX = 32;
    constexpr int PER = NC * 64 / kBlock;  // staged U values per thread and chunk
    const int tid = threadIdx.x, N = f.N;
    const int np2 = (k + 1) >> 1;
    const int pr = min(PRMAX, kBlock / np2);
    float* us = &sm.tmpf[0][0];                                       // NC x 64 floats
    uint2* rs = reinterpret_cast<uint2*>(&sm.tmpf[0][0] + NC * 64);  // pr x NC cells
    const uint2* R = static_cast<const uint2*>(f.R);
    const int nchunks = (N + NC - 1) / NC;
    for (int pa = p0; pa < p1; pa += pr) {
        const int pn = min(pr, p1 - pa);
        const bool live = tid < pn * np2;
        const int pl = live ? tid / np2 : 0;
        const int i0 = live ? 2 * (tid % np2) : 0;
        float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
        float nx[PER];
        uint2 nr;
        auto fetch = [&](int c) {
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int e = tid + j * kBlock, n = c * NC + (e >> 6), i = e & 63;
                nx[j] = (c < nchunks && n < N && i < k) ? ldcg(f.U + (size_t)n * f.ldu + i) : 0.f;
            }
            const int pp = tid / NC, n = c * NC + tid % NC;
            nr = (c < nchunks && pp < pn && n < N) ? ldcg(R + (size_t)(pa + pp) * f.ldp + n) : make_uint2(0u, 0u);
        };
        auto put = [&]() {
#pragma unroll
            for (int j = 0; j < PER; ++j) us[tid + j * kBlock] = nx[j];
            if (tid < pn * NC) rs[tid] = nr;
        };
        fetch(0);
        __syncthreads();
        put();
        fetch(1);
        __syncthreads();
        for (int c = 0; c < nchunks; ++c) {
            const int nn = min(NC, N - c * NC);
            if (live) {
                const uint2* rp = rs + pl * NC;
#pragma unroll 4
                for (int n = 0; n < nn; ++n) {
                    const float4 x = bf_unpack(rp[n]);
                    const float2 uu = *reinterpret_cast<const float2*>(us + n * 64 + i0);
                    a0[0] = fmaf(x.x, uu.x, a0[0]);
                    a1[0] = fmaf(x.x, uu.y, a1[0]);
                    a0[1] = fmaf(x.y, uu.x, a0[1]);
                    a1[1] = fmaf(x.y, uu.y, a1[1]);
                    a0[2] = fmaf(x.z, uu.x, a0[2]);
                    a1[2] = fmaf(x.z, uu.y, a1[2]);
                    a0[3] = fmaf(x.w, uu.x, a0[3]);
                    a1[3] = fmaf(x.w, uu.y, a1[3]);
                }
            }
            __syncthreads();
            put();
            fetch(c + 2);
            __syncthreads();
        }
        if (live)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float* row = Ql + (size_t)(4 * (pa + pl) + q) * f.ldv;
                row[i0] = a0[q];
                if (i0 + 1 < k) row[i0 + 1] = a1[q];
            }
    }
}

template <int CPT, class E, bool WARM, class Team, bool CG2 = false, bool WIDE = false>
__device__ FitOutcome fit_one(const FitArgs& f, const Team& tm, SmemFit& sm, unsigned char* dyn_smem, Ring& rg,
                              float threshf, unsigned& epoch) {
    constexpr int PPR = PassShape<CPT>::PPR;
    constexpr bool kWide = WIDE;
    const int G = tm.G, g = tm.g, tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int N = f.N, K = f.K;
    const int p0 = (int)(((long long)g * f.np) / G), p1 = (int)(((long long)(g + 1) * f.np) / G);
    const int r0 = min(p0 * 4, f.M), r1 = min(p1 * 4, f.M);
    const int n0 = (int)(((long long)g * N) / G), n1 = (int)(((long long)(g + 1) * N) / G);
    const bool gs = (f.algo == 1);
    float* pA = f.partA + (size_t)g * f.LA;
    float* pB = f.partB + (size_t)g * f.LB;
    const bool two = f.dot_groups == 2;
    const int ring_ppr = two ? 1 : PPR;
    // reduced pass partials: this CTA's N-slice, then the k-vector (b' or the Gram row)
    float* rb = reinterpret_cast<float*>(dyn_smem + f.ring_bytes);
    // with the two-reduction step rb also holds c' after b', and 3 ldk floats follow ka
    const bool gs2 = kGs2Step<CPT, E, WARM, Team> && !CG2 && f.gs2 != 0;
    const bool cgs2 = CG2 && f.algo == 1;  // a second classical pass on each half-iteration
    float* ka = rb + f.max_slice + (gs2 ? 2 : 1) * f.ldk;
    float* kx3 = ka + f.ldk;
    const int nc1 = n1 - n0;
    float* sv = rb;
    float* kb = rb + nc1;
    auto slice_then_k = [&](int v) { return v < nc1 ? n0 + v : N + (v - nc1); };
    auto ident = [](int v) { return v; };
    const float tolf = (float)f.tol;
    (void)warp;
    (void)lane;
    // This CTA's rows of V and slices of U and W: in shared memory when resident
    // (V and U are also written to global memory when a component finishes).
    float* Vl = f.V;
    float* Ul = f.U;
    float* Wl = f.W;
    // Two-reduction GS step (f.gs2): this CTA's rows of Q and the matrices Z and
    // GV = V^T V, column-major with leading dimension ldk (element (i, j) at j ldk + i).
    float* Ql = nullptr;
    float* Zs = nullptr;
    float* GVs = nullptr;
    if (f.res_rows > 0) {
        float* rbase = reinterpret_cast<float*>(dyn_smem + f.res_off);
        const int nres = f.res_rows * f.ldv + f.max_slice * (f.ldu + f.ldw) +
                         (gs2 ? f.res_rows * f.ldv + 2 * f.ldk * f.ldk : 0);
        for (int i = tid; i < nres; i += T) rbase[i] = 0.f;
        Vl = rbase - (size_t)r0 * f.ldv;
        Ul = rbase + (size_t)f.res_rows * f.ldv - (size_t)n0 * f.ldu;
        Wl = rbase + (size_t)f.res_rows * f.ldv + (size_t)f.max_slice * f.ldu - (size_t)n0 * f.ldw;
        if (gs2) {
            float* qbase = rbase + (size_t)f.res_rows * f.ldv + (size_t)f.max_slice * (f.ldu + f.ldw);
            Ql = qbase - (size_t)r0 * f.ldv;
            Zs = qbase + (size_t)f.res_rows * f.ldv;
            GVs = Zs + (size_t)f.ldk * f.ldk;
        }
        __syncthreads();
    }
    double lam0 = 0.0;  // lambda of component 0 (the two-reduction step's range guard)
    // WIDE: ||X||_F for the bounds of the fixed-point sums; the accumulators start at zero
    // (this CTA's share; the first barrier orders the stores before any use)
    const float xnorm = WIDE ? (float)sqrt(sm.dsc[0]) : 0.f;
    if constexpr (WIDE)
        for (int i = g * T + tid; i < 2 * f.ldk; i += G * T) f.facc[i] = 0;

    int status = kStOK, found = K;
    long long total = 0;
    double lam_prev = 0.0;  // lambda of the last finished component
    float vinv_prev = 0.f;  // 1/||v' - V b'|| of its last pass (GS)
    float inv_nu = 0.f;     // 1/||ut[buf]||
    int buf = 0;
    float uc[CPT], sacc[CPT];
    ff sc;
    bool alive = true;

#define GS_SYNC()                         \
    do {                                  \
        if (!tm.sync(epoch, &sm.flag)) {  \
            alive = false;                \
            goto leave;                   \
        }                                 \
    } while (0)

    for (int k = 0; k < K && found == K; ++k) {
        // ------------- start: deflate component k-1 inside the pass that takes R(k)
        __syncthreads();
        PHASE_MARK(0);
        if (gs2 && k > 1)  // a' of component k-1's last iteration: Z(i, k-1) before its h term
            for (int i = tid; i < k - 1; i += T) Zs[(size_t)(k - 1) * f.ldk + i] = vinv_prev * ka[i];
        const bool defl = k > 0;
        const float lamf = gs ? (float)lam_prev : 1.f;
        // learned warm start (the WARM instantiations only): features, network output, and a
        // first pass with both starts
        const bool wsk = WARM && gs && f.ws_net != nullptr;
        bool cand = false;
        if constexpr (WARM) if (wsk) {
            PHASE_MARK(5);
            if (k == 0 && !ws_sketch_init<E>(f, tm, sm, epoch, p0, p1, n0, n1)) {
                alive = false;
                goto leave;
            }
            double ww = 0.0;
            float* stage = f.ring_bytes >= kWsParams * (int)sizeof(float) ? reinterpret_cast<float*>(dyn_smem)
                                                                          : nullptr;
            if (!ws_prepare(f, tm, sm, epoch, k, r0, r1, n0, n1, lam_prev, vinv_prev, stage, &ww)) {
                alive = false;
                goto leave;
            }
            cand = ww > 0.0 && isfinite(ww);
            PHASE_MARK(9);
            if (cand) {
                ff sa, sb;
                ws_start_pass<CPT, E>(f, sm, g, p0, p1, k, defl, lamf, k - 1, buf, inv_nu, ww, pA, &sa, &sb);
                write_scalar(f, g, 0, sa);
                write_scalar(f, g, 1, sb);
            }
            PHASE_MARK(12);
        }
        if (!cand) {
            if constexpr (kStartColPass<Team>) {
                pass_start_col<CPT, E>(f, sm, p0, p1, k, defl, lamf, k - 1, f.ut + (size_t)buf * N, inv_nu, pA,
                                       &sc);
            } else {
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int c = tid + i * T;
                    uc[i] = (defl && c < N) ? ldcg(f.ut + (size_t)buf * N + c) * inv_nu : 0.f;
                }
                if (!row_pass<CPT, kPassCol, E>(f, sm, rg, p0, p1, uc, k, defl, lamf, k - 1, sacc, sc)) {
                    if (tm.fail(f)) {
                        alive = false;
                        goto leave;
                    }
                    sc = ff{__int_as_float(0x7fc00000), 0.f};
                }
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int c = tid + i * T;
                    if (c < N) pA[c] = sacc[i];
                }
            }
            write_scalar(f, g, 0, sc);
        }
        if (gs && k > 0)  // Gram row (V^T v_{k-1})_j over this CTA's rows
            rows_times_matrix<kWide>(Vl, f.ldv, r0, r1, k, [&](int r) { return Vl[(size_t)r * f.ldv + (k - 1)]; },
                              pA + N, sm);
        if (defl) fence_proxy_async_global();
        GS_SYNC();

        const bool small_k = k <= f.redundant_max;  // k-vectors reduced by every CTA
        const int nk0 = (gs && k > 0 && small_k) ? k : 0;
        gather_reduce(f, sm, G, cand ? 2 : 1, 0, 1, f.partA, f.LA, nc1 + nk0, slice_then_k, rb);
        if constexpr (WARM) {
            if (cand) {
                PHASE_MARK(13);
                if (!ws_select(f, tm, sm, epoch, k, n0, nc1, sv, ka + f.ldk)) {
                    alive = false;
                    goto leave;
                }
                PHASE_MARK(0);
            } else if (wsk && g == 0 && tid == 0 && f.ws_choice) {
                f.ws_choice[k] = 0;
            }
        }
        if (sm.sff[0].hi == 0.f && sm.sff[0].lo == 0.f) {
            // Zero start column: restart from the residual column of largest
            // norm (lowest index on ties); every column zero => rank exhausted.
            if (!row_pass<CPT, kPassSq, E>(f, sm, rg, p0, p1, uc, 0, false, 0.f, 0, sacc, sc) && tm.fail(f)) {
                alive = false;
                goto leave;
            }
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const int c = tid + i * T;
                if (c < N) pA[c] = sacc[i];
            }
            GS_SYNC();
            reduce_cols_distributed(f.partA, G, g, f.LA, 0, N, f.red);
            GS_SYNC();
            if (warp == 0) {
                double best = 0.0;
                int bi = N;
                for (int c = lane; c < N; c += 32) {
                    const double v = ldcg(f.red + c);
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
            pass_start_col<CPT, E>(f, sm, p0, p1, kcol, false, 0.f, 0, f.ut, 0.f, pA, &sc);
            write_scalar(f, g, 0, sc);
            GS_SYNC();
            gather_reduce(f, sm, G, 1, 0, 0, f.partA, f.LA, nc1 + nk0, slice_then_k, rb);
        }
        // ||x||^2 rescales the new loading so that its norm stays O(1).
        const float xx_inv = __fdiv_rn(1.f, __fadd_rn(sm.sff[0].hi, sm.sff[0].lo));
        const int nb = buf ^ 1;
        ff nq = ff_zero();
        if (gs && k > 0) {
            // Gram row -> kb; then W <- R_k^T V for the deflation of component k-1:
            // W(:, j) -= lambda u (v_{k-1}.v_j), new column R_{k-1}^T v_{k-1} - lambda u |v_{k-1}|^2
            if (!small_k) {
                reduce_cols_distributed(f.partA, G, g, f.LA, N, k, f.red);
                GS_SYNC();
                for (int j = tid; j < k; j += T) kb[j] = (float)ldcg(f.red + j);
                __syncthreads();
            }
            if (gs2) {
                // this CTA's slice of U_(k)^T u_{k-1} (h, ending with u_{k-1}.u_{k-1}),
                // W^T u_{k-1} (r) and u_{k-1}.u_pre (s1) of component k-1's last iteration,
                // taken before W and u_pre change: pB[k, 3k)
                const int km = k - 1;
                auto uk = [&](int n) { return Ul[(size_t)n * f.ldu + km]; };
                // (W's column k-1, not yet formed, lands in pB[3k-1] and is replaced by s1)
                rows_times_two(Ul, Wl, f.ldu, n0, n1, k, uk, pB + k, pB + 2 * k, sm);
                ff su = ff_zero();
                for (int n = n0 + tid; n < n1; n += T) su = ff_add(su, ff_mul_ff(uk(n), ldcg(f.upre + n)));
                su = block_sum_ff(su, sm);
                if (tid == 0) pB[3 * k - 1] = __fadd_rn(su.hi, su.lo);
            }
            {
                const int km = k - 1;
                const float lpf = (float)lam_prev;
                for (int e = tid; e < (n1 - n0) * k; e += T) {
                    const int n = n0 + e / k, jj = e % k;
                    const float un = Ul[(size_t)n * f.ldu + km];
                    float* w = Wl + (size_t)n * f.ldw + jj;
                    if (jj < km)
                        *w = fmaf(-lpf * un, kb[jj], *w);
                    else
                        *w = (float)((double)f.upre[n] * (double)vinv_prev - lam_prev * (double)un * (double)kb[km]);
                }
            }
            __syncthreads();
            // u_pre = s0; a = U_(k)^T u_pre; ut = (u_pre - U a) / ||x||^2
            for (int n = n0 + tid; n < n1; n += T) f.upre[n] = sv[n - n0];
            __syncthreads();
            rows_times_matrix<kWide>(Ul, f.ldu, n0, n1, k, [&](int n) { return sv[n - n0]; }, pB, sm);
            GS_SYNC();
            if (small_k && gs2) {
                gather_reduce<4>(f, sm, G, 0, 0, 0, f.partB, f.LB, 3 * k, ident, kx3);
                for (int j = tid; j < k; j += T) ka[j] = kx3[j];
                // Keep Z = U^T W, GV = V^T V and Q = R_k U_(k) for the deflation of component
                // k-1 (the same rank-1 algebra as W): kb holds the Gram row v_{k-1}.v_j
                const int km = k - 1;
                const float lpf = (float)lam_prev;
                const float* h = kx3 + k;
                const float* rr = kx3 + 2 * k;
                const float s1 = kx3[3 * k - 1], s2 = kx3[k + km];
                for (int e = tid; e < k * k; e += T) {
                    const int i = e / k, j = e % k;
                    float* z = Zs + (size_t)j * f.ldk + i;
                    if (i < km && j < km)
                        *z = fmaf(-lpf * h[i], kb[j], *z);
                    else if (i < km)  // j = k-1: vinv a'_i was stored at the start
                        *z = fmaf(-lpf * h[i], kb[km], *z);
                    else if (j < km)  // i = k-1
                        *z = fmaf(-lpf * s2, kb[j], rr[j]);
                    else
                        *z = fmaf(-lpf * s2, kb[km], vinv_prev * s1);
                    if (i == km || j == km) GVs[(size_t)j * f.ldk + i] = kb[i == km ? j : i];
                }
                if constexpr (Cell<E>::kBytes == 8) {
                    q_rows_from_residual<E>(f, sm, Ql, p0, p1, k);
                } else {
                    for (int e = tid; e < (r1 - r0) * k; e += T) {
                        const int r = r0 + e / k, i = e % k;
                        const float vk = lpf * Vl[(size_t)r * f.ldv + km];
                        float* q = Ql + (size_t)r * f.ldv + i;
                        *q = (i < km) ? fmaf(-vk, h[i], *q) : fmaf(-vk, s2, ldcg(f.vraw + r) * inv_nu);
                    }
                }
                __syncthreads();
            } else if (small_k) {
                gather_reduce(f, sm, G, 0, 0, 0, f.partB, f.LB, k, ident, ka);
            } else {
                reduce_cols_distributed(f.partB, G, g, f.LB, 0, k, f.red);
                GS_SYNC();
                for (int j = tid; j < k; j += T) ka[j] = (float)ldcg(f.red + j);
                __syncthreads();
            }
            matrix_times_vector<kWide>(
                Ul, f.ldu, n0, n1, k, ka, [&](int n) { return sv[n - n0]; },
                [&](int n, float s, float p) {
                    const float un = (p - s) * xx_inv;
                    f.ut[(size_t)nb * N + n] = un;
                    nq = ff_add(nq, ff_sqr(un));
                });
            if constexpr (CG2) {  // second pass on the first loading: a2 = U_(k)^T ut -> pB[ldk, 2 ldk)
                ff q;
                if (!cgs_second_pass(f, tm, sm, epoch, Ul, f.ldu, n0, n1, k, f.ut + (size_t)nb * N, f.ldk, small_k,
                                     ka, &q)) {
                    alive = false;
                    goto leave;
                }
                nq = tid == 0 ? q : ff_zero();
            }
        } else {
            for (int n = n0 + tid; n < n1; n += T) {
                const float un = sv[n - n0] * xx_inv;
                f.ut[(size_t)nb * N + n] = un;
                nq = ff_add(nq, ff_sqr(un));
            }
        }
        nq = block_sum_ff(nq, sm);
        write_scalar(f, g, 2 + nb, nq);
        buf = nb;
        ring_prefetch<E>(f, rg, p0, p1, ring_ppr);
        GS_SYNC();

        // ------------- power iterations
        ff mu = ff_zero();
        int j = 0;
        for (;;) {
            PHASE_MARK(1);
            bool pass_ok = true, two_done = false;
            if constexpr (CPT <= 2) {
                if (f.narrow) {
                    PHASE_MARK(2);
                    pass_ok = pass_narrow<CPT, E>(f, sm, p0, p1, f.ut + (size_t)buf * N, pA, sc, dyn_smem);
                    two_done = true;
                }
            }
            if constexpr (CPT <= 4) {
                if (two && !two_done) {
                    float uc2[2 * CPT], sacc2[2 * CPT];
#pragma unroll
                    for (int i = 0; i < 2 * CPT; ++i) {
                        const int c = (tid & 255) + i * 256;
                        uc2[i] = (c < N) ? ldcg(f.ut + (size_t)buf * N + c) : 0.f;
                    }
                    PHASE_MARK(2);
                    pass_ok = pass_dot2<CPT, E>(f, sm, rg, p0, p1, uc2, sacc2, sc);
                    if (tid < 256)
#pragma unroll
                        for (int i = 0; i < 2 * CPT; ++i) {
                            const int c = tid + i * 256;
                            if (c < N) pA[c] = sacc2[i];
                        }
                    two_done = true;
                }
            }
            bool packed = false;
            if constexpr (Cell<E>::kBytes == 8 && kStartColPass<Team> && CPT <= 8) {
                if (!two_done && rg.S == 0) {
                    PHASE_MARK(2);
                    pass_dot_reg_bf16<CPT>(f, sm, p0, p1, f.ut + (size_t)buf * N, pA, &sc);
                    packed = true;
                }
            }
            if (!two_done && !packed) {
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int c = tid + i * T;
                    uc[i] = (c < N) ? ldcg(f.ut + (size_t)buf * N + c) : 0.f;
                }
                PHASE_MARK(2);
                pass_ok = row_pass<CPT, kPassDot, E>(f, sm, rg, p0, p1, uc, 0, false, 0.f, 0, sacc, sc);
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int c = tid + i * T;
                    if (c < N) pA[c] = sacc[i];
                }
            }
            if (!pass_ok) {
                if (tm.fail(f)) {
                    alive = false;
                    goto leave;
                }
                sc = ff{__int_as_float(0x7fc00000), 0.f};
            }
            write_scalar(f, g, 0, sc);
            // The two-reduction step is tried once the spectrum seen so far spans at most 64x
            // (lambda_0 <= 64 mu): there Q and Z track R_k U and U^T W to the accuracy of the
            // direct products.  Every CTA decides alike from the same reduced values.
            const bool try2 = gs2 && gs && k > 0 && mu.hi > 0.f && (float)lam0 <= 64.f * mu.hi;
            // WIDE past 128 components: b' and a' through the fixed-point accumulators
            const bool fxk = WIDE && gs && k > f.redundant_max;
            int fx_b = 0, fx_a = 0;  // scale exponents S of the b' and a' sums
            if (try2) {  // b' = V_(k)^T v' and c' = Q^T v' = U^T s' over this CTA's rows
                rows_times_two(Vl, Ql, f.ldv, r0, r1, k, [&](int r) { return f.vraw[r]; }, pA + N, pA + N + k, sm);
            } else if (fxk) {
                // |b'_j| over any rows <= ||v'|| <= ||R||_F ||u'|| <= ||X||_F ||u'||: ||u'||^2 from the
                // CTA partials of the last loading (every CTA alike), a factor 4 to spare
                if (warp == 0) {
                    ff a = ff_zero();
                    for (int i = lane; i < G; i += 32) {
                        const float2 q = ldcg(f.spart + (size_t)i * 4 + 2 + buf);
                        a = ff_add(a, ff{q.x, q.y});
                    }
                    a = warp_sum_ff(a);
                    if (lane == 0) sm.tmpf[0][0] = __fadd_rn(a.hi, a.lo);
                }
                // a' of the last iteration was read before the last barrier: clear its accumulators
                for (int i = g * T + tid; i < k; i += G * T) f.facc[f.ldk + i] = 0;
                __syncthreads();
                fx_b = fx_shift(4.f * xnorm, sqrtf(fmaxf(sm.tmpf[0][0], 0.f)), G);
                rows_times_matrix_wide_out(Vl, f.ldv, r0, r1, k, [&](int r) { return f.vraw[r]; },
                                           [&](int jj, float s) { fx_add(f.facc + jj, s, fx_b, G); });
            } else if (gs && k > 0) {  // b' = V_(k)^T v' over this CTA's rows
                rows_times_matrix<kWide>(Vl, f.ldv, r0, r1, k, [&](int r) { return f.vraw[r]; }, pA + N, sm);
            }
            PHASE_MARK(3);
            GS_SYNC();
            PHASE_MARK(4);
            ++j;
            ++total;
            const bool small_k = k <= f.redundant_max;
            // sff[0] = ||u'||^2 (pass input), sff[1] = ||v'||^2; this CTA's slice of s' (+ b')
            if (try2)  // the slice, b' and c': up to 128 values per round trip
                gather_reduce<4>(f, sm, G, 2, 2 + buf, 0, f.partA, f.LA, nc1 + 2 * k, slice_then_k, rb);
            else
                gather_reduce(f, sm, G, 2, 2 + buf, 0, f.partA, f.LA, nc1 + ((gs && k > 0 && small_k) ? k : 0),
                              slice_then_k, rb);
            const ff nu2 = sm.sff[0];
            const ff nvp = sm.sff[1];
            const float nu2f = __fadd_rn(nu2.hi, nu2.lo);
            if (!(nu2f > 0.f)) {
                found = k;
                status = kStDegenerate;
                break;
            }
            inv_nu = __fdiv_rn(1.f, __fsqrt_rn(nu2f));
            ff lam2p;  // ||v' - V b'||^2 in pass scale
            const int nbuf = buf ^ 1;
            bool step2 = false;  // this iteration took the two-reduction GS step
            if (!gs || k == 0) {
                lam2p = nvp;
                PHASE_MARK(6);
            } else {
                // b' -> kb; v_corr' = v' - V b' (rows); u_pre' = s' - W b' (slice);
                // a' = U^T u_pre' (partials)
                if (fxk) {
                    for (int jj = tid; jj < k; jj += T) kb[jj] = fx_get(f.facc + jj, fx_b);
                    __syncthreads();
                } else if (!small_k) {
                    reduce_cols_distributed(f.partA, G, g, f.LA, N, k, f.red);
                    GS_SYNC();
                    for (int jj = tid; jj < k; jj += T) kb[jj] = (float)ldcg(f.red + jj);
                    __syncthreads();
                }
                PHASE_MARK(6);
                if (try2) {
                    // a' = U^T (s' - W b') = c' - Z b' and ||v' - V b'||^2 = ||v'||^2 - 2 b'.b' +
                    // b'^T (V^T V) b' from reduced values only (fixed order); taken when the
                    // subtraction loses little (b'.b' <= ||v'||^2 / 4).  Warp w sums the rows j
                    // of its chunk of V^T V and Z against b' for every column i (k <= 64), then
                    // warp 0 adds the 16 warp partials in warp order.
                    {
                        const int jc = (k + kMaxWarps - 1) / kMaxWarps;
                        const int ja = warp * jc, jb = min(k, ja + jc);
                        for (int i = lane; i < k; i += 32) {
                            float t = 0.f, z = 0.f;
                            for (int jj = ja; jj < jb; ++jj) {
                                const float b = kb[jj];
                                t = fmaf(GVs[(size_t)jj * f.ldk + i], b, t);
                                z = fmaf(Zs[(size_t)jj * f.ldk + i], b, z);
                            }
                            sm.tmpf[warp][i] = t;
                            sm.tmpf[warp][64 + i] = z;
                        }
                    }
                    __syncthreads();
                    if (warp == 0) {
                        const float* kc = kb + k;
                        ff bb = ff_zero(), bg = ff_zero();
                        for (int i = lane; i < k; i += 32) {
                            float t = 0.f, z = 0.f;
#pragma unroll
                            for (int w = 0; w < kMaxWarps; ++w) {
                                t += sm.tmpf[w][i];
                                z += sm.tmpf[w][64 + i];
                            }
                            ka[i] = kc[i] - z;
                            bb = ff_add(bb, ff_sqr(kb[i]));
                            bg = ff_add(bg, ff_mul_ff(kb[i], t));
                        }
                        bb = warp_sum_ff(bb);
                        bg = warp_sum_ff(bg);
                        if (lane == 0) {
                            sm.lam2s = ff_add(nvp, ff_add(bg, ff_neg(ff_add(bb, bb))));
                            sm.step2 = 4.f * (bb.hi + bb.lo) <= nvp.hi + nvp.lo;
                        }
                    }
                    __syncthreads();
                    step2 = sm.step2 != 0;
                }
                if (step2) {
                    lam2p = sm.lam2s;  // s' - W b' is formed with the next loading below
                } else {
                    ff l2 = ff_zero();
                    if constexpr (!CG2) {
                        matrix_times_vector<kWide>(
                            Vl, f.ldv, r0, r1, k, kb, [&](int r) { return ldcg(f.vraw + r); },
                            [&](int r, float s, float p) {
                                const float vc = p - s;
                                f.vcorr[r] = vc;
                                l2 = ff_add(l2, ff_sqr(vc));
                            });
                    } else {
                        // first pass v' - V b', then b2 = V^T (v' - V b') reduced across the grid and
                        // the second pass (pB[2 ldk, 3 ldk)); the loading side then uses b' + b2
                        matrix_times_vector<kWide>(
                            Vl, f.ldv, r0, r1, k, kb, [&](int r) { return ldcg(f.vraw + r); },
                            [&](int r, float s, float p) { f.vcorr[r] = p - s; });
                        ff q;
                        if (!cgs_second_pass(f, tm, sm, epoch, Vl, f.ldv, r0, r1, k, f.vcorr, 2 * f.ldk, small_k,
                                             ka, &q)) {
                            alive = false;
                            goto leave;
                        }
                        l2 = tid == 0 ? q : ff_zero();
                        for (int jj = tid; jj < k; jj += T) kb[jj] += ka[jj];
                        __syncthreads();
                    }
                    matrix_times_vector<kWide>(
                        Wl, f.ldw, n0, n1, k, kb, [&](int n) { return sv[n - n0]; },
                        [&](int n, float s, float p) { f.upre[n] = p - s; });
                    __syncthreads();
                    if (fxk) {
                        // |a'_j| over any slice <= ||u_pre'|| <= ||R||_F ||v' - V b'|| <= 2 ||X||_F ||v'||,
                        // a factor 4 to spare
                        fx_a = fx_shift(8.f * xnorm, sqrtf(fmaxf(__fadd_rn(nvp.hi, nvp.lo), 0.f)), G);
                        rows_times_matrix_wide_out(Ul, f.ldu, n0, n1, k, [&](int n) { return f.upre[n]; },
                                                   [&](int jj, float s) { fx_add(f.facc + f.ldk + jj, s, fx_a, G); });
                    } else {
                        rows_times_matrix<kWide>(Ul, f.ldu, n0, n1, k, [&](int n) { return f.upre[n]; }, pB, sm);
                    }
                    l2 = block_sum_ff(l2, sm);
                    write_scalar(f, g, 1, l2);
                    PHASE_MARK(7);
                    GS_SYNC();
                    PHASE_MARK(8);
                    gather_reduce(f, sm, G, 1, 1, 0, f.partB, f.LB, small_k ? k : 0, ident, ka);
                    lam2p = sm.sff[0];
                    if (fxk) {
                        for (int jj = tid; jj < k; jj += T) ka[jj] = fx_get(f.facc + f.ldk + jj, fx_a);
                        // every CTA read b' before this barrier: clear its accumulators (this CTA's share)
                        for (int i = g * T + tid; i < k; i += G * T) f.facc[i] = 0;
                        __syncthreads();
                    } else if (!small_k) {
                        reduce_cols_distributed(f.partB, G, g, f.LB, 0, k, f.red);
                        GS_SYNC();
                        for (int jj = tid; jj < k; jj += T) ka[jj] = (float)ldcg(f.red + jj);
                        __syncthreads();
                    }
                }
                PHASE_MARK(10);
            }
            // Thread 0: lambda = sqrt(lam2p / nu2) in FP64 and the test; the other
            // threads form the next loading speculatively meanwhile.
            if (tid == 0) {
                const ff lamff = ff_sqrt(ff_div(lam2p, nu2));
                int stop;
                if (!(lamff.hi > threshf)) {
                    stop = 2;
                } else if (f.iters_lock != nullptr) {
                    stop = j >= f.iters_lock[k];
                } else {
                    const ff d = ff_add(mu, ff_neg(lamff));
                    stop = fabsf(__fadd_rn(d.hi, d.lo)) < __fmul_rn(tolf, lamff.hi);
                    if (!stop && j >= f.max_iter) stop = 3;
                }
                sm.lamff = lamff;
                sm.stop = stop;
            }
            const float l2f = __fadd_rn(lam2p.hi, lam2p.lo);
            const float nscale = __fdiv_rn(__fsqrt_rn(nu2f), l2f);  // keeps ||ut|| ~ 1
            ff nq2 = ff_zero();
            if (!gs || k == 0) {
                for (int n = n0 + tid; n < n1; n += T) {
                    const float un = sv[n - n0] * nscale;
                    f.ut[(size_t)nbuf * N + n] = un;
                    nq2 = ff_add(nq2, ff_sqr(un));
                    if (gs) f.upre[n] = sv[n - n0];
                }
            } else if (step2) {
                // u_pre = s' - W b' and the next loading (u_pre - U a') nscale in one sweep
                matrix_times_two(
                    Wl, Ul, f.ldw, n0, n1, k, kb, ka, [&](int n) { return sv[n - n0]; },
                    [&](int n, float sw, float su, float s0) {
                        const float up = s0 - sw;
                        f.upre[n] = up;
                        const float un = (up - su) * nscale;
                        f.ut[(size_t)nbuf * N + n] = un;
                        nq2 = ff_add(nq2, ff_sqr(un));
                    });
            } else {
                matrix_times_vector<kWide>(
                    Ul, f.ldu, n0, n1, k, ka, [&](int n) { return ldcg(f.upre + n); },
                    [&](int n, float s, float p) {
                        const float un = (p - s) * nscale;
                        f.ut[(size_t)nbuf * N + n] = un;
                        nq2 = ff_add(nq2, ff_sqr(un));
                    });
            }
            nq2 = block_sum_ff(nq2, sm);  // its barriers also publish sm.stop / sm.lamff
            const int stop = sm.stop;
            const ff lamff = sm.lamff;
            if (stop == 2) {
                found = k;
                status = kStDegenerate;
                break;
            }
            if (stop) {
                if (stop == 3 && status == kStOK) status = kStNotConverged;
                // finalize component k: V(k), U(k), lambda_k, iters_k
                if (step2) {  // v' - V b' for this CTA's rows (the two-reduction step skipped it)
                    matrix_times_vector<kWide>(
                        Vl, f.ldv, r0, r1, k, kb, [&](int r) { return ldcg(f.vraw + r); },
                        [&](int r, float s, float p) { f.vcorr[r] = p - s; });
                    __syncthreads();
                }
                if (f.coef_trace != nullptr && gs && k > 0) {
                    float* tr = f.coef_trace + (size_t)k * (2 * K + f.M + N);
                    if (g == 0)
                        for (int i = tid; i < k; i += T) {
                            tr[i] = kb[i];
                            tr[K + i] = ka[i];
                        }
                    for (int r = r0 + tid; r < r1; r += T) tr[2 * K + r] = ldcg(f.vraw + r);
                    for (int n = n0 + tid; n < n1; n += T) tr[2 * K + f.M + n] = ldcg(f.upre + n);
                }
                const float vinv = __fdiv_rn(1.f, __fsqrt_rn(l2f));
                const bool res = f.res_rows > 0;
                for (int r = r0 + tid; r < r1; r += T) {
                    const float v = gs ? ((k > 0) ? f.vcorr[r] : f.vraw[r]) * vinv : f.vraw[r] * inv_nu;
                    f.V[(size_t)r * f.ldv + k] = v;
                    if (res) Vl[(size_t)r * f.ldv + k] = v;
                }
                for (int n = n0 + tid; n < n1; n += T) {
                    const float u = ldcg(f.ut + (size_t)buf * N + n) * inv_nu;
                    f.U[(size_t)n * f.ldu + k] = u;
                    if (res) Ul[(size_t)n * f.ldu + k] = u;
                }
                lam_prev = ff_to_double(lamff);
                if (k == 0) lam0 = lam_prev;
                if (g == 0 && tid == 0) {
                    f.lam[k] = lam_prev;
                    f.iters[k] = j;
                }
                vinv_prev = vinv;
                break;
            }
            if constexpr (CG2) {
                if (cgs2 && k > 0) {  // second pass on the next loading: a2 = U_(k)^T ut -> pB[ldk, 2 ldk)
                    if (!cgs_second_pass(f, tm, sm, epoch, Ul, f.ldu, n0, n1, k, f.ut + (size_t)nbuf * N, f.ldk,
                                         small_k, ka, &nq2)) {
                        alive = false;
                        goto leave;
                    }
                }
            }
            mu = lamff;
            write_scalar(f, g, 2 + nbuf, nq2);
            buf = nbuf;
            ring_prefetch<E>(f, rg, p0, p1, ring_ppr);
            PHASE_MARK(11);
            GS_SYNC();
        }
    }
#undef GS_SYNC
leave:
    if (!alive) ring_drain(f, rg);
    return FitOutcome{status, found, total, alive};
}

// ------------------------------------------------------------------ kernels

// Single problem, whole grid (cooperative launch).  CG2: two classical
// Gram-Schmidt passes per half-iteration; WIDE: factor products for more than
// 128 components (see fit_one).
template <int CPT, class E, bool WARM, bool CG2 = false, bool WIDE = false>
__global__ void __launch_bounds__(kBlock, 1) fit_kernel(const FitArgs f) {
    __shared__ SmemFit sm;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TeamGrid tm{(int)gridDim.x, (int)blockIdx.x, GridBarrier{f.flags, f.abort, f.timeout_ns}};
    if (tid == 0) sm.mbar_live = 0;
#ifdef GSPCA_PHASE_TIMING
    if (tid == 0) {
        for (int i = 0; i < 16; ++i) sm.tacc[i] = 0;
        sm.tlast = globaltimer_ns();
        sm.tcur = 0;
        sm.tmark = blockIdx.x == 0;
    }
#endif
    // ||X||_F^2 from the pack kernel's partials (fixed order, every CTA).
    if (warp == 0) {
        double t = 0.0;
        for (int i = lane; i < f.nxpart; i += 32) t += f.xpart[i];
        t = warp_sum(t);
        if (lane == 0) sm.dsc[0] = t;
    }
    __syncthreads();
    const float threshf = (float)(f.eps_thresh * sqrt(sm.dsc[0]));
    Ring rg;
    ring_setup(rg, sm, dyn_smem, f.tma_stages, f.dot_groups == 2 ? 1 : PassShape<CPT>::PPR,
               f.ldp * Cell<E>::kBytes);
    unsigned epoch = 0;
    const FitOutcome r = fit_one<CPT, E, WARM, TeamGrid, CG2, WIDE>(f, tm, sm, dyn_smem, rg, threshf, epoch);
#ifdef GSPCA_PHASE_TIMING
    PHASE_MARK(15);
    if (blockIdx.x == 0 && tid == 0 && f.timing)
        for (int i = 0; i < 16; ++i) f.timing[i] = sm.tacc[i];
#endif
    if (r.alive && blockIdx.x == 0 && tid == 0) {
        f.info[kInfoStatus] = r.status;
        f.info[kInfoFound] = r.found;
        f.info[kInfoItersLo] = (int)(r.total & 0x7fffffff);
        f.info[kInfoItersHi] = (int)(r.total >> 31);
    }
}

}  // namespace gspca
