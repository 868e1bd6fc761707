// Host-side helpers shared by the entry points: workspace layout, launch plan
// (grid size, TMA ring depth, shared memory) and the enqueue sequence
//   [centring means] -> pack -> persistent fit kernel -> epilogue [-> unpack]
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstddef>

#include "../../include/gspca.h"
#include "fit_kernel.cuh"
#include "prep_kernels.cuh"
#include "workspace.cuh"

namespace gspca {

constexpr int kMaxCols = 16 * kBlock;   // columns one CTA holds (CPT <= 16)
constexpr int kRedundantMax = 128;      // k up to which every CTA reduces a k-vector itself

struct Plan {
    int cpt, ppr, G, S, ldk, max_slice, groups;
    int res_rows;   // > 0: the factor rows and slices are kept in shared memory (see FitArgs)
    size_t res;     // their bytes
    int cb;     // bytes of one cell of R: 16 (FP32 storage) or 8 (bfloat16 storage)
    bool warm;  // the kernel with the learned warm start
    int gs2;    // GS-PCA iterations may take the two-reduction step (see FitArgs::gs2)
    int gs_passes;  // classical Gram-Schmidt passes per half-iteration: 2 selects the CGS2 kernels
    int svd_form;   // 1: the epilogue writes the unit score directions (gspca_opts::svd_form)
    int variant;    // kernel variant (fit_variant)
    size_t dyn;
};

// Largest resident factor block chosen automatically.
constexpr size_t kResMaxBytes = 48 * 1024;
// The two-reduction GS step: up to this many components, and a resident block
// (with Q rows and the matrices Z and V^T V) of at most this size.
constexpr int kGs2MaxK = 64;
constexpr size_t kResGs2MaxBytes = 96 * 1024;

// Shared memory after the ring: the CTA's slice of the pass result, two
// k-vectors, and the slice of the learned start's second pass result.  With the
// two-reduction GS step: the slice, b' and c' (max_slice + 2 ldk), a' (ldk) and
// the component-start products (3 ldk).
inline size_t vec_bytes(int ldk, int max_slice, int gs2) {
    return (sizeof(float) * ((gs2 ? 6 : 2) * (size_t)ldk + 2 * (size_t)max_slice) + 15) / 16 * 16;
}

// Bytes of one cell of R (4 rows x 1 column) for a storage type.
inline int cell_bytes(gspca_dtype dt) { return dt == GSPCA_BF16 ? 8 : 16; }

inline int cpt_for(int N) {
    int c = 1;
    while (c * kBlock < N) c *= 2;
    return c;
}

// Checks of the fields of gspca_opts shared by gspca_fit, gspca_fit_host and
// gspca_fit_noalloc (the warm-start pointer is checked by each entry point,
// since its support differs).  opts may be null.
inline gspca_status check_opts(const gspca_opts* opts, int K) {
    if (!opts) return GSPCA_OK;
    if (opts->center < 0 || opts->center > 2 || opts->grid_ctas < 0 || !(opts->timeout_s >= 0) ||
        opts->test_stall < 0 || opts->test_stall > 1 || opts->resident < 0 || opts->resident > 2 ||
        opts->load_path < 0 || opts->load_path > 2 || opts->gs_step < 0 || opts->gs_step > 1 ||
        opts->gs_passes < 0 || opts->gs_passes > 2 || opts->svd_form < 0 || opts->svd_form > 1)
        return GSPCA_ERR_INVALID_ARG;
    if (opts->iters_lock)
        for (int k = 0; k < K; ++k)
            if (opts->iters_lock[k] < 1) return GSPCA_ERR_INVALID_ARG;
    return GSPCA_OK;
}

// Kernel attributes and launches per (columns per thread, storage type).  They
// are defined beside the kernels (fit_inst.cuh) and instantiated once each in
// the fit_*.cu translation units, so the host-side units compile no kernel.
template <int CPT, class E, bool WARM, bool CG2, bool WIDE>
cudaError_t fit_attrs(size_t dyn, int* bps, int* static_smem);
template <int CPT, class E, bool WARM, bool CG2, bool WIDE>
cudaError_t launch_fit_t(const FitArgs& a, int G, size_t dyn, cudaStream_t s);

// The learned warm start is compiled into the fit kernels for up to this many
// columns per thread (2048 columns); wider problems fit without it.
constexpr int kWarmMaxCpt = 4;
template <class E>
void launch_pack(dim3 grid, cudaStream_t s, const float* X, int layout, long ldx, int M, int N, int np, int ldp,
                 int center, const double* cmean, const double* rmean, void* R, double* xpart, unsigned* flags,
                 int nflags, int* abort, int* info, int ninfo);
template <class E>
void launch_unpack(dim3 grid, cudaStream_t s, const void* R, int M, int N, int np, int ldp, const float* V, int ldv,
                   const float* U, int ldu, const double* lam, const int* info, int K, int gs, float* R_out);

// The kernel variant of a plan: 0 plain, 1 learned warm start, 2 CGS2 (wide
// products included), 3 wide products (more than 128 components).
inline int fit_variant(bool warm, bool cg2, bool wide) { return warm ? 1 : cg2 ? 2 : wide ? 3 : 0; }

template <class E, bool WARM, bool CG2, bool WIDE>
inline cudaError_t fit_attrs_v(int cpt, size_t dyn, int* bps, int* st) {
    switch (cpt) {
        case 1: return fit_attrs<1, E, WARM, CG2, WIDE>(dyn, bps, st);
        case 2: return fit_attrs<2, E, WARM, CG2, WIDE>(dyn, bps, st);
        case 4: return fit_attrs<4, E, WARM, CG2, WIDE>(dyn, bps, st);
        case 8: return fit_attrs<8, E, WARM, CG2, WIDE>(dyn, bps, st);
        default: return fit_attrs<16, E, WARM, CG2, WIDE>(dyn, bps, st);
    }
}

template <class E>
inline cudaError_t fit_attrs_e(int cpt, int variant, size_t dyn, int* bps, int* st) {
    switch (variant) {
        case 1:  // learned warm start: up to 4 columns per thread
            if (cpt > 4) return cudaErrorInvalidValue;
            switch (cpt) {
                case 1: return fit_attrs<1, E, true, false, false>(dyn, bps, st);
                case 2: return fit_attrs<2, E, true, false, false>(dyn, bps, st);
                default: return fit_attrs<4, E, true, false, false>(dyn, bps, st);
            }
        case 2: return fit_attrs_v<E, false, true, true>(cpt, dyn, bps, st);
        case 3: return fit_attrs_v<E, false, false, true>(cpt, dyn, bps, st);
        default: return fit_attrs_v<E, false, false, false>(cpt, dyn, bps, st);
    }
}

inline cudaError_t fit_attrs_any(int cpt, int cb, int variant, size_t dyn, int* bps, int* st) {
    return cb == 8 ? fit_attrs_e<__nv_bfloat16>(cpt, variant, dyn, bps, st)
                   : fit_attrs_e<float>(cpt, variant, dyn, bps, st);
}

// Grid size, ring depth and shared memory for one problem.  Gcap bounds the
// grid (the partial buffers' row count).
// ldf: leading dimension of the factor workspaces V, U, W the kernel indexes with
// (the workspace's, which may exceed ws_ld(K)); it sizes the resident block.
inline cudaError_t plan_fit(int device, int num_sms, int Gcap, int M, int N, int K, int cb, bool gs, int ldf,
                            const gspca_opts* opts, Plan* p) {
    p->cb = cb;
    p->warm = opts && opts->warm;
    p->gs_passes = (opts && opts->gs_passes == 2) ? 2 : 1;
    p->svd_form = (opts && opts->svd_form == 1) ? 1 : 0;
    p->variant = fit_variant(p->warm, p->gs_passes == 2, K > kRedundantMax);
    p->cpt = cpt_for(N);
    p->ppr = p->cpt >= 8 ? 1 : 8 / p->cpt;
    const int np = (M + 3) / 4;
    int G = num_sms;  // one CTA per SM (512 threads, >= 64 registers each)
    const int want = (np + p->ppr - 1) / p->ppr;
    if (G > want) G = want;
    if (opts && opts->grid_ctas > 0 && opts->grid_ctas < G) G = opts->grid_ctas;
    if (G > Gcap) G = Gcap;
    if (G < 1) G = 1;
    p->G = G;
    p->ldk = ws_ld(K);
    p->max_slice = (N + G - 1) / G + 1;
    // GS-PCA: keep this CTA's rows of V and slices of U and W in shared memory when
    // they take at most kResMaxBytes (auto) or when asked to (opts->resident = 1)
    const int np_cta = (np + G - 1) / G;
    const size_t res = sizeof(float) * ((size_t)4 * np_cta * ldf + 2 * (size_t)p->max_slice * ldf);
    const int rmode = opts ? opts->resident : 0;
    p->res_rows = 0;
    p->res = 0;
    p->gs2 = 0;
    if (gs && rmode != 2 && (rmode == 1 || res <= kResMaxBytes)) {
        p->res_rows = 4 * np_cta;
        p->res = res;
        // the two-reduction GS step adds this CTA's rows of Q and the two ldk x ldk
        // matrices (with bfloat16 storage the kernel recomputes Q's rows from the stored
        // residual after each deflation instead of following it by the rank-1 algebra),
        // up to 4096 columns (wider rows are dominated by the pass over R)
        const size_t extra = sizeof(float) * ((size_t)4 * np_cta * ldf + 2 * (size_t)p->ldk * p->ldk);
        if (!p->warm && p->cpt <= 8 && (!opts || opts->gs_step == 0) && p->gs_passes == 1 &&
            K <= kGs2MaxK &&
            K <= kRedundantMax &&
            res + extra <= kResGs2MaxBytes) {
            p->gs2 = 1;
            p->res = res + extra;
        }
    }
    const size_t vec = vec_bytes(p->ldk, p->max_slice, p->gs2);
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    int bps = 0, st = 0;
    e = fit_attrs_any(p->cpt, cb, p->variant, vec, &bps, &st);
    if (e != cudaSuccess) return e;
    const long avail = (long)optin - st - (long)vec - (long)p->res - 1024;
    // Preferred: the two-group loading pass with one panel per ring stage and an
    // even stage count; otherwise one group with PPR panels per stage.
    p->groups = 1;
    const size_t panel = (size_t)panel_cells(N, cb) * cb;
    size_t stage = panel;
    int S = avail > 0 ? (int)(avail / (long)stage) : 0;
    if (S > kMaxStages) S = kMaxStages;
    S &= ~1;
    const int lpath = opts ? opts->load_path : 0;
    // bfloat16 cells at 2049-4096 columns: the packed register pass (two rounds in
    // flight) streams faster than the ring's few wide stages (measured on GB300)
    const bool packed = cb == 8 && p->cpt == 8 && lpath == 0;
    if (lpath == 2 || packed) {
        S = 0;  // register loads
    } else if (p->cpt >= 2 && p->cpt <= 4 && S >= 4) {
        p->groups = 2;
    } else {
        stage = (size_t)p->ppr * panel;
        S = avail > 0 ? (int)(avail / (long)stage) : 0;
        if (S > kMaxStages) S = kMaxStages;
        if (S < 2) S = 0;
    }
    p->S = S;
    p->dyn = vec + p->res + (size_t)S * stage;
    e = fit_attrs_any(p->cpt, cb, p->variant, p->dyn, &bps, &st);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    return cudaSuccess;
}

template <class E, bool WARM, bool CG2, bool WIDE>
inline cudaError_t launch_fit_v(const FitArgs& a, const Plan& p, cudaStream_t s) {
    switch (p.cpt) {
        case 1: return launch_fit_t<1, E, WARM, CG2, WIDE>(a, p.G, p.dyn, s);
        case 2: return launch_fit_t<2, E, WARM, CG2, WIDE>(a, p.G, p.dyn, s);
        case 4: return launch_fit_t<4, E, WARM, CG2, WIDE>(a, p.G, p.dyn, s);
        case 8: return launch_fit_t<8, E, WARM, CG2, WIDE>(a, p.G, p.dyn, s);
        default: return launch_fit_t<16, E, WARM, CG2, WIDE>(a, p.G, p.dyn, s);
    }
}

template <class E>
inline cudaError_t launch_fit_e(const FitArgs& a, const Plan& p, cudaStream_t s) {
    switch (p.variant) {
        case 1:
            switch (p.cpt) {
                case 1: return launch_fit_t<1, E, true, false, false>(a, p.G, p.dyn, s);
                case 2: return launch_fit_t<2, E, true, false, false>(a, p.G, p.dyn, s);
                case 4: return launch_fit_t<4, E, true, false, false>(a, p.G, p.dyn, s);
                default: return cudaErrorInvalidValue;
            }
        case 2: return launch_fit_v<E, false, true, true>(a, p, s);
        case 3: return launch_fit_v<E, false, false, true>(a, p, s);
        default: return launch_fit_v<E, false, false, false>(a, p, s);
    }
}

inline cudaError_t launch_fit(const FitArgs& a, const Plan& p, cudaStream_t s) {
    return p.cb == 8 ? launch_fit_e<__nv_bfloat16>(a, p, s) : launch_fit_e<float>(a, p, s);
}

// FitArgs for a problem on a carved workspace.
inline FitArgs make_args(const Workspace& w, const Plan& p, int M, int N, int K, double tol, int max_iter,
                         gspca_algo algo, const int* lock_dev, double timeout_s, int nxpart) {
    FitArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.np = (M + 3) / 4;
    a.algo = (int)algo;
    a.max_iter = max_iter;
    a.tol = tol;
    a.eps_thresh = 64.0 * (double)FLT_EPSILON;
    a.xpart = w.xpart;
    a.nxpart = nxpart;
    a.R = w.R;
    a.ldp = panel_cells(N, p.cb);
    a.V = w.V;
    a.ldv = w.ld;
    a.U = w.U;
    a.ldu = w.ld;
    a.W = w.W;
    a.ldw = w.ld;
    a.vraw = w.vraw;
    a.vcorr = w.vcorr;
    a.ut = w.ut;
    a.upre = w.upre;
    a.partA = w.partA;
    a.LA = w.LA;
    a.partB = w.partB;
    a.LB = w.LB;
    a.spart = w.spart;
    a.red = w.red;
    a.lam = w.lam;
    a.iters = w.iters;
    a.info = w.info;
    a.flags = w.flags;
    a.abort = w.abort;
    a.facc = w.facc;
    a.iters_lock = lock_dev;
    a.timeout_ns = (unsigned long long)(timeout_s * 1e9);
    a.timing = nullptr;
    a.tma_stages = p.S;
    a.dot_groups = p.groups;
    a.ring_bytes = (int)(p.dyn - vec_bytes(p.ldk, p.max_slice, p.gs2) - p.res);
    a.gs2 = p.gs2;
    a.res_rows = p.res_rows;
    a.res_off = (int)(p.dyn - p.res);  // after the ring and the vectors
    a.ldk = p.ldk;
    a.max_slice = p.max_slice;
    a.redundant_max = kRedundantMax;
    return a;
}

// Enqueue the launch sequence of one fit on `s` (no synchronisation).
// Returns the number of kernels enqueued through *launches.
inline cudaError_t enqueue_sequence(const Workspace& w, const Plan& p, FitArgs a, cudaStream_t s, const float* X,
                                    gspca_layout layout, long ldx, int center, float* T, float* P,
                                    double* lambda, int* iters, float* R_out, cudaEvent_t ev0, cudaEvent_t ev1,
                                    int* launches) {
    const int M = a.M, N = a.N, K = a.K, np = a.np;
    int n = 0;
    if (center == 1) {
        colmean_kernel<<<(N + 7) / 8, 256, 0, s>>>(X, (int)layout, ldx, M, N, w.cmean);
        ++n;
    } else if (center == 2) {
        rowmean_kernel<<<(M + 7) / 8, 256, 0, s>>>(X, (int)layout, ldx, M, N, w.rmean);
        ++n;
    }
    const dim3 pgrid((N + 31) / 32, (np + 31) / 32);
    if (p.cb == 8)
        launch_pack<__nv_bfloat16>(pgrid, s, X, (int)layout, ldx, M, N, np, a.ldp, center, w.cmean, w.rmean, w.R,
                                   w.xpart, w.flags, 1, w.abort, w.info, kInfoWords);
    else
        launch_pack<float>(pgrid, s, X, (int)layout, ldx, M, N, np, a.ldp, center, w.cmean, w.rmean, w.R, w.xpart,
                           w.flags, 1, w.abort, w.info, kInfoWords);
    ++n;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev0 && (e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
    if ((e = launch_fit(a, p, s)) != cudaSuccess) return e;
    ++n;
    if (ev1 && (e = cudaEventRecord(ev1, s)) != cudaSuccess) return e;
    const dim3 egrid((M + 31) / 32 + (N + 31) / 32, (K + 31) / 32);
    epilogue_kernel<<<egrid, 256, 0, s>>>(w.V, w.ld, w.U, w.ld, w.lam, w.iters, w.info, M, N, K,
                                          a.algo == GSPCA_GS, p.svd_form, T, P, lambda, iters);
    ++n;
    if (R_out) {
        if (p.cb == 8)
            launch_unpack<__nv_bfloat16>(pgrid, s, w.R, M, N, np, a.ldp, w.V, w.ld, w.U, w.ld, w.lam, w.info, K,
                                         a.algo == GSPCA_GS, R_out);
        else
            launch_unpack<float>(pgrid, s, w.R, M, N, np, a.ldp, w.V, w.ld, w.U, w.ld, w.lam, w.info, K,
                                 a.algo == GSPCA_GS, R_out);
        ++n;
    }
    *launches = n;
    return cudaGetLastError();
}

}  // namespace gspca
