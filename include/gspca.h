/*
 * gspca.h -- C ABI of the GB300 (sm_103a) implementation of the iterative PCA
 * algorithms of M. Andrecut, "Parallel GPU Implementation of Iterative PCA
 * Algorithms" (arXiv:0811.1081): NIPALS-PCA (Sec. 2.2) and GS-PCA (Sec. 2.3).
 *
 * Problem statement (Sec. 2.1, Eq. 2-5): X is M x N, columns are attributes,
 * rows are observations.  K components are extracted one at a time by power
 * iteration on the residual R (R <- X first), each followed by the rank-1
 * deflation R <- R - T(k) P(k)^T (Eq. 3), so that X = T_(K) P_(K)^T + R
 * (Eq. 4).  GS-PCA re-orthogonalises the loading against P_(k) and the score
 * direction against the normalised earlier scores at every iteration with one
 * classical Gram-Schmidt pass, and returns T = V Lambda, P = U (Eq. 5).
 *
 * Conventions shared by every entry point
 *   - All pointers are plain pointers.  Unless an entry point says "host",
 *     data pointers are device pointers on the handle's device, and the
 *     caller owns them.  The library never frees caller memory.
 *   - X is FP32.  It is read only.  layout = GSPCA_COL_MAJOR means element
 *     (m, n) at X[n*ldx + m] (ldx >= M; the paper's storage, Sec. 3);
 *     GSPCA_ROW_MAJOR means X[m*ldx + n] (ldx >= N).
 *   - Outputs are column-major with leading dimension = rows:
 *     T is M x K (T[k*M + m]), P is N x K (P[k*N + n]), lambda holds K
 *     doubles, iters K ints, R_out (optional) is M x N (R_out[n*M + m]).
 *     GS-PCA: T = V Lambda and lambda_k = ||V(k)|| before normalisation
 *     (a singular value of the residual).  NIPALS-PCA: T holds the
 *     unnormalised scores t_k and lambda_k = ||t_k|| (Sec. 2.2).
 *   - The convergence test is relative and strict: stop when
 *     |lambda_j - lambda_{j-1}| < tol * lambda_j (lambda_{-1} = 0), or after
 *     max_iter iterations (the test of the paper's appendix programs).
 *   - Components past the last one found (status GSPCA_ERR_DEGENERATE) are
 *     zero in T, P, lambda and iters.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     All device work of a call is enqueued on it.  A handle must not be used
 *     by two calls at once (its workspace is shared by its calls).
 *   - Errors are reported only through the return value; nothing is printed.
 */
#ifndef GSPCA_H
#define GSPCA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gspca_handle *gspca_t;

typedef enum { GSPCA_NIPALS = 0, GSPCA_GS = 1 } gspca_algo;

/* Storage type of the residual R inside the library.
 * GSPCA_F32, GSPCA_BF16: X is FP32 (gspca_fit and the other entry points);
 *   GSPCA_BF16 rounds X to bfloat16 once; every product uses FP32 accumulation
 *   and the Gram-Schmidt coefficients, norms and the test stay in float-float /
 *   FP64-combined FP32 sums.
 * GSPCA_F64: the paper's own precision (Sec. 3): X, R, the factors, every
 *   product, the outputs and the test in IEEE double; only gspca_fit_f64 takes
 *   such a handle. */
typedef enum { GSPCA_F32 = 0, GSPCA_BF16 = 1, GSPCA_F64 = 2 } gspca_dtype;

typedef enum { GSPCA_COL_MAJOR = 0, GSPCA_ROW_MAJOR = 1 } gspca_layout;

/* Optional centring before the fit (Sec. 2.1, Eq. 1).
 *   GSPCA_CENTER_COLUMNS: every column loses its own mean (the prose of
 *                         Sec. 2.1, standard PCA).
 *   GSPCA_CENTER_ROWS:    Eq. 1 as printed: the average column is subtracted
 *                         from every column (each row ends with zero mean). */
typedef enum { GSPCA_CENTER_NONE = 0, GSPCA_CENTER_COLUMNS = 1, GSPCA_CENTER_ROWS = 2 } gspca_center;

typedef enum {
    GSPCA_OK = 0,
    GSPCA_ERR_INVALID_ARG = 1,      /* bad size, pointer, tolerance, ... ; nothing was launched */
    GSPCA_ERR_CUDA = 2,             /* a CUDA call failed; see gspca_last_cuda_error */
    GSPCA_ERR_OOM = 3,              /* workspace allocation failed */
    GSPCA_WARN_NOT_CONVERGED = 4,   /* results valid; >= 1 component stopped at max_iter */
    GSPCA_ERR_DEGENERATE = 5,       /* rank exhausted: fewer than K components found */
    GSPCA_ERR_TIMEOUT = 6,          /* a bounded device wait gave up; results invalid */
    GSPCA_ERR_NOT_SUPPORTED = 7     /* sizes beyond what this build handles */
} gspca_status;

/* Learned warm start of GS-PCA.  The paper has no counterpart: it is a
 * growth direction of the loop of Sec. 2.3, whose start is the residual
 * column v = R(k).  At the start of component k a small network proposes a
 * loading p0 from per-column features of the residual R, and the first pass
 * over R evaluates both starts:
 *   features of column n: x_n = [c_n, s_n] / rho with c_n = ||R(n)||,
 *     s_n = G^T R(n) (16 values, G the sketch below), rho^2 = sum_n c_n^2 / N;
 *     they are computed once per fit from the packed R and then follow every
 *     deflation (Eq. 3) exactly, at O(16 (M + N)) work per component;
 *   network (weights shared by all columns): h1 = gelu(W1 x + b1),
 *     h2 = gelu(W2 h1 + b2), w_n = W3 . h2 + b3, gelu(z) = z (1 + erf(z/sqrt 2))/2,
 *     p0 = w / ||w||;
 *   choice: with v_a = R(k) (the paper's start) and v_b = R p0, the loop
 *     starts from v_b when ||R^T v_b||^2 / ||v_b||^2 > ||R^T v_a||^2 / ||v_a||^2,
 *     otherwise from v_a, exactly as the paper; the candidate is skipped when
 *     w is zero or not finite, or R(k) is zero (the zero-column rule applies).
 * GS-PCA only.  Parameter layout (FP32, GSPCA_WS_PARAMS values): W1 (64 x 17,
 * row-major), b1 (64), W2 (64 x 64, row-major), b2 (64), W3 (64), b3 (1). */
#define GSPCA_WS_SKETCH 16
#define GSPCA_WS_FEATURES 17
#define GSPCA_WS_PARAMS 5377

typedef struct {
    const float *net;   /* device: GSPCA_WS_PARAMS network parameters */
    const float *G;     /* device: sketch, G_rows x 16 row-major (entries drawn by the caller,
                           N(0, 1/16) in the intended use); a problem of M rows uses rows 0..M-1 */
    long G_rows;        /* must be >= M of every problem */
    int *choice;        /* device, nullable (gspca_fit only): K ints, 1 where the learned start
                           was used, 0 where the paper's start was */
} gspca_warm_start;

typedef struct {
    int center;             /* gspca_center, default GSPCA_CENTER_NONE */
    const int *iters_lock;  /* host array of K counts, nullable: run exactly iters_lock[k]
                               iterations for component k and ignore the test */
    int grid_ctas;          /* CTAs of the persistent kernel; 0 = automatic */
    double timeout_s;       /* limit of every device-side wait; 0 = 2 seconds */
    int cluster_ctas;       /* batched form: CTAs per problem team (1, 2, 4, 8 or 16);
                               0 = chosen by the library's autotuner */
    int batch_pass;         /* batched form: loading pass of the iterations; 1 = independent
                               warp groups (no CTA-wide barrier per round), 2 = CTA-wide
                               rounds through the shared-memory TMA ring; 0 = autotuned */
    int test_stall;         /* testing only, default 0: when 1, the first wait on the shared-
                               memory ring in every pass first waits for a device word that
                               nothing sets, so the wait limit (timeout_s) runs out and the
                               call reports GSPCA_ERR_TIMEOUT; exercises the timeout path
                               without a fault */
    const gspca_warm_start *warm;  /* host pointer, nullable: learned warm start (GS-PCA only;
                               gspca_fit, gspca_fit_host, gspca_fit_batched[_async]).  The first
                               call on a handle that uses it grows the handle's workspace. */
    int resident;           /* single-problem GS-PCA: 0 = automatic, 1 = keep each CTA's rows of the
                               score factors and slices of the loading factors in shared memory
                               (fewer pipeline stages for R), 2 = keep them in global memory.  The
                               results do not depend on it. */
    int load_path;          /* single-problem fit: how the passes read R; 0 = automatic, 1 = through
                               the shared-memory ring of TMA bulk copies where it fits, 2 = straight
                               into registers.  The results do not depend on it. */
    int gs_step;            /* single-problem GS-PCA with resident factors: 0 = automatic (the
                               Gram-Schmidt step of an iteration takes two grid-wide reductions
                               where that is numerically safe, by keeping Q = R U, Z = U^T W and
                               V^T V up to date per component; otherwise three), 1 = always the
                               three-reduction step of Sec. 2.3.  The two agree to FP32 rounding. */
    int gs_passes;          /* GS-PCA, single-problem entry points: classical Gram-Schmidt passes per
                               half-iteration.  0 or 1 = one pass (the Sec. 2.3 pseudo-code and the
                               appendix programs); 2 = the iterated form Sec. 2.3 mentions (CGS2):
                               the second pass takes its coefficients from the vector the first
                               pass left, at the cost of one more grid-wide reduction per
                               half-iteration (it implies the three-reduction step).  The batched
                               entry points, and the learned warm start, accept 0 or 1 only
                               (GSPCA_ERR_NOT_SUPPORTED). */
    int svd_form;           /* single-problem entry points: 0 (default) = T holds the scores, T = V
                               Lambda for GS-PCA and t_k for NIPALS-PCA; 1 = T holds the unit score
                               directions, the SVD form X = V Lambda P^T + R of Eq. 5 (Sec. 2.3):
                               V(k) for GS-PCA, t_k / lambda_k for NIPALS-PCA.  With K = N and every
                               component converged, R vanishes and (T, lambda, P) is the full SVD.
                               The batched entry points accept 0 only (GSPCA_ERR_NOT_SUPPORTED). */
    float *coef_trace;      /* testing aid, nullable; gspca_fit only (device pointer, ignored by the
                               other entry points): K * (2K + M + N) floats.  For every GS-PCA
                               component k >= 1 the last iteration's Gram-Schmidt coefficients
                               b' = V_(k)^T v' (floats [k(2K+M+N), +k)) and a' = U_(k)^T u_pre'
                               ([k(2K+M+N) + K, +k)), and the vectors they were formed from: v' = R u'
                               (M floats from k(2K+M+N) + 2K) and u_pre' = R^T (v' - V_(k) b')
                               (N floats after v'), both in the pass's scale.  Other entries are
                               left untouched. */
} gspca_opts;

/* Per-call record of the last fit on a handle (host memory). */
typedef struct {
    int found;              /* components extracted */
    long long total_iters;  /* sum of iters over the components */
    int kernel_launches;    /* kernels this call enqueued */
    int grid_ctas;          /* CTAs of the persistent kernel */
    int block_threads;
    double alg_bytes;       /* algorithmic bytes of the persistent kernel (one read of R per
                               pass, deflation write, Gram-Schmidt factor reads) */
    double kernel_ms;       /* device time of the persistent kernel, from CUDA events recorded
                               around its launch on the caller's stream */
    int team_ctas;          /* batched form: CTAs per problem team; single fit: grid_ctas */
    int batch_pass;         /* batched form: loading pass used (1 or 2, see gspca_opts); else 0 */
} gspca_info;

/* Create a handle on `device` with workspace for problems up to
 * max_M x max_N and max_K components stored as `dtype`.  The handle owns that
 * workspace (device memory, freed by gspca_destroy).
 * Errors: GSPCA_ERR_INVALID_ARG (h NULL, sizes < 1), GSPCA_ERR_NOT_SUPPORTED
 * (max_N above the per-CTA column limit of this build, 8192), GSPCA_ERR_OOM,
 * GSPCA_ERR_CUDA. */
gspca_status gspca_create(gspca_t *h, int device, long max_M, long max_N, int max_K,
                          gspca_dtype dtype);

/* Fit K components of X (device pointers, see the conventions above).
 * Sec. 2.2 / 2.3 pseudo-code with a device-resident loop: one persistent
 * kernel runs every iteration and every convergence decision; the host only
 * enqueues it and, at the end, synchronises `stream` and reads the status.
 * Requirements: a GSPCA_F32 or GSPCA_BF16 handle, 1 <= K <= min(M, N),
 * M <= max_M, N <= max_N, K <= max_K, tol > 0, max_iter >= 1, T, P, lambda
 * non-NULL; iters, R_out, opts nullable.
 * Returns GSPCA_OK, GSPCA_WARN_NOT_CONVERGED or GSPCA_ERR_DEGENERATE with valid
 * outputs; other codes leave the outputs unspecified. */
gspca_status gspca_fit(gspca_t h, void *stream, const float *X, gspca_layout layout, long ldx,
                       int M, int N, int K, double tol, int max_iter, gspca_algo algo,
                       float *T, float *P, double *lambda, int *iters, float *R_out,
                       const gspca_opts *opts);

/* Same as gspca_fit with HOST pointers for X, T, P, lambda, iters and R_out:
 * the call copies X to the handle's device staging buffer, fits, and copies
 * the results back, all on `stream`, and returns once they are in host
 * memory.  The staging buffers are allocated on the first call and owned by
 * the handle. */
gspca_status gspca_fit_host(gspca_t h, void *stream, const float *X, gspca_layout layout,
                            long ldx, int M, int N, int K, double tol, int max_iter,
                            gspca_algo algo, float *T, float *P, double *lambda, int *iters,
                            float *R_out, const gspca_opts *opts);

/* Fit in FP64 (the precision of the paper's programs, Sec. 3): NIPALS-PCA or
 * GS-PCA (Sec. 2.2 / 2.3) with X, R, the factors, every product and sum, the
 * outputs and the convergence test in IEEE double, on a handle created with
 * GSPCA_F64.  Same arguments and conventions as gspca_fit with double for X, T,
 * P and R_out (device pointers).  Cross-CTA sums run in a fixed order, so two
 * runs give the same bits; the results match an FP64 evaluation in another
 * summation order to rounding.  opts: center, iters_lock, grid_ctas, timeout_s
 * and svd_form apply; warm, gs_passes = 2 and coef_trace give
 * GSPCA_ERR_NOT_SUPPORTED.  Also GSPCA_ERR_INVALID_ARG for a handle of another
 * dtype, GSPCA_ERR_NOT_SUPPORTED when one row of N doubles (and the loop's
 * vectors) does not fit a CTA's shared memory (about N > 8192). */
gspca_status gspca_fit_f64(gspca_t h, void *stream, const double *X, gspca_layout layout, long ldx, int M, int N,
                           int K, double tol, int max_iter, gspca_algo algo, double *T, double *P, double *lambda,
                           int *iters, double *R_out, const gspca_opts *opts);

/* Block power iteration: components `block` at a time (1 <= block <= 32), the
 * block form of the Sec. 2.3 loop; the paper has no counterpart (it extracts one
 * component at a time).  For a block of width b starting at component k0:
 *   U = R^T R(:, k0 .. k0+b-1), made orthogonal to P(:, 0:k0) and orthonormal;
 *   repeat: Y = R U, made orthogonal to the earlier score directions, V = qr(Y);
 *           Z = R^T V, made orthogonal to P(:, 0:k0); Ritz values s = singular
 *           values of Z; stop when every |s_i - s_i(previous)| < tol s_i, after
 *           max_iter iterations or after iters_lock[k0] (opts); else U = qr(Z);
 *   Rayleigh-Ritz: B = V^T R U = Yh diag(sigma) Zh^T (sigma decreasing),
 *   V <- V Yh, U <- U Zh, lambda = sigma; R <- R - V diag(lambda) U^T (Eq. 3).
 * Outputs as gspca_fit (T = V Lambda, or V with opts->svd_form = 1; P = U; every
 * component of a block reports the block's iteration count).  The products with
 * R and the projections are FP32 matrix products (cuBLAS); qr is Cholesky QR
 * applied twice with FP64 Gram matrices.  A GSPCA_F32 handle; X FP32 device
 * memory; opts: center, iters_lock, svd_form apply (warm, gs_passes = 2 and
 * coef_trace give GSPCA_ERR_NOT_SUPPORTED).  A block whose start or iterate has
 * numerically dependent columns ends the fit with GSPCA_ERR_DEGENERATE (earlier
 * blocks kept).  The first call on a handle allocates the block workspace and a
 * cuBLAS handle (owned by the handle).  Synchronises `stream` once per iteration. */
gspca_status gspca_fit_block(gspca_t h, void *stream, const float *X, gspca_layout layout, long ldx, int M, int N,
                             int K, int block, double tol, int max_iter, float *T, float *P, double *lambda,
                             int *iters, float *R_out, const gspca_opts *opts);

/* One independent problem of a batch (device pointers, same conventions as
 * gspca_fit, column-major X with leading dimension ldx). */
typedef struct {
    const float *X;
    long ldx;
    int M, N, K;
    float *T, *P;
    double *lambda;
    int *iters;             /* nullable */
    int *status;            /* nullable: per-problem gspca_status (device int) */
    int *ws_choice;         /* nullable: K device ints, 1 where the learned start was used
                               (opts->warm set) */
} gspca_problem;

/* Fit `count` independent problems (problems[] is a HOST array of
 * descriptors; every pointer inside is a device pointer) with one algorithm,
 * tolerance and iteration cap.  Not in the paper: the same per-component loop
 * (Sec. 2.2 / 2.3) run for many small problems at once.
 *
 * Execution: one persistent launch per 256 problems.  The grid is made of
 * thread-block clusters; each cluster is a team of cluster_ctas CTAs that
 * takes the next problem from a device work queue (largest M*N first), packs
 * its X, fits it and writes its T, P, lambda, iters and status, then takes the
 * next.  opts->center must be GSPCA_CENTER_NONE and opts->iters_lock NULL.
 * Requirements per problem: 1 <= K <= min(M, N), N <= 1024, ldx >= M,
 * M <= max_M, N <= max_N and K <= max_K of the handle; X, T, P, lambda
 * non-NULL.  count >= 1.
 *
 * Team size: opts->cluster_ctas, or (0) the autotuner's choice for this list
 * of shapes: on the first call with a new shape list that is not being
 * captured, every feasible team size is timed on the real batch and the
 * fastest is kept in the handle (the outputs are those of a final run with
 * it).  The batch workspace (one private panel copy of the largest problem per
 * cluster) is allocated, or grown, by calls that are not being captured and
 * owned by the handle.
 *
 * gspca_fit_batched synchronises `stream` and returns the worst
 * per-problem status (GSPCA_OK < GSPCA_WARN_NOT_CONVERGED <
 * GSPCA_ERR_DEGENERATE < GSPCA_ERR_TIMEOUT). */
gspca_status gspca_fit_batched(gspca_t h, void *stream, const gspca_problem *problems, int count,
                               double tol, int max_iter, gspca_algo algo, const gspca_opts *opts);

/* Asynchronous form of gspca_fit_batched, usable inside CUDA stream capture:
 * enqueues the batch on `stream` and returns GSPCA_OK without waiting; the
 * per-problem status words and *worst_status (a device int, nullable) are
 * written by the GPU.  Under capture the call launches with the team size and
 * workspace of an earlier uncaptured call on the same shape list (without one
 * it returns GSPCA_ERR_NOT_SUPPORTED and enqueues nothing); the descriptors are
 * copied into the launch parameters, so the captured graph does not depend on
 * problems[] afterwards. */
gspca_status gspca_fit_batched_async(gspca_t h, void *stream, const gspca_problem *problems,
                                     int count, double tol, int max_iter, gspca_algo algo,
                                     const gspca_opts *opts, int *worst_status);

/* Fit without allocating.  The paper has no counterpart to this entry point;
 * it exists for callers that must not allocate device memory themselves or
 * through the library: for example a plug-in running inside an application
 * whose own allocator owns the device memory (an outside cudaMalloc can fail
 * or break that allocator's budget), or a latency-critical loop that cannot
 * afford a cudaMalloc/cudaFree pair (cudaFree can synchronise the device).
 *
 * Same computation and conventions as gspca_fit (device pointers for X, T,
 * P, lambda, iters, R_out), but no handle: the scratch workspace is a
 * file-scope device array of GSPCA_NOALLOC_SCRATCH_BYTES bytes inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  The call runs on the current device and never calls cudaMalloc,
 * cudaFree or any allocating routine.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress)
 *     with the current device, so the address stays right after a
 *     cudaDeviceReset reloads the library's device code.  The first call on a
 *     device also loads that code; make it before any stream capture.
 *   - Every call shares the one array and leaves its contents behind; the
 *     words that must start at zero (grid barrier, abort flag, status) are
 *     cleared by the call's own first kernel.  Calls whose work overlaps on
 *     the GPU (other streams, other host threads) race on the array: order
 *     them on one stream or synchronise between them.
 *   - Limit: the scratch this problem needs (about 4*(M+3)*(N+K) +
 *     8*(M+N)*(K+2) bytes plus per-CTA partial sums) must fit in
 *     GSPCA_NOALLOC_SCRATCH_BYTES; otherwise the call returns
 *     GSPCA_ERR_NOT_SUPPORTED and launches nothing.  Other errors as for
 *     gspca_fit.  The call synchronises `stream` before returning. */
#define GSPCA_NOALLOC_SCRATCH_BYTES (64u << 20)
gspca_status gspca_fit_noalloc(void *stream, const float *X, gspca_layout layout, long ldx, int M,
                               int N, int K, double tol, int max_iter, gspca_algo algo, float *T,
                               float *P, double *lambda, int *iters, float *R_out,
                               const gspca_opts *opts);

/* Learned warm start: features of the columns of R_k = X - T(:, 0:k) P(:, 0:k)^T
 * (the residual before component k of a finished fit; X column-major, ldx >= M;
 * T M x >=k and P N x >=k column-major with leading dimensions M and N, as gspca_fit
 * writes them; k = 0 ignores T and P).  feat (N x 17, row-major) receives
 * x_n = [||R_k(n)||, G^T R_k(n)] / rho as defined above.  Device pointers; runs on
 * `stream` without waiting; allocates nothing.  Used to build training data. */
gspca_status gspca_ws_features(void *stream, const float *X, long ldx, int M, int N, const float *T,
                               const float *P, int k, const float *G, float *feat);

/* Learned warm start: w[n] = network(feat[n]) for n < count (feat row-major, 17 per
 * row).  Device pointers; runs on `stream` without waiting; allocates nothing. */
gspca_status gspca_ws_forward(void *stream, const float *net, const float *feat, long count, float *w);

/* Learned warm start: one training step on a minibatch of ninst instances.  Instance
 * i owns feature rows offsets[i] .. offsets[i+1]-1 (offsets: device, ninst + 1 ints,
 * offsets[0] = 0, offsets[ninst] = ncols) and target[] holds its target loading p*
 * on those rows (unit norm).  Loss of an instance: 1 - (w . p*)^2 / (w . w) (1 with
 * zero gradient when w = 0); the step minimises the mean over the minibatch with one
 * Adam update (step t >= 1, bias-corrected, beta1 0.9, beta2 0.999, eps 1e-8) of net
 * with its moment buffers adam_m, adam_v (GSPCA_WS_PARAMS each, zero before t = 1).
 * lr = 0 leaves net, adam_m and adam_v unchanged.  loss (device float) and grad
 * (device, GSPCA_WS_PARAMS) are nullable outputs: the minibatch loss and gradient
 * before the update.  The handle owns the step's scratch, grown on demand (not under
 * stream capture).  Runs on `stream` without waiting. */
gspca_status gspca_ws_train_step(gspca_t h, void *stream, float *net, float *adam_m, float *adam_v, int step,
                                 float lr, const float *feat, const float *target, const int *offsets,
                                 int ninst, long ncols, float *loss, float *grad);

/* Record of the last call on h. */
gspca_status gspca_get_info(gspca_t h, gspca_info *info);

/* Release the handle and its workspace.  NULL is accepted. */
gspca_status gspca_destroy(gspca_t h);

/* Static English description of a status code (never NULL). */
const char *gspca_status_string(gspca_status s);

/* Text of the last CUDA error seen by the library in this process (static
 * storage, never NULL). */
const char *gspca_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GSPCA_H */
