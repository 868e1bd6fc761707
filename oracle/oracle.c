/*
 * FP64 CPU oracle for NIPALS-PCA and GS-PCA, written from Andrecut,
 * "Parallel GPU Implementation of Iterative PCA Algorithms" (arXiv:0811.1081).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header or constant with the CUDA library it checks, and it never
 * calls it.
 *
 * Conventions
 *   - Every matrix is column-major with leading dimension = its row count:
 *     element (m, n) of an M x N matrix lives at [n*M + m] (Sec. 3: "Matrix A
 *     is stored in column major format").
 *   - Arithmetic is IEEE-754 double, round to nearest, one rounding per
 *     operation (build with -ffp-contract=off), every sum in plain index
 *     order.  No blocking, no reordering, no BLAS.
 *   - Readings of points the paper leaves open (each one is listed with its
 *     reason in the design notes of the repository):
 *       * convergence test: relative and strict, |lambda' - lambda| < tol*lambda',
 *         lambda starting at 0, at most max_iter iterations (the test used in
 *         all four appendix programs; Sec. 2.2/2.3 print it as absolute);
 *       * Gram-Schmidt: one classical pass per half-iteration (Sec. 2.3
 *         pseudo-code, as in the appendix programs); gs_passes = 2 applies
 *         the classical pass twice ("applied iteratively", the remark of
 *         Sec. 2.3 before the GS-PCA pseudo-code), every pass taking its
 *         coefficients from the vector the previous pass left;
 *       * zero start column: when column k of the residual is exactly zero,
 *         start from the residual column of largest norm (lowest index on
 *         ties); when every column is zero the fit stops as degenerate;
 *       * rank exhausted: a norm <= 64*eps64*||X||_F stops the fit as
 *         degenerate; the components found so far are kept, the rest are 0;
 *       * NIPALS returns lambda_k = ||t_k|| (the pseudo-code's lambda');
 *       * storage 1 ("R held in bfloat16", a precision variant of Sec. 3's
 *         remark that the programs switch precision by their type alone): the
 *         residual is rounded to the nearest bfloat16 after centring and after
 *         every deflation (Eq. 3), and used exactly as stored; all arithmetic
 *         on it stays FP64.
 *   - Status codes: 0 ok, 1 invalid argument, 4 at least one component hit
 *     max_iter, 5 degenerate (fewer than K components found).
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID 1
#define OR_NOT_CONVERGED 4
#define OR_DEGENERATE 5

/* Learned warm start (warmstart.c). */
int oracle_ws_choose_start(const double *R, int M, int N, int col, const double *G, const double *net, double *v,
                           double *rho);

/* ---------------------------------------------------------------- helpers */

/* Largest finite bfloat16: (2 - 2^-7) * 2^127. */
#define BF16_MAX (0x1.fep127)

/* Round x to the nearest bfloat16 value, ties to even.  bfloat16 keeps the
 * 8-bit exponent of IEEE binary32 and 8 significant bits (7 stored): for
 * |x| in [2^(e-1), 2^e) with e-1 >= -126 the representable values are the
 * multiples of 2^(e-8); below 2^-126 (subnormal) the multiples of 2^-133.
 * Magnitudes that round beyond BF16_MAX become infinities. */
double oracle_round_bf16(double x)
{
    if (x == 0.0 || !isfinite(x))
        return x;
    int e;
    frexp(x, &e);
    if (e < -125)
        e = -125;
    const double q = ldexp(1.0, e - 8);
    const double r = nearbyint(x / q) * q; /* default rounding mode: to nearest, ties to even */
    if (fabs(r) > BF16_MAX)
        return copysign(INFINITY, x);
    return r;
}

/* Apply the storage rounding of R (storage 1: bfloat16) to n values. */
static void store_round(double *R, size_t n, int storage)
{
    if (storage != 1)
        return;
    for (size_t i = 0; i < n; i++)
        R[i] = oracle_round_bf16(R[i]);
}

static double dot(const double *x, const double *y, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; i++)
        s += x[i] * y[i];
    return s;
}

/* Euclidean norm, Sec. 3 (nrm2): square root of the sum of squares. */
static double nrm2(const double *x, int n)
{
    return sqrt(dot(x, x, n));
}

static void scal(double *x, int n, double alpha)
{
    for (int i = 0; i < n; i++)
        x[i] *= alpha;
}

/* Multi-threaded builds (-fopenmp, used only to time the oracle on many host
 * cores) split the loops below over independent output elements; every
 * element still receives its terms in the same index order, so the results
 * are the single-threaded ones bit for bit.  Without -fopenmp the pragmas are
 * ignored.  Rows are split in blocks of ROW_BLOCK. */
#define ROW_BLOCK 512

/* y = A^T x for A (rows x cols), i.e. y[c] = sum_r A[r,c] x[r]  (gemv 't'). */
static void gemv_t(const double *A, int rows, int cols, const double *x, double *y)
{
#pragma omp parallel for schedule(static) if (cols > 64)
    for (int c = 0; c < cols; c++)
        y[c] = dot(A + (size_t)c * rows, x, rows);
}

/* y = A x for A (rows x cols), i.e. y[r] = sum_c A[r,c] x[c]  (gemv 'n').
 * Every y[r] receives its terms in index order c = 0, 1, ...; within a block
 * of rows the loop runs over columns so that the column-major matrix is read
 * contiguously. */
static void gemv_n(const double *A, int rows, int cols, const double *x, double *y)
{
    const int nb = (rows + ROW_BLOCK - 1) / ROW_BLOCK;
#pragma omp parallel for schedule(static) if (nb > 1)
    for (int b = 0; b < nb; b++) {
        const int r0 = b * ROW_BLOCK, r1 = r0 + ROW_BLOCK < rows ? r0 + ROW_BLOCK : rows;
        for (int r = r0; r < r1; r++)
            y[r] = 0.0;
        for (int c = 0; c < cols; c++) {
            const double *col = A + (size_t)c * rows;
            const double xc = x[c];
            for (int r = r0; r < r1; r++)
                y[r] += col[r] * xc;
        }
    }
}

/* A <- A + alpha x y^T  (ger, Eq. 3 deflation). */
static void ger(double *A, int rows, int cols, double alpha, const double *x, const double *y)
{
#pragma omp parallel for schedule(static) if (cols > 64)
    for (int c = 0; c < cols; c++) {
        double ay = alpha * y[c];
        double *col = A + (size_t)c * rows;
        for (int r = 0; r < rows; r++)
            col[r] += x[r] * ay;
    }
}

/* One classical Gram-Schmidt pass of x against the first k columns of Q
 * (Sec. 2.3): coef = Q_(k)^T x, then x <- x - Q_(k) coef.  All k coefficients
 * are taken from the unmodified x (classical, not modified, Gram-Schmidt);
 * every x[r] loses its k terms in order j = 0, 1, ... */
static void cgs_pass(const double *Q, int rows, int k, double *x, double *coef)
{
    gemv_t(Q, rows, k, x, coef);
    const int nb = (rows + ROW_BLOCK - 1) / ROW_BLOCK;
#pragma omp parallel for schedule(static) if (nb > 1)
    for (int b = 0; b < nb; b++) {
        const int r0 = b * ROW_BLOCK, r1 = r0 + ROW_BLOCK < rows ? r0 + ROW_BLOCK : rows;
        for (int j = 0; j < k; j++) {
            const double *q = Q + (size_t)j * rows;
            for (int r = r0; r < r1; r++)
                x[r] -= q[r] * coef[j];
        }
    }
}

/* Exported for the pins: `passes` classical Gram-Schmidt passes of x against
 * the first k columns of Q (rows x k, column-major).  coef receives the
 * coefficients of the last pass.  Returns 0, or 1 on bad arguments. */
int oracle_cgs(const double *Q, int rows, int k, double *x, double *coef, int passes)
{
    if (!Q || !x || !coef || rows < 1 || k < 1 || passes < 1)
        return 1;
    for (int p = 0; p < passes; p++)
        cgs_pass(Q, rows, k, x, coef);
    return 0;
}

static double frob(const double *A, int rows, int cols)
{
    return nrm2(A, rows * cols);
}

/* Start column for component k: column k of the residual, unless it is
 * exactly zero; then the column of largest norm (lowest index on ties).
 * Returns -1 when every column is zero. */
static int start_column(const double *R, int M, int N, int k)
{
    if (nrm2(R + (size_t)k * M, M) != 0.0)
        return k;
    int best = -1;
    double bestn = 0.0;
    for (int c = 0; c < N; c++) {
        double n = nrm2(R + (size_t)c * M, M);
        if (n > bestn) {
            bestn = n;
            best = c;
        }
    }
    return best;
}

/* Convergence bookkeeping shared by both algorithms.  j is the number of
 * completed iterations.  Returns 1 when the loop must stop. */
static int stop_now(int j, double prev, double cur, double tol, int max_iter,
                    const int *iters_lock, int k, int *not_converged)
{
    if (iters_lock)
        return j >= iters_lock[k];
    if (fabs(prev - cur) < tol * cur)
        return 1;
    if (j >= max_iter) {
        *not_converged = 1;
        return 1;
    }
    return 0;
}

static void zero_tail(double *T, double *P, double *lambda, int *iters,
                      int M, int N, int K, int k)
{
    for (int j = k; j < K; j++) {
        memset(T + (size_t)j * M, 0, sizeof(double) * M);
        memset(P + (size_t)j * N, 0, sizeof(double) * N);
        lambda[j] = 0.0;
        iters[j] = 0;
    }
}

/* ------------------------------------------------------------- centring */

/* mode 1: every column loses its own mean (the prose of Sec. 2.1: "each
 *         column is mean centered").
 * mode 2: Eq. 1 as printed: the average column N^-1 sum_n X^(n) is
 *         subtracted from every column, so each row ends with zero mean. */
int oracle_center(double *R, int M, int N, int mode)
{
    if (M < 1 || N < 1)
        return OR_INVALID;
    if (mode == 0)
        return OR_OK;
    if (mode == 1) {
        for (int c = 0; c < N; c++) {
            double *col = R + (size_t)c * M;
            double s = 0.0;
            for (int r = 0; r < M; r++)
                s += col[r];
            double mean = s / M;
            for (int r = 0; r < M; r++)
                col[r] -= mean;
        }
        return OR_OK;
    }
    if (mode == 2) {
        double *avg = calloc((size_t)M, sizeof(double));
        if (!avg)
            return OR_INVALID;
        for (int c = 0; c < N; c++)
            for (int r = 0; r < M; r++)
                avg[r] += R[(size_t)c * M + r];
        for (int r = 0; r < M; r++)
            avg[r] /= N;
        for (int c = 0; c < N; c++)
            for (int r = 0; r < M; r++)
                R[(size_t)c * M + r] -= avg[r];
        free(avg);
        return OR_OK;
    }
    return OR_INVALID;
}

/* --------------------------------------------------------------- NIPALS */

/* NIPALS-PCA, Sec. 2.2 pseudo-code:
 *   R <- X
 *   for k: lambda = 0; T(k) <- R(k)
 *     repeat: P(k) <- R^T T(k); P(k) <- P(k)/||P(k)||; T(k) <- R P(k);
 *             lambda' <- ||T(k)||; stop when converged; lambda <- lambda'
 *     R <- R - T(k) P(k)^T            (Eq. 3)
 * T keeps the unnormalised scores, so X = T P^T + R (Eq. 4). */
static int nipals(double *R, int M, int N, int K, double tol, int max_iter,
                  const int *iters_lock, double thresh, int storage,
                  double *T, double *P, double *lambda, int *iters, int *found)
{
    int not_converged = 0;
    for (int k = 0; k < K; k++) {
        double *t = T + (size_t)k * M;
        double *p = P + (size_t)k * N;
        int c = start_column(R, M, N, k);
        if (c < 0) {
            *found = k;
            zero_tail(T, P, lambda, iters, M, N, K, k);
            return OR_DEGENERATE;
        }
        memcpy(t, R + (size_t)c * M, sizeof(double) * M);
        double prev = 0.0, cur = 0.0;
        int j = 0;
        for (;;) {
            gemv_t(R, M, N, t, p);
            double np = nrm2(p, N);
            if (np == 0.0) {
                *found = k;
                zero_tail(T, P, lambda, iters, M, N, K, k);
                return OR_DEGENERATE;
            }
            scal(p, N, 1.0 / np);
            gemv_n(R, M, N, p, t);
            cur = nrm2(t, M);
            if (cur <= thresh) {
                *found = k;
                zero_tail(T, P, lambda, iters, M, N, K, k);
                return OR_DEGENERATE;
            }
            j++;
            if (stop_now(j, prev, cur, tol, max_iter, iters_lock, k, &not_converged))
                break;
            prev = cur;
        }
        lambda[k] = cur;
        iters[k] = j;
        ger(R, M, N, -1.0, t, p);
        store_round(R, (size_t)M * N, storage);
    }
    *found = K;
    return not_converged ? OR_NOT_CONVERGED : OR_OK;
}

/* ------------------------------------------------------------------ GS-PCA */

/* GS-PCA, Sec. 2.3 pseudo-code (truncated-SVD form, Eq. 5):
 *   R <- X
 *   for k: mu = 0; V(k) <- R(k)
 *     repeat: U(k) <- R^T V(k)
 *             if k>0: A <- U_(k)^T U(k); U(k) <- U(k) - U_(k) A   (gs_passes times)
 *             U(k) <- U(k)/||U(k)||
 *             V(k) <- R U(k)
 *             if k>0: B <- V_(k)^T V(k); V(k) <- V(k) - V_(k) B   (gs_passes times)
 *             lambda_k <- ||V(k)||; V(k) <- V(k)/lambda_k
 *             stop when converged; mu <- lambda_k
 *     R <- R - lambda_k V(k) U(k)^T
 *   T <- V Lambda; P <- U
 * While a component is being extracted, column j < k of T holds V(j) (unit
 * norm); the scaling T = V Lambda happens once at the end. */
static int gspca(double *R, int M, int N, int K, double tol, int max_iter,
                 const int *iters_lock, double thresh, int storage, int gs_passes,
                 const double *ws_net, const double *ws_G, int *ws_choice, double *ws_rho,
                 double *T, double *P, double *lambda, int *iters, int *found)
{
    int not_converged = 0, status = OR_OK, kfound = K;
    double *coef = malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    if (!coef)
        return OR_INVALID;
    for (int k = 0; k < K; k++) {
        double *v = T + (size_t)k * M;
        double *u = P + (size_t)k * N;
        int c = start_column(R, M, N, k);
        if (c < 0) {
            kfound = k;
            status = OR_DEGENERATE;
            break;
        }
        memcpy(v, R + (size_t)c * M, sizeof(double) * M);
        if (ws_net) {
            /* learned candidate, considered only when the paper's start column is nonzero */
            int use = 0;
            if (c == k)
                use = oracle_ws_choose_start(R, M, N, c, ws_G, ws_net, v, ws_rho ? ws_rho + 2 * k : NULL);
            if (ws_choice)
                ws_choice[k] = use;
        }
        double mu = 0.0, lam = 0.0;
        int j = 0, degenerate = 0;
        for (;;) {
            gemv_t(R, M, N, v, u);
            for (int pass = 0; k > 0 && pass < gs_passes; pass++)
                cgs_pass(P, N, k, u, coef);
            double nu = nrm2(u, N);
            if (nu == 0.0) {
                degenerate = 1;
                break;
            }
            scal(u, N, 1.0 / nu);
            gemv_n(R, M, N, u, v);
            for (int pass = 0; k > 0 && pass < gs_passes; pass++)
                cgs_pass(T, M, k, v, coef);
            lam = nrm2(v, M);
            if (lam <= thresh) {
                degenerate = 1;
                break;
            }
            scal(v, M, 1.0 / lam);
            j++;
            if (stop_now(j, mu, lam, tol, max_iter, iters_lock, k, &not_converged))
                break;
            mu = lam;
        }
        if (degenerate) {
            kfound = k;
            status = OR_DEGENERATE;
            break;
        }
        lambda[k] = lam;
        iters[k] = j;
        ger(R, M, N, -lam, v, u);
        store_round(R, (size_t)M * N, storage);
    }
    free(coef);
    for (int k = 0; k < kfound; k++)
        scal(T + (size_t)k * M, M, lambda[k]);
    if (kfound < K)
        zero_tail(T, P, lambda, iters, M, N, K, kfound);
    *found = kfound;
    if (status == OR_OK && not_converged)
        status = OR_NOT_CONVERGED;
    return status;
}

/* ------------------------------------------------------------ entry point */

/* algo 0 = NIPALS-PCA, 1 = GS-PCA.  X (M x N) is read only; R receives the
 * final residual (X, centred as requested, minus every extracted component).
 * iters_lock (nullable): run exactly iters_lock[k] iterations for component k
 * and ignore the convergence test (used to replay another implementation's
 * iteration counts).  storage: 0 = R kept in FP64; 1 = R rounded to bfloat16
 * after centring and after every deflation.  gs_passes (GS-PCA): classical
 * Gram-Schmidt passes per half-iteration, 1 (the pseudo-code) or 2 (CGS2).
 * ws_net / ws_G (nullable, GS-PCA
 * only): parameters and sketch of the learned warm start (warmstart.c);
 * ws_choice (K ints) and ws_rho (2K doubles) receive, per component, whether
 * the learned start was used and the two Rayleigh quotients compared.
 * Outputs: T (M x K), P (N x K), lambda (K), iters (K), found (number of
 * components extracted). */
int oracle_fit(int algo, const double *X, int M, int N, int K, double tol, int max_iter,
               int center, const int *iters_lock, int storage, int gs_passes,
               const double *ws_net, const double *ws_G, int *ws_choice, double *ws_rho,
               double *T, double *P, double *lambda, int *iters, double *R, int *found)
{
    if (!X || !T || !P || !lambda || !iters || !R || !found)
        return OR_INVALID;
    if (M < 1 || N < 1 || K < 1 || K > M || K > N || !(tol > 0.0) || max_iter < 1)
        return OR_INVALID;
    if (algo != 0 && algo != 1)
        return OR_INVALID;
    if (storage != 0 && storage != 1)
        return OR_INVALID;
    if (gs_passes != 1 && gs_passes != 2)
        return OR_INVALID;
    if (ws_net && (algo != 1 || !ws_G))
        return OR_INVALID;
    if (ws_choice)
        for (int k = 0; k < K; k++)
            ws_choice[k] = 0;
    if (iters_lock)
        for (int k = 0; k < K; k++)
            if (iters_lock[k] < 1)
                return OR_INVALID;
    memcpy(R, X, sizeof(double) * (size_t)M * N);
    int st = oracle_center(R, M, N, center);
    if (st != OR_OK)
        return st;
    store_round(R, (size_t)M * N, storage);
    double thresh = 64.0 * DBL_EPSILON * frob(R, M, N);
    if (algo == 0)
        return nipals(R, M, N, K, tol, max_iter, iters_lock, thresh, storage, T, P, lambda, iters, found);
    return gspca(R, M, N, K, tol, max_iter, iters_lock, thresh, storage, gs_passes, ws_net, ws_G, ws_choice, ws_rho,
                 T, P, lambda, iters, found);
}

/* ------------------------------------------------------- Jacobi eigensolver */

/* Cyclic-by-row Jacobi method for a symmetric n x n matrix A (Golub & Van
 * Loan, "Matrix Computations", Sec. 8.5): sweep over every pair (p, q),
 * p < q, and zero A[p,q] with the rotation J = [[c, s], [-s, c]] that solves
 * the 2 x 2 symmetric Schur problem, A <- J^T A J, W <- W J; stop when the
 * off-diagonal Frobenius norm is at most tol * ||A||_F.  A is overwritten;
 * evals/evecs return the eigenpairs sorted by decreasing eigenvalue
 * (evecs column-major, n x n).  Returns the number of sweeps, -1 on bad
 * arguments, -2 when max_sweeps was reached. */
int oracle_jacobi_eigh(double *A, int n, double tol, int max_sweeps, double *evals, double *evecs)
{
    if (!A || !evals || !evecs || n < 1 || max_sweeps < 1)
        return -1;
    double *W = calloc((size_t)n * n, sizeof(double));
    if (!W)
        return -1;
    for (int i = 0; i < n; i++)
        W[(size_t)i * n + i] = 1.0;
    double anorm = frob(A, n, n);
    int sweep = 0, done = 0;
    while (sweep < max_sweeps) {
        double off = 0.0;
        for (int q = 0; q < n; q++)
            for (int p = 0; p < n; p++)
                if (p != q)
                    off += A[(size_t)q * n + p] * A[(size_t)q * n + p];
        if (sqrt(off) <= tol * anorm) {
            done = 1;
            break;
        }
        sweep++;
        for (int p = 0; p < n - 1; p++) {
            for (int q = p + 1; q < n; q++) {
                double apq = A[(size_t)q * n + p];
                if (apq == 0.0)
                    continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* A <- A J (columns p and q) */
                for (int i = 0; i < n; i++) {
                    double aip = A[(size_t)p * n + i], aiq = A[(size_t)q * n + i];
                    A[(size_t)p * n + i] = c * aip - s * aiq;
                    A[(size_t)q * n + i] = s * aip + c * aiq;
                }
                /* A <- J^T A (rows p and q) */
                for (int i = 0; i < n; i++) {
                    double api = A[(size_t)i * n + p], aqi = A[(size_t)i * n + q];
                    A[(size_t)i * n + p] = c * api - s * aqi;
                    A[(size_t)i * n + q] = s * api + c * aqi;
                }
                /* W <- W J */
                for (int i = 0; i < n; i++) {
                    double wip = W[(size_t)p * n + i], wiq = W[(size_t)q * n + i];
                    W[(size_t)p * n + i] = c * wip - s * wiq;
                    W[(size_t)q * n + i] = s * wip + c * wiq;
                }
            }
        }
    }
    if (!done) {
        double off = 0.0;
        for (int q = 0; q < n; q++)
            for (int p = 0; p < n; p++)
                if (p != q)
                    off += A[(size_t)q * n + p] * A[(size_t)q * n + p];
        done = sqrt(off) <= tol * anorm;
    }
    /* selection sort by decreasing eigenvalue */
    int *order = malloc(sizeof(int) * (size_t)n);
    if (!order) {
        free(W);
        return -1;
    }
    for (int i = 0; i < n; i++)
        order[i] = i;
    for (int i = 0; i < n; i++) {
        int best = i;
        for (int j = i + 1; j < n; j++)
            if (A[(size_t)order[j] * n + order[j]] > A[(size_t)order[best] * n + order[best]])
                best = j;
        int tmp = order[i];
        order[i] = order[best];
        order[best] = tmp;
    }
    for (int i = 0; i < n; i++) {
        evals[i] = A[(size_t)order[i] * n + order[i]];
        memcpy(evecs + (size_t)i * n, W + (size_t)order[i] * n, sizeof(double) * n);
    }
    free(order);
    free(W);
    return done ? sweep : -2;
}

/* ------------------------------------------------ block (subspace) iteration */

/* Thin QR of the rows x cols matrix A (column-major) by classical Gram-Schmidt
 * applied twice per column (CGS2): A <- Q with orthonormal columns, Rf (cols x
 * cols, column-major, upper triangular, positive diagonal) with A_in = Q Rf.
 * Returns the index of the first column that is numerically dependent
 * (norm after projection <= 64 eps of its norm before), or -1. */
static int qr_cgs2(double *A, int rows, int cols, double *Rf)
{
    for (int i = 0; i < cols * cols; i++)
        Rf[i] = 0.0;
    double *c = malloc(sizeof(double) * (size_t)(cols > 0 ? cols : 1));
    if (!c)
        return 0;
    for (int j = 0; j < cols; j++) {
        double *a = A + (size_t)j * rows;
        const double n0 = nrm2(a, rows);
        for (int pass = 0; pass < 2 && j > 0; pass++) {
            gemv_t(A, rows, j, a, c);
            for (int i = 0; i < j; i++) {
                const double *q = A + (size_t)i * rows;
                for (int r = 0; r < rows; r++)
                    a[r] -= q[r] * c[i];
                Rf[(size_t)j * cols + i] += c[i];
            }
        }
        const double n1 = nrm2(a, rows);
        if (!(n1 > 64.0 * DBL_EPSILON * n0) || n1 == 0.0) {
            free(c);
            return j;
        }
        scal(a, rows, 1.0 / n1);
        Rf[(size_t)j * cols + j] = n1;
    }
    free(c);
    return -1;
}

/* C (m x n) = A^T B for A (rows x m), B (rows x n), column-major. */
static void gemm_tn(const double *A, const double *B, int rows, int m, int n, double *C)
{
    for (int j = 0; j < n; j++)
        gemv_t(A, rows, m, B + (size_t)j * rows, C + (size_t)j * m);
}

/* Y (rows x n) = A (rows x cols) B (cols x n), column-major. */
static void gemm_nn(const double *A, const double *B, int rows, int cols, int n, double *Y)
{
    for (int j = 0; j < n; j++)
        gemv_n(A, rows, cols, B + (size_t)j * cols, Y + (size_t)j * rows);
}

/* X <- X - Q (Q^T X) for Q (rows x k, orthonormal columns) and X (rows x n). */
static void project_out(const double *Q, int rows, int k, double *X, int n, double *tmp)
{
    if (k == 0)
        return;
    gemm_tn(Q, X, rows, k, n, tmp);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < k; i++) {
            const double c = tmp[(size_t)j * k + i];
            const double *q = Q + (size_t)i * rows;
            double *x = X + (size_t)j * rows;
            for (int r = 0; r < rows; r++)
                x[r] -= q[r] * c;
        }
}

/* Block power iteration (subspace iteration with Rayleigh-Ritz), the block
 * form of the GS-PCA loop of Sec. 2.3 (not in the paper): components are
 * extracted b at a time.  For a block of width b (the last one narrower):
 *   U <- R^T R(:, k0 .. k0+b-1)  (the paper's start v = R(k), u = R^T v, for b columns)
 *   U <- U - U_(k0) U_(k0)^T U ; U <- qr(U)
 *   repeat: Y <- R U ; Y <- Y - V_(k0) V_(k0)^T Y ; V <- qr(Y)
 *           Z <- R^T V ; Z <- Z - U_(k0) U_(k0)^T Z
 *           s <- singular values of Z, decreasing (the Ritz values)
 *           stop when |s_i - s_i'| < tol s_i for every i (s' of the previous iteration,
 *           0 at first) or after max_iter iterations; otherwise U <- qr(Z)
 *   Rayleigh-Ritz: B = V^T R U = Z^T U (b x b), B = Yh diag(sigma) Zh^T (decreasing),
 *   V <- V Yh, U <- U Zh, lambda = sigma;  R <- R - V diag(lambda) U^T (Eq. 3 for b columns).
 * T = V Lambda, P = U (Eq. 5).  qr is CGS2; the singular values come from the
 * Jacobi eigensolver below applied to Z^T Z and B^T B.  A start or iterate whose
 * columns become numerically dependent stops the fit as degenerate (the
 * components of earlier blocks are kept).  iters_lock (nullable, K entries):
 * block starting at k0 runs exactly iters_lock[k0] iterations.  Every component
 * of a block reports the block's iteration count. */
int oracle_block_fit(const double *X, int M, int N, int K, int b, double tol, int max_iter, const int *iters_lock,
                     double *T, double *P, double *lambda, int *iters, double *R, int *found)
{
    if (!X || !T || !P || !lambda || !iters || !R || !found)
        return OR_INVALID;
    if (M < 1 || N < 1 || K < 1 || K > M || K > N || b < 1 || !(tol > 0.0) || max_iter < 1)
        return OR_INVALID;
    memcpy(R, X, sizeof(double) * (size_t)M * N);
    const int B = b < K ? b : K;
    double *U = malloc(sizeof(double) * (size_t)N * B), *Y = malloc(sizeof(double) * (size_t)M * B);
    double *Z = malloc(sizeof(double) * (size_t)N * B), *Rf = malloc(sizeof(double) * (size_t)B * B);
    double *G = malloc(sizeof(double) * (size_t)B * B), *E = malloc(sizeof(double) * (size_t)B * B);
    double *s = malloc(sizeof(double) * (size_t)B), *sp = malloc(sizeof(double) * (size_t)B);
    double *tmp = malloc(sizeof(double) * (size_t)K * B), *Bm = malloc(sizeof(double) * (size_t)B * B);
    double *Zh = malloc(sizeof(double) * (size_t)B * B), *Yh = malloc(sizeof(double) * (size_t)M * B);
    double *Un = malloc(sizeof(double) * (size_t)N * B);
    int status = OR_OK, kf = 0, not_converged = 0;
    if (!U || !Y || !Z || !Rf || !G || !E || !s || !sp || !tmp || !Bm || !Zh || !Yh || !Un) {
        status = OR_INVALID;
        goto out;
    }
    for (int k0 = 0; k0 < K; k0 += B) {
        const int bw = (K - k0) < B ? (K - k0) : B;
        double *Vp = T, *Up = P; /* V_(k0), U_(k0): the first k0 columns (unit columns until the end) */
        gemm_tn(R, R + (size_t)k0 * M, M, N, bw, U); /* U = R^T R(:, k0 .. k0+bw-1) */
        project_out(Up, N, k0, U, bw, tmp);
        if (qr_cgs2(U, N, bw, Rf) >= 0) {
            status = OR_DEGENERATE;
            break;
        }
        for (int i = 0; i < bw; i++)
            sp[i] = 0.0;
        int j = 0;
        for (;;) {
            gemm_nn(R, U, M, N, bw, Y);
            project_out(Vp, M, k0, Y, bw, tmp);
            if (qr_cgs2(Y, M, bw, Rf) >= 0) {
                status = OR_DEGENERATE;
                break;
            }
            gemm_tn(R, Y, M, N, bw, Z); /* Z = R^T V */
            project_out(Up, N, k0, Z, bw, tmp);
            gemm_tn(Z, Z, N, bw, bw, G);
            if (oracle_jacobi_eigh(G, bw, 1e-15, 100, s, E) == -1) {
                status = OR_INVALID;
                break;
            }
            for (int i = 0; i < bw; i++)
                s[i] = sqrt(s[i] > 0.0 ? s[i] : 0.0);
            j++;
            int stop;
            if (iters_lock) {
                stop = j >= iters_lock[k0];
            } else {
                stop = 1;
                for (int i = 0; i < bw; i++)
                    if (!(fabs(sp[i] - s[i]) < tol * s[i]))
                        stop = 0;
                if (!stop && j >= max_iter) {
                    stop = 1;
                    not_converged = 1;
                }
            }
            if (stop)
                break;
            for (int i = 0; i < bw; i++)
                sp[i] = s[i];
            memcpy(U, Z, sizeof(double) * (size_t)N * bw);
            if (qr_cgs2(U, N, bw, Rf) >= 0) {
                status = OR_DEGENERATE;
                break;
            }
        }
        if (status != OR_OK)
            break;
        /* Rayleigh-Ritz: B = Z^T U, B^T B = Zh diag(sigma^2) Zh^T, Yh = B Zh / sigma */
        gemm_tn(Z, U, N, bw, bw, Bm);
        gemm_tn(Bm, Bm, bw, bw, bw, G);
        if (oracle_jacobi_eigh(G, bw, 1e-15, 100, s, Zh) == -1) {
            status = OR_INVALID;
            break;
        }
        int deg = 0;
        for (int i = 0; i < bw; i++) {
            s[i] = sqrt(s[i] > 0.0 ? s[i] : 0.0);
            if (!(s[i] > 0.0))
                deg = 1;
        }
        if (deg) {
            status = OR_DEGENERATE;
            break;
        }
        gemm_nn(Bm, Zh, bw, bw, bw, E); /* E = B Zh (columns sigma_i times Yh) */
        for (int i = 0; i < bw; i++)
            scal(E + (size_t)i * bw, bw, 1.0 / s[i]);
        gemm_nn(Y, E, M, bw, bw, Yh); /* V Yh */
        gemm_nn(U, Zh, N, bw, bw, Un); /* U Zh */
        for (int i = 0; i < bw; i++) {
            memcpy(T + (size_t)(k0 + i) * M, Yh + (size_t)i * M, sizeof(double) * M);
            memcpy(P + (size_t)(k0 + i) * N, Un + (size_t)i * N, sizeof(double) * N);
            lambda[k0 + i] = s[i];
            iters[k0 + i] = j;
        }
        for (int i = 0; i < bw; i++)
            ger(R, M, N, -s[i], T + (size_t)(k0 + i) * M, P + (size_t)(k0 + i) * N);
        kf = k0 + bw;
    }
    if (status == OR_OK && not_converged)
        status = OR_NOT_CONVERGED;
out:
    if (status != OR_INVALID) {
        for (int k = 0; k < kf; k++)
            scal(T + (size_t)k * M, M, lambda[k]);
        if (kf < K)
            zero_tail(T, P, lambda, iters, M, N, K, kf);
        *found = kf;
    }
    free(U), free(Y), free(Z), free(Rf), free(G), free(E), free(s), free(sp), free(tmp), free(Bm), free(Zh), free(Yh),
        free(Un);
    return status;
}
