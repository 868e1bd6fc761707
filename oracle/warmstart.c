/*
 * FP64 CPU oracle for the learned warm start of GS-PCA (not in the paper:
 * a growth direction of the method, see the repository's design notes).
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: used by the test-suite and the
 * smoke/benchmark checkers, never by the CUDA library, and sharing no code
 * with it.
 *
 * Definitions (the CUDA path implements the same ones independently):
 *   - Sketch: G is M x 16, row-major (G[r*16 + j]), entries drawn N(0, 1/16)
 *     by the caller.  For a residual R (M x N, column-major) and column n:
 *       c_n = ||R(n)||_2,  s_n = G^T R(n) (16 values),
 *       rho = sqrt(sum_n c_n^2 / N)  (root-mean-square column norm),
 *       features x_n = [c_n / rho, s_n / rho]  (17 values; all zero if rho = 0).
 *   - Network (per column, weights shared): 17 -> 64 -> 64 -> 1,
 *       h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), w = W3 . h2 + b3,
 *     gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.  Parameters in one
 *     array: W1 (64 x 17 row-major), b1 (64), W2 (64 x 64 row-major), b2 (64),
 *     W3 (64), b3 (1): 5377 values.
 *   - Start loading p0 = w / ||w||.
 *   - Loss of one instance (columns of one residual, target loading p*):
 *       L = 1 - (w . p*)^2 / (w . w)   (1 with zero gradient when w = 0);
 *     the loss of a set of instances is their mean.
 *   - Choice of the start of component k (GS-PCA): the paper's start is
 *     v_a = R(k) (Sec. 2.3); the learned candidate is v_b = R p0.  With
 *     rho_x = ||R^T v_x||^2 / ||v_x||^2 (the Rayleigh quotient of R R^T at
 *     v_x), v_b replaces v_a when rho_b > rho_a.  The candidate is not
 *     considered when R(k) is zero (the zero-column rule picks the start) or
 *     when w is zero or not finite.
 *   - Optimiser: Adam (Kingma & Ba 2015) with bias correction.
 *
 * Parity pins: tests/test_oracle_warmstart.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define WS_SK 16
#define WS_IN 17
#define WS_H 64
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + WS_H * WS_IN)
#define OFF_W2 (OFF_B1 + WS_H)
#define OFF_B2 (OFF_W2 + WS_H * WS_H)
#define OFF_W3 (OFF_B2 + WS_H)
#define OFF_B3 (OFF_W3 + WS_H)
#define WS_NPAR (OFF_B3 + 1)

int oracle_ws_nparams(void) { return WS_NPAR; }

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }

/* d/dz [z Phi(z)] = Phi(z) + z phi(z). */
static double gelu_d(double z)
{
    const double Phi = 0.5 * (1.0 + erf(z / sqrt(2.0)));
    const double phi = exp(-0.5 * z * z) / sqrt(2.0 * M_PI);
    return Phi + z * phi;
}

int oracle_ws_features(const double *R, int M, int N, const double *G, double *feat)
{
    if (!R || !G || !feat || M < 1 || N < 1)
        return 1;
    double sum_c2 = 0.0;
    for (int n = 0; n < N; n++) {
        const double *col = R + (size_t)n * M;
        double c2 = 0.0;
        double s[WS_SK] = {0};
        for (int r = 0; r < M; r++) {
            c2 += col[r] * col[r];
            for (int j = 0; j < WS_SK; j++)
                s[j] += G[(size_t)r * WS_SK + j] * col[r];
        }
        feat[(size_t)n * WS_IN] = sqrt(c2);
        for (int j = 0; j < WS_SK; j++)
            feat[(size_t)n * WS_IN + 1 + j] = s[j];
        sum_c2 += c2;
    }
    const double rho = sqrt(sum_c2 / N);
    for (size_t i = 0; i < (size_t)N * WS_IN; i++)
        feat[i] = rho > 0.0 ? feat[i] / rho : 0.0;
    return 0;
}

/* Forward pass of one column; keeps the pre-activations for the backward pass. */
static double forward1(const double *net, const double *x, double *z1, double *h1, double *z2, double *h2)
{
    for (int i = 0; i < WS_H; i++) {
        double a = net[OFF_B1 + i];
        for (int f = 0; f < WS_IN; f++)
            a += net[OFF_W1 + i * WS_IN + f] * x[f];
        z1[i] = a;
        h1[i] = gelu(a);
    }
    for (int i = 0; i < WS_H; i++) {
        double a = net[OFF_B2 + i];
        for (int j = 0; j < WS_H; j++)
            a += net[OFF_W2 + i * WS_H + j] * h1[j];
        z2[i] = a;
        h2[i] = gelu(a);
    }
    double w = net[OFF_B3];
    for (int i = 0; i < WS_H; i++)
        w += net[OFF_W3 + i] * h2[i];
    return w;
}

void oracle_ws_forward(const double *net, const double *feat, int n, double *w)
{
    double z1[WS_H], h1[WS_H], z2[WS_H], h2[WS_H];
    for (int c = 0; c < n; c++)
        w[c] = forward1(net, feat + (size_t)c * WS_IN, z1, h1, z2, h2);
}

/* Mean loss over the instances; grad (nullable) receives its gradient with
 * respect to every parameter.  Instance i owns columns [offsets[i], offsets[i+1]). */
double oracle_ws_loss_grad(const double *net, const double *feat, const double *target, const int *offsets,
                           int ninst, double *grad)
{
    if (grad)
        memset(grad, 0, sizeof(double) * WS_NPAR);
    double total = 0.0;
    double z1[WS_H], h1[WS_H], z2[WS_H], h2[WS_H], d2[WS_H];
    for (int i = 0; i < ninst; i++) {
        const int c0 = offsets[i], c1 = offsets[i + 1];
        double *w = malloc(sizeof(double) * (size_t)(c1 > c0 ? c1 - c0 : 1));
        double a = 0.0, b = 0.0;
        for (int c = c0; c < c1; c++) {
            w[c - c0] = forward1(net, feat + (size_t)c * WS_IN, z1, h1, z2, h2);
            a += w[c - c0] * target[c];
            b += w[c - c0] * w[c - c0];
        }
        if (!(b > 0.0)) {
            total += 1.0;
            free(w);
            continue;
        }
        total += 1.0 - a * a / b;
        if (grad) {
            for (int c = c0; c < c1; c++) {
                /* dL_i/dw_c, divided by ninst for the mean */
                const double g = (-2.0 * a * target[c] / b + 2.0 * a * a * w[c - c0] / (b * b)) / ninst;
                const double *x = feat + (size_t)c * WS_IN;
                forward1(net, x, z1, h1, z2, h2);
                grad[OFF_B3] += g;
                for (int k = 0; k < WS_H; k++) {
                    grad[OFF_W3 + k] += g * h2[k];
                    d2[k] = g * net[OFF_W3 + k] * gelu_d(z2[k]);
                    grad[OFF_B2 + k] += d2[k];
                    for (int j = 0; j < WS_H; j++)
                        grad[OFF_W2 + k * WS_H + j] += d2[k] * h1[j];
                }
                for (int j = 0; j < WS_H; j++) {
                    double d1 = 0.0;
                    for (int k = 0; k < WS_H; k++)
                        d1 += net[OFF_W2 + k * WS_H + j] * d2[k];
                    d1 *= gelu_d(z1[j]);
                    grad[OFF_B1 + j] += d1;
                    for (int f = 0; f < WS_IN; f++)
                        grad[OFF_W1 + j * WS_IN + f] += d1 * x[f];
                }
            }
        }
        free(w);
    }
    return ninst > 0 ? total / ninst : 0.0;
}

/* One Adam step (t >= 1): m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
 * theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void oracle_ws_adam(double *net, double *m, double *v, const double *grad, int t, double lr, double b1,
                    double b2, double eps, int n)
{
    const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int i = 0; i < n; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        net[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* Start of GS-PCA component k on the residual R: returns 1 and the learned
 * candidate in v when it beats the paper's start R(col) by the rule above,
 * else 0 (v untouched).  rho (nullable) receives rho_a, rho_b. */
int oracle_ws_choose_start(const double *R, int M, int N, int col, const double *G, const double *net, double *v,
                           double *rho)
{
    double *feat = malloc(sizeof(double) * (size_t)N * WS_IN);
    double *w = malloc(sizeof(double) * (size_t)N);
    double *vb = malloc(sizeof(double) * (size_t)M);
    double *t = malloc(sizeof(double) * (size_t)N);
    int use = 0;
    if (!feat || !w || !vb || !t)
        goto done;
    oracle_ws_features(R, M, N, G, feat);
    oracle_ws_forward(net, feat, N, w);
    double ww = 0.0;
    for (int n = 0; n < N; n++)
        ww += w[n] * w[n];
    if (!(ww > 0.0) || !isfinite(ww))
        goto done;
    const double inv = 1.0 / sqrt(ww);
    for (int r = 0; r < M; r++)
        vb[r] = 0.0;
    for (int n = 0; n < N; n++) {
        const double pn = w[n] * inv;
        for (int r = 0; r < M; r++)
            vb[r] += R[(size_t)n * M + r] * pn;
    }
    const double *va = R + (size_t)col * M;
    double rho_x[2];
    for (int x = 0; x < 2; x++) {
        const double *vx = x == 0 ? va : vb;
        double nv = 0.0, nt = 0.0;
        for (int r = 0; r < M; r++)
            nv += vx[r] * vx[r];
        for (int n = 0; n < N; n++) {
            double s = 0.0;
            for (int r = 0; r < M; r++)
                s += R[(size_t)n * M + r] * vx[r];
            t[n] = s;
            nt += s * s;
        }
        rho_x[x] = nv > 0.0 ? nt / nv : -1.0;
    }
    if (rho) {
        rho[0] = rho_x[0];
        rho[1] = rho_x[1];
    }
    if (rho_x[1] > rho_x[0]) {
        memcpy(v, vb, sizeof(double) * (size_t)M);
        use = 1;
    }
done:
    free(feat);
    free(w);
    free(vb);
    free(t);
    return use;
}
