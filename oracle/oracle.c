/*
 * FP64 CPU oracle for the F-BMP hot path (arXiv 2103.09943).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The CUDA path shares no
 * code with it.
 *
 * Plain loops in double precision, written for a reader checking them
 * against the paper, not for speed. Images are row-major H x W (row y,
 * column x); every index wraps around the torus (circular convolution,
 * Sec. II-A, "Notation"). A blur kernel u has n = 2R+1 taps per side, tap
 * (i, j) in [-R, R]^2 stored at u[(i+R)*n + (j+R)].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static long wrap(long i, long n)
{
    long m = i % n;
    return m < 0 ? m + n : m;
}

/* (D B(u) z)(k, l) = sum_{i,j} u(i,j) z(c k - i, c l - j).
 * B(u) is circular convolution with u, D keeps every c-th sample at phase 0
 * (Sec. II-A, Eq. objective0). Output is h x w with h = H/c, w = W/c. */
void or_blur_decimate(const double *z, long H, long W, const double *u, int R,
                      int c, double *v)
{
    long h = H / c, w = W / c;
    int n = 2 * R + 1;
    for (long k = 0; k < h; ++k)
        for (long l = 0; l < w; ++l) {
            double s = 0.0;
            for (int i = -R; i <= R; ++i)
                for (int j = -R; j <= R; ++j)
                    s += u[(i + R) * n + (j + R)] *
                         z[wrap(c * k - i, H) * W + wrap(c * l - j, W)];
            v[k * w + l] = s;
        }
}

/* B^T D^T v: the transpose of the loop above, written as the scatter of
 * every LR sample back onto the HR taps it was built from. */
void or_blur_decimate_adj(const double *v, long H, long W, const double *u,
                          int R, int c, double *z)
{
    long h = H / c, w = W / c;
    int n = 2 * R + 1;
    memset(z, 0, sizeof(double) * H * W);
    for (long k = 0; k < h; ++k)
        for (long l = 0; l < w; ++l)
            for (int i = -R; i <= R; ++i)
                for (int j = -R; j <= R; ++j)
                    z[wrap(c * k - i, H) * W + wrap(c * l - j, W)] +=
                        u[(i + R) * n + (j + R)] * v[k * w + l];
}

/* L z = z circularly convolved with S = [[0,-1,0],[-1,4,-1],[0,-1,0]]
 * (Sec. II-C, Eq. reg2). S is symmetric, so L^T = L. */
void or_laplacian(const double *z, long H, long W, double *out)
{
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x)
            out[y * W + x] = 4.0 * z[y * W + x] - z[wrap(y - 1, H) * W + x] -
                             z[wrap(y + 1, H) * W + x] - z[y * W + wrap(x - 1, W)] -
                             z[y * W + wrap(x + 1, W)];
}

/* Sum of a over the (2r+1)^2 window centred at every pixel (torus). */
static void window_sum(const double *a, long H, long W, int r, double *out)
{
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            double s = 0.0;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx)
                    s += a[wrap(y + dy, H) * W + wrap(x + dx, W)];
            out[y * W + x] = s;
        }
}

/* PAN window statistics (Algorithm 2, step 3; Eq. matting_matrix and
 * Eq. ac_h_compute): the guide I = L Y, and for every window w_j its mean
 * mu_j, population variance var_j and s_j = 1 / (var_j + eps). */
void or_pan_stats(const double *Y, long H, long W, int r, double eps,
                  double *I, double *mu, double *var, double *s)
{
    long P = H * W;
    double nw = (double)((2 * r + 1) * (2 * r + 1));
    double *I2 = malloc(sizeof(double) * P);
    double *S2 = malloc(sizeof(double) * P);
    or_laplacian(Y, H, W, I);
    for (long m = 0; m < P; ++m) I2[m] = I[m] * I[m];
    window_sum(I, H, W, r, mu);
    window_sum(I2, H, W, r, S2);
    for (long m = 0; m < P; ++m) {
        mu[m] /= nw;
        var[m] = S2[m] / nw - mu[m] * mu[m];
        s[m] = 1.0 / (var[m] + eps);
    }
    free(I2);
    free(S2);
}

/* Per-window affine fit of q against the guide I (Eq. ac_h_compute):
 * a_j = (mean_j(I q) - mu_j mean_j(q)) s_j,  c_j = mean_j(q) - a_j mu_j. */
static void window_affine(const double *q, const double *I, const double *mu,
                          const double *s, long H, long W, int r, double *a,
                          double *c)
{
    long P = H * W;
    double nw = (double)((2 * r + 1) * (2 * r + 1));
    double *Iq = malloc(sizeof(double) * P);
    double *qm = malloc(sizeof(double) * P);
    for (long m = 0; m < P; ++m) Iq[m] = I[m] * q[m];
    window_sum(q, H, W, r, qm);
    window_sum(Iq, H, W, r, a);
    for (long m = 0; m < P; ++m) {
        qm[m] /= nw;
        a[m] = (a[m] / nw - mu[m] * qm[m]) * s[m];
        c[m] = qm[m] - a[m] * mu[m];
    }
    free(Iq);
    free(qm);
}

/* Matting matrix product M alpha (Eq. matting_matrix, reading sigma^2 + eps
 * for the denominator). Each window's term in alpha^T M alpha is the residual
 * of its best affine fit (Eq. pansharp_penalty); differentiating gives
 * (M alpha)_m = sum_{j : m in w_j} (alpha_m - a_j I_m - c_j)
 *             = |w| alpha_m - I_m sum_{j in w_m} a_j - sum_{j in w_m} c_j. */
void or_matting_apply(const double *alpha, const double *I, const double *mu,
                      const double *s, long H, long W, int r, double *out)
{
    long P = H * W;
    double nw = (double)((2 * r + 1) * (2 * r + 1));
    double *a = malloc(sizeof(double) * P), *c = malloc(sizeof(double) * P);
    double *sa = malloc(sizeof(double) * P), *sc = malloc(sizeof(double) * P);
    window_affine(alpha, I, mu, s, H, W, r, a, c);
    window_sum(a, H, W, r, sa);
    window_sum(c, H, W, r, sc);
    for (long m = 0; m < P; ++m) out[m] = nw * alpha[m] - I[m] * sa[m] - sc[m];
    free(a);
    free(c);
    free(sa);
    free(sc);
}

/* Guided filter output (Sec. III-B, Eq. ac_h_compute and the text before
 * Eq. Z_solution): with a_j, c_j fitted per window,
 * out_k = mean_{j in w_k}(a_j) I_k + mean_{j in w_k}(c_j). */
void or_guided_filter(const double *q, const double *I, const double *mu,
                      const double *s, long H, long W, int r, double *out)
{
    long P = H * W;
    double nw = (double)((2 * r + 1) * (2 * r + 1));
    double *a = malloc(sizeof(double) * P), *c = malloc(sizeof(double) * P);
    double *sa = malloc(sizeof(double) * P), *sc = malloc(sizeof(double) * P);
    window_affine(q, I, mu, s, H, W, r, a, c);
    window_sum(a, H, W, r, sa);
    window_sum(c, H, W, r, sc);
    for (long m = 0; m < P; ++m) out[m] = (sa[m] * I[m] + sc[m]) / nw;
    free(a);
    free(c);
    free(sa);
    free(sc);
}

/* Problem description shared by the two HRMS linear systems. */
typedef struct {
    long H, W;
    int c, R, r;
    const double *u;           /* kernel, n*n */
    const double *I, *mu, *s;  /* PAN statistics (Z0 system only) */
    double lam;                /* weight of the prior term */
    int op;                    /* 0: Z0 system, 1: Z-step system */
} or_system;

/* op 0 (Eq. Z_ini_matting): (B^T D^T D B + lam L^T M L) z.
 * op 1 (Eq. Z_solution):    (B^T D^T D B + lam L^T L) z. */
static void apply_system(const or_system *S, const double *z, double *out)
{
    long H = S->H, W = S->W, P = H * W;
    long h = H / S->c, w = W / S->c;
    double *v = malloc(sizeof(double) * h * w);
    double *Lz = malloc(sizeof(double) * P);
    double *t = malloc(sizeof(double) * P);
    double *Lt = malloc(sizeof(double) * P);
    or_blur_decimate(z, H, W, S->u, S->R, S->c, v);
    or_blur_decimate_adj(v, H, W, S->u, S->R, S->c, out);
    or_laplacian(z, H, W, Lz);
    if (S->op == 0)
        or_matting_apply(Lz, S->I, S->mu, S->s, H, W, S->r, t);
    else
        memcpy(t, Lz, sizeof(double) * P);
    or_laplacian(t, H, W, Lt);
    for (long m = 0; m < P; ++m) out[m] += S->lam * Lt[m];
    free(v);
    free(Lz);
    free(t);
    free(Lt);
}

void or_apply_system(long H, long W, int c, const double *u, int R,
                     const double *I, const double *mu, const double *s, int r,
                     double lam, int op, const double *z, double *out)
{
    or_system S = {H, W, c, R, r, u, I, mu, s, lam, op};
    apply_system(&S, z, out);
}

static double dot(const double *a, const double *b, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Conjugate gradient (Hestenes-Stiefel) on the SPD system above, from the
 * start x (overwritten with the result). Stops when ||b - A x|| / ||b|| <= tol
 * (recursive residual) or after maxit iterations. Returns the iteration
 * count; *relres receives the final TRUE relative residual. */
int or_cg(long H, long W, int c, const double *u, int R, const double *I,
          const double *mu, const double *s, int r, double lam, int op,
          const double *b, double *x, double tol, int maxit, double *relres)
{
    or_system S = {H, W, c, R, r, u, I, mu, s, lam, op};
    long P = H * W;
    double *res = malloc(sizeof(double) * P), *p = malloc(sizeof(double) * P);
    double *Ap = malloc(sizeof(double) * P);
    apply_system(&S, x, Ap);
    for (long m = 0; m < P; ++m) res[m] = b[m] - Ap[m];
    memcpy(p, res, sizeof(double) * P);
    double bb = dot(b, b, P), rr = dot(res, res, P);
    int it = 0;
    if (bb == 0.0) bb = 1.0;
    while (it < maxit && sqrt(rr / bb) > tol) {
        apply_system(&S, p, Ap);
        double alpha = rr / dot(p, Ap, P);
        for (long m = 0; m < P; ++m) {
            x[m] += alpha * p[m];
            res[m] -= alpha * Ap[m];
        }
        double rr_new = dot(res, res, P);
        double beta = rr_new / rr;
        rr = rr_new;
        for (long m = 0; m < P; ++m) p[m] = res[m] + beta * p[m];
        ++it;
    }
    apply_system(&S, x, Ap);
    for (long m = 0; m < P; ++m) res[m] = b[m] - Ap[m];
    *relres = sqrt(dot(res, res, P) / bb);
    free(res);
    free(p);
    free(Ap);
    return it;
}

/* Unit-gain (2*half+1)^2 box filter on the torus (the low-pass filters u1,
 * u2 of Eq. objective3). */
void or_box_filter(const double *a, long H, long W, int half, double *out)
{
    double nw = (double)((2 * half + 1) * (2 * half + 1));
    window_sum(a, H, W, half, out);
    for (long m = 0; m < H * W; ++m) out[m] /= nw;
}

/* Kernel normal equations (Eq. z_update, Eq. z_solution): E = D C(Y) has one
 * row per LR site q, E[q, a] = Y(c q - a) for every tap a, so that E u equals
 * D B(u) Y. Accumulates E^T E (n^2 x n^2, full) and E^T f (n^2). */
void or_kernel_normal_eq(const double *Y, long H, long W, int c, int R,
                         const double *f, double *EtE, double *Etf)
{
    long h = H / c, w = W / c;
    int n = 2 * R + 1, nn = n * n;
    double *e = malloc(sizeof(double) * nn);
    memset(EtE, 0, sizeof(double) * nn * nn);
    memset(Etf, 0, sizeof(double) * nn);
    for (long k = 0; k < h; ++k)
        for (long l = 0; l < w; ++l) {
            for (int i = -R; i <= R; ++i)
                for (int j = -R; j <= R; ++j)
                    e[(i + R) * n + (j + R)] =
                        Y[wrap(c * k - i, H) * W + wrap(c * l - j, W)];
            double fq = f[k * w + l];
            for (int a = 0; a < nn; ++a) {
                Etf[a] += e[a] * fq;
                for (int b = a; b < nn; ++b) EtE[a * nn + b] += e[a] * e[b];
            }
        }
    for (int a = 0; a < nn; ++a)
        for (int b = 0; b < a; ++b) EtE[a * nn + b] = EtE[b * nn + a];
    free(e);
}
