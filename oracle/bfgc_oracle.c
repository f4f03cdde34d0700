/*
 * FP64 CPU oracle for the Gauss-Chebyshev bilateral filter
 * (Ghosh & Chaudhury, "Fast and High-Quality Bilateral Filtering Using
 * Gauss-Chebyshev Approximation", 2016).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; it is compiled by oracle/build.py and used by tests/,
 * the smoke check and the CPU-baseline leg of the benchmark.  It shares no
 * code with the CUDA library.
 *
 * Everything is plain double precision, row-major (index y*W + x, H rows,
 * W columns), written for clarity rather than speed.  OpenMP (when the
 * compiler provides it) only splits the outermost pixel loops.
 *
 * Readings of points where the paper is silent or ambiguous:
 *  - symmetric extension (Sec. I): half-sample mirror per axis,
 *    ... f1 f0 | f0 f1 ... f(n-1) | f(n-1) f(n-2) ..., repeated with
 *    period 2n when the window is wider than the image;
 *  - the window half-width W = 3 sigma_s of Sec. I is called R here and is
 *    chosen by the caller (the Python wrapper uses ceil(3 sigma_s - 1e-9));
 *  - division guard (paper assumes Q > 0): when |Q| < delta * Qabs, with
 *    Qabs the sum of the absolute values of the terms of Q, the output is
 *    the input pixel and the pixel is counted as guarded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Half-sample symmetric extension of index p into [0, n). */
static long mirror_index(long p, long n)
{
    long period = 2 * n;
    long q = p % period;
    if (q < 0) q += period;
    return (q < n) ? q : (period - 1 - q);
}

int oracle_mirror_index(long p, long n) { return (int)mirror_index(p, n); }

/* ------------------------------------------------------------------------
 * Eq. (1): the Gaussian bilateral filter, evaluated by brute force over the
 * square window [-R, R]^2 with the unnormalised spatial and range Gaussians
 * of Sec. I.
 * ---------------------------------------------------------------------- */
static double exact_bf_pixel(const double *f, long H, long W, long y, long x,
                             double sigma_s, double sigma_r, int R)
{
    const double fi = f[y * W + x];
    double num = 0.0, den = 0.0;
    for (int jy = -R; jy <= R; ++jy) {
        long yy = mirror_index(y - jy, H);
        for (int jx = -R; jx <= R; ++jx) {
            long xx = mirror_index(x - jx, W);
            double t = f[yy * W + xx];
            double gs = exp(-(double)(jy * jy + jx * jx) / (2.0 * sigma_s * sigma_s));
            double gr = exp(-(t - fi) * (t - fi) / (2.0 * sigma_r * sigma_r));
            num += gs * gr * t;
            den += gs * gr;
        }
    }
    return num / den;
}

int oracle_exact_bf(const double *f, int H, int W, double sigma_s, double sigma_r,
                    int R, double *out)
{
    if (!f || !out || H < 1 || W < 1 || R < 0 || !(sigma_s > 0) || !(sigma_r > 0)) return 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x)
            out[y * W + x] = exact_bf_pixel(f, H, W, y, x, sigma_s, sigma_r, R);
    return 0;
}

/* Eq. (1) at the listed flat pixel indices only. */
int oracle_exact_bf_at(const double *f, int H, int W, double sigma_s, double sigma_r,
                       int R, const int64_t *idx, long n_idx, double *out)
{
    if (!f || !out || !idx || H < 1 || W < 1 || R < 0) return 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (long k = 0; k < n_idx; ++k) {
        long p = (long)idx[k];
        out[k] = exact_bf_pixel(f, H, W, p / W, p % W, sigma_s, sigma_r, R);
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Sec. III-A: Chebyshev polynomials and the coefficient fit.
 *   T_l by the three-term recurrence, eq. (12);
 *   zeros xi_k of T_{N+1}, k = 1..N+1;
 *   d_l of the rescaled expansion eq. (18) (the formula that follows it):
 *      d_0 = 1/(N+1) sum_k exp(mu xi_k),
 *      d_l = 2/(N+1) sum_k exp(mu xi_k) T_l(xi_k);
 *   a_{l,n}, the monomial coefficients of T_l, eq. (13), by the recursion
 *   that eq. (12) induces on them;
 *   c_n = mu^{-n} sum_{l=n}^{N} d_l a_{l,n}, eq. (19).
 * ---------------------------------------------------------------------- */

/* Value of T_l(x) by eq. (12). */
double oracle_cheb_T(int l, double x)
{
    if (l == 0) return 1.0;
    double tm1 = 1.0, t = x;
    for (int k = 1; k < l; ++k) {
        double tp1 = 2.0 * x * t - tm1;
        tm1 = t;
        t = tp1;
    }
    return t;
}

/* a[l*(N+1) + n] = coefficient of x^n in T_l(x), l, n = 0..N. */
int oracle_cheb_monomials(int N, double *a)
{
    if (N < 0 || !a) return 1;
    const int M = N + 1;
    memset(a, 0, sizeof(double) * (size_t)M * M);
    a[0] = 1.0;                       /* T_0 = 1 */
    if (N >= 1) a[1 * M + 1] = 1.0;   /* T_1 = x */
    for (int l = 1; l < N; ++l) {     /* T_{l+1} = 2 x T_l - T_{l-1} */
        for (int n = 0; n <= l + 1; ++n) {
            double v = -a[(l - 1) * M + n];
            if (n >= 1) v += 2.0 * a[l * M + (n - 1)];
            a[(l + 1) * M + n] = v;
        }
    }
    return 0;
}

/* Chebyshev nodes, d_l, a_{l,n} and c_n for degree N on [-mu, mu]. */
int oracle_cheb_fit(int N, double mu, double *xi, double *d, double *a, double *c)
{
    if (N < 0 || !(mu > 0) || !xi || !d || !a || !c) return 1;
    const int M = N + 1;
    for (int k = 1; k <= M; ++k)
        xi[k - 1] = cos(M_PI * (2.0 * k - 1.0) / (2.0 * M));
    for (int l = 0; l <= N; ++l) {
        double s = 0.0;
        for (int k = 0; k < M; ++k)
            s += exp(mu * xi[k]) * oracle_cheb_T(l, xi[k]);
        d[l] = (l == 0 ? 1.0 : 2.0) * s / (double)M;
    }
    oracle_cheb_monomials(N, a);
    for (int n = 0; n <= N; ++n) {
        double s = 0.0;
        for (int l = n; l <= N; ++l) s += d[l] * a[l * M + n];
        c[n] = s * pow(mu, -(double)n);
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Eq. (7): spatial Gaussian of one image over the window [-R, R]^2 with
 * symmetric extension.  Two evaluations are provided:
 *   spatial_2d        - the double sum exactly as written;
 *   spatial_separable - the same sum taken one axis at a time (the product
 *                       form of the spatial Gaussian makes this exact up to
 *                       rounding order; the paper relies on separability).
 * ---------------------------------------------------------------------- */
int oracle_spatial_2d(const double *F, int H, int W, double sigma_s, int R, double *out)
{
    if (!F || !out || H < 1 || W < 1 || R < 0) return 1;
#pragma omp parallel for schedule(static)
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            double s = 0.0;
            for (int jy = -R; jy <= R; ++jy)
                for (int jx = -R; jx <= R; ++jx)
                    s += exp(-(double)(jy * jy + jx * jx) / (2.0 * sigma_s * sigma_s)) *
                         F[mirror_index(y - jy, H) * W + mirror_index(x - jx, W)];
            out[y * W + x] = s;
        }
    return 0;
}

int oracle_spatial_separable(const double *F, int H, int W, double sigma_s, int R, double *out)
{
    if (!F || !out || H < 1 || W < 1 || R < 0) return 1;
    double *g = (double *)malloc(sizeof(double) * (2 * (size_t)R + 1));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)H * W);
    if (!g || !tmp) { free(g); free(tmp); return 2; }
    for (int j = -R; j <= R; ++j) g[j + R] = exp(-(double)(j * j) / (2.0 * sigma_s * sigma_s));
    /* along x (within each row) */
#pragma omp parallel for schedule(static)
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            double s = 0.0;
            for (int j = -R; j <= R; ++j) s += g[j + R] * F[y * W + mirror_index(x - j, W)];
            tmp[y * W + x] = s;
        }
    /* along y (within each column) */
#pragma omp parallel for schedule(static)
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            double s = 0.0;
            for (int j = -R; j <= R; ++j) s += g[j + R] * tmp[mirror_index(y - j, H) * W + x];
            out[y * W + x] = s;
        }
    free(g);
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------
 * Recursive Gaussian: the third-order causal + anti-causal filter of
 * I. T. Young and L. J. van Vliet, "Recursive implementation of the
 * Gaussian filter", Signal Processing 44 (1995): coefficients b0..b3 as
 * cubic polynomials in a scale parameter q, B = 1 - (b1 + b2 + b3)/b0.
 * The paper under test computes eq. (7) "using separability and recursion"
 * without fixing a recursive filter; this is the one used here.
 *
 * The scale parameter follows the published fit, q = 0.98711 sigma - 0.96330
 * for sigma >= 2.5 and q = 3.97156 - 4.14554 sqrt(1 - 0.26891 sigma) below.
 *
 * Boundary reading: the 1-D signal is extended by P samples of half-sample
 * mirror on each side; the causal pass starts from the steady state of the
 * first extended sample, the anti-causal pass from the steady state of the
 * last causal output; the central n samples are returned.
 * ---------------------------------------------------------------------- */
static void yvv_from_q(double q, double *b)
{
    double q2 = q * q, q3 = q2 * q;
    double b0 = 1.57825 + 2.44413 * q + 1.4281 * q2 + 0.422205 * q3;
    double b1 = 2.44413 * q + 2.85619 * q2 + 1.26661 * q3;
    double b2 = -(1.4281 * q2 + 1.26661 * q3);
    double b3 = 0.422205 * q3;
    b[0] = b0; b[1] = b1; b[2] = b2; b[3] = b3;
    b[4] = 1.0 - (b1 + b2 + b3) / b0;
}

int oracle_yvv_coeffs(double sigma, double *b /* b0,b1,b2,b3,B */)
{
    if (!(sigma >= 0.5) || !b) return 1;
    double q = (sigma >= 2.5) ? (0.98711 * sigma - 0.96330)
                              : (3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * sigma));
    yvv_from_q(q, b);
    return 0;
}

/* One line of n samples read with stride `stride`, written to out with the same stride. */
static void yvv_line(const double *x, long n, long stride, const double *b, long P, double *out,
                     double *work /* n + 2P */)
{
    const double b0 = b[0], b1 = b[1] / b0, b2 = b[2] / b0, b3 = b[3] / b0, B = b[4];
    const long m = n + 2 * P;
    /* causal pass over the extended signal */
    double x0 = x[mirror_index(-P, n) * stride];
    double w1 = x0, w2 = x0, w3 = x0;
    for (long k = 0; k < m; ++k) {
        double xv = x[mirror_index(k - P, n) * stride];
        double w = B * xv + b1 * w1 + b2 * w2 + b3 * w3;
        work[k] = w;
        w3 = w2; w2 = w1; w1 = w;
    }
    /* anti-causal pass */
    double wl = work[m - 1];
    double y1 = wl, y2 = wl, y3 = wl;
    for (long k = m - 1; k >= 0; --k) {
        double y = B * work[k] + b1 * y1 + b2 * y2 + b3 * y3;
        y3 = y2; y2 = y1; y1 = y;
        if (k >= P && k < P + n) out[(k - P) * stride] = y;
    }
}

int oracle_yvv_1d(const double *x, long n, double sigma, long P, double *out)
{
    double b[5];
    if (!x || !out || n < 1 || P < 0 || oracle_yvv_coeffs(sigma, b)) return 1;
    double *work = (double *)malloc(sizeof(double) * (size_t)(n + 2 * P));
    if (!work) return 2;
    yvv_line(x, n, 1, b, P, out, work);
    free(work);
    return 0;
}

/* Recursive stand-in for eq. (7): rows first, then columns, padding P = R. */
int oracle_spatial_recursive(const double *F, int H, int W, double sigma_s, int R, double *out)
{
    double b[5];
    if (!F || !out || H < 1 || W < 1 || R < 0 || oracle_yvv_coeffs(sigma_s, b)) return 1;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)H * W);
    if (!tmp) return 2;
    int err = 0;
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * (size_t)((H > W ? H : W) + 2 * R));
        if (!work) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(static)
            for (long y = 0; y < H; ++y) yvv_line(F + y * W, W, 1, b, R, tmp + y * W, work);
#pragma omp for schedule(static)
            for (long x = 0; x < W; ++x) yvv_line(tmp + x, H, W, b, R, out + x, work);
            free(work);
        }
    }
    free(tmp);
    return err;
}

/* ------------------------------------------------------------------------
 * Fast algorithm of Sec. II with the Gauss-Chebyshev coefficients, in the
 * order the paper gives (Sec. III-B summary):
 *   centre, eq. (17):  g = f - t_c,  t_c = (L + U)/2;
 *   auxiliary images, eq. (6), n = 0..N+1:
 *       G_n = (g / sigma_r)^n,  F_n = exp(-g^2 / (2 sigma_r^2)) G_n;
 *   spatial filter, eq. (7):  Fbar_n = g_s * F_n;
 *   eq. (8): P = sigma_r sum_{n=0}^{N} c_n G_n Fbar_{n+1};
 *   eq. (9): Q = sum_{n=0}^{N} c_n G_n Fbar_n;
 *   eq. (10) and un-centring: out = P / Q + t_c.
 * spatial_mode: 0 = eq. (7) evaluated separably, 1 = recursive stand-in,
 *               2 = eq. (7) as the literal double sum.
 * P_out, Q_out, Qabs_out, Pabs_out may be NULL (Qabs / Pabs: sums of the
 * absolute values of the terms of Q / P).  Returns the number of guarded
 * pixels in *n_guard (may be NULL).
 * ---------------------------------------------------------------------- */
int oracle_gcf(const double *f, int H, int W, double sigma_s, double sigma_r, int N, int R,
               double L, double U, const double *c, double delta, int spatial_mode,
               double *out, double *P_out, double *Q_out, double *Qabs_out, double *Pabs_out,
               long *n_guard)
{
    if (!f || !out || !c || H < 1 || W < 1 || N < 0 || R < 0 || !(sigma_r > 0) || !(sigma_s > 0))
        return 1;
    const long px = (long)H * W;
    const int C = N + 2;
    const double tc = 0.5 * (L + U);
    double *G = (double *)malloc(sizeof(double) * (size_t)C * px);
    double *F = (double *)malloc(sizeof(double) * (size_t)C * px);
    double *Fb = (double *)malloc(sizeof(double) * (size_t)C * px);
    if (!G || !F || !Fb) { free(G); free(F); free(Fb); return 2; }

    /* eqs. (17) and (6) */
    for (long i = 0; i < px; ++i) {
        double g = f[i] - tc;
        double e = exp(-g * g / (2.0 * sigma_r * sigma_r));
        for (int n = 0; n < C; ++n) {
            double Gn = pow(g / sigma_r, (double)n);
            G[(long)n * px + i] = Gn;
            F[(long)n * px + i] = e * Gn;
        }
    }
    /* eq. (7) */
    int err = 0;
    for (int n = 0; n < C && !err; ++n) {
        const double *Fn = F + (long)n * px;
        double *Fbn = Fb + (long)n * px;
        if (spatial_mode == 0) err = oracle_spatial_separable(Fn, H, W, sigma_s, R, Fbn);
        else if (spatial_mode == 1) err = oracle_spatial_recursive(Fn, H, W, sigma_s, R, Fbn);
        else err = oracle_spatial_2d(Fn, H, W, sigma_s, R, Fbn);
    }
    long guarded = 0;
    if (!err) {
        /* eqs. (8), (9), (10) */
        for (long i = 0; i < px; ++i) {
            double P = 0.0, Q = 0.0, Qabs = 0.0, Pabs = 0.0;
            for (int n = 0; n <= N; ++n) {
                double cg = c[n] * G[(long)n * px + i];
                double pt = cg * Fb[(long)(n + 1) * px + i];
                P += pt;
                Pabs += fabs(pt);
                double q = cg * Fb[(long)n * px + i];
                Q += q;
                Qabs += fabs(q);
            }
            P *= sigma_r;
            Pabs *= sigma_r;
            if (fabs(Q) < delta * Qabs || Qabs == 0.0) {
                out[i] = f[i];
                ++guarded;
            } else {
                out[i] = P / Q + tc;
            }
            if (P_out) P_out[i] = P;
            if (Q_out) Q_out[i] = Q;
            if (Qabs_out) Qabs_out[i] = Qabs;
            if (Pabs_out) Pabs_out[i] = Pabs;
        }
    }
    if (n_guard) *n_guard = guarded;
    free(G);
    free(F);
    free(Fb);
    return err;
}

/* The same fast algorithm evaluated at listed pixels only, with eq. (7)
 * taken as the literal double sum at each listed pixel.  Used to check
 * large images at sampled outputs. */
int oracle_gcf_at(const double *f, int H, int W, double sigma_s, double sigma_r, int N, int R,
                  double L, double U, const double *c, double delta, const int64_t *idx,
                  long n_idx, double *out, double *P_out, double *Q_out)
{
    if (!f || !out || !c || !idx || H < 1 || W < 1 || N < 0 || R < 0) return 1;
    const int C = N + 2;
    const double tc = 0.5 * (L + U);
    int err = 0;
#pragma omp parallel
    {
        double *Fb = (double *)malloc(sizeof(double) * (size_t)C);
        if (!Fb) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (long k = 0; k < n_idx; ++k) {
                long p = (long)idx[k], y = p / W, x = p % W;
                for (int n = 0; n < C; ++n) Fb[n] = 0.0;
                for (int jy = -R; jy <= R; ++jy) {
                    long yy = mirror_index(y - jy, H);
                    for (int jx = -R; jx <= R; ++jx) {
                        long xx = mirror_index(x - jx, W);
                        double gs = exp(-(double)(jy * jy + jx * jx) / (2.0 * sigma_s * sigma_s));
                        double g = f[yy * W + xx] - tc;
                        double e = exp(-g * g / (2.0 * sigma_r * sigma_r));
                        for (int n = 0; n < C; ++n)
                            Fb[n] += gs * e * pow(g / sigma_r, (double)n);
                    }
                }
                double gi = f[p] - tc, P = 0.0, Q = 0.0, Qabs = 0.0;
                for (int n = 0; n <= N; ++n) {
                    double cg = c[n] * pow(gi / sigma_r, (double)n);
                    P += cg * Fb[n + 1];
                    Q += cg * Fb[n];
                    Qabs += fabs(cg * Fb[n]);
                }
                P *= sigma_r;
                out[k] = (fabs(Q) < delta * Qabs || Qabs == 0.0) ? f[p] : P / Q + tc;
                if (P_out) P_out[k] = P;
                if (Q_out) Q_out[k] = Q;
            }
            free(Fb);
        }
    }
    return err;
}

/* ------------------------------------------------------------------------
 * Eq. (4) with the coefficients of eq. (19), used directly as the range
 * kernel in eq. (1) (after the centring of eq. (17)):
 *   k(tau, t) = exp(-tau^2/2sr^2) exp(-t^2/2sr^2) sum_n c_n (tau t / sr^2)^n,
 *   out(i) = sum_j g_s(j) k(g(i), g(i-j)) g(i-j) / sum_j g_s(j) k(...) + t_c.
 * Exchanging the order of summation (Sec. II) turns this into eqs. (8)-(10)
 * exactly, so it must agree with oracle_gcf to rounding.  den_out (may be
 * NULL) receives the denominator sum_j g_s(j) k(g(i), g(i-j)), which the same
 * exchange equals exp(-g(i)^2/2sr^2) times Q of eq. (9).
 * ---------------------------------------------------------------------- */
int oracle_gcf_kernel_direct(const double *f, int H, int W, double sigma_s, double sigma_r,
                             int N, int R, double L, double U, const double *c, double *out,
                             double *den_out)
{
    if (!f || !out || !c || H < 1 || W < 1 || N < 0 || R < 0) return 1;
    const double tc = 0.5 * (L + U);
#pragma omp parallel for schedule(dynamic, 1)
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            double tau = f[y * W + x] - tc;
            double num = 0.0, den = 0.0;
            for (int jy = -R; jy <= R; ++jy)
                for (int jx = -R; jx <= R; ++jx) {
                    double t = f[mirror_index(y - jy, H) * W + mirror_index(x - jx, W)] - tc;
                    double gs = exp(-(double)(jy * jy + jx * jx) / (2.0 * sigma_s * sigma_s));
                    double poly = 0.0;
                    for (int n = 0; n <= N; ++n)
                        poly += c[n] * pow(tau * t / (sigma_r * sigma_r), (double)n);
                    double k = exp(-tau * tau / (2.0 * sigma_r * sigma_r)) *
                               exp(-t * t / (2.0 * sigma_r * sigma_r)) * poly;
                    num += gs * k * t;
                    den += gs * k;
                }
            out[y * W + x] = num / den + tc;
            if (den_out) den_out[y * W + x] = den;
        }
    return 0;
}

int oracle_have_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}
