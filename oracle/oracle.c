/*
 * FP64 CPU oracle for the long-range ("history") part of the 2D modified Helmholtz layer and
 * volume potentials.  TEST INFRASTRUCTURE ONLY: it is called by the tests, by the smoke check
 * and by the benchmark's CPU-baseline leg, never by the library's product path, and it shares no
 * code, header, table or constant with the CUDA implementation.
 *
 * What it computes (Section 2.1, eqs. H_ker and sl_sh; Section 5.1, eq. sh):
 *
 *   u_H(x_i) = sum_j q_j G_H(|x_i - y_j|),
 *   G_H(r)   = int_delta^inf exp(-r^2/(4t) - alpha^2 t) / (4 pi t) dt
 *            = (1/(2pi)^2) int_{R^2} exp(-delta(alpha^2+|k|^2)) / (alpha^2+|k|^2) e^{ik.x} dk
 *            = (1/(2pi)) int_0^inf exp(-delta(alpha^2+k^2)) / (alpha^2+k^2) J0(k r) k dk.
 *
 * The last line is the radial (Hankel) form of the 2-D inverse Fourier transform of a radial
 * symbol.  G_H is obtained from it by composite Gauss-Legendre quadrature in k (J0 from the C
 * library), tabulated as piecewise Chebyshev series on [0, r_max], and summed directly over all
 * source/target pairs with Neumaier-compensated FP64 summation.
 *
 * Second oracle: the paper's own discrete formula (Section 5.2, eqs. disrete_sigma_hat and
 * sh_fourier) on the symmetric mode set |m_x|,|m_y| <= M with Delta k = 2 pi / P:
 *
 *   c_m    = sum_j q_j exp(-i k_m . y_j),
 *   u(x)   = (Delta k)^2/(2pi)^2 sum_m exp(-delta(alpha^2+|k_m|^2))/(alpha^2+|k_m|^2) c_m e^{ik_m.x}
 *
 * evaluated as plain double loops.
 *
 * Double layer (Section 2, eq. dlp; its split D = D_L + D_H in Section 2.1; Section 5.1, the D_H
 * formula after eq. kmax_dlp): a dipole source at y with vector strength s = mu w nu contributes
 *
 *   s . grad_y G_H(x - y) = F_D(|x - y|) (x - y) . s,
 *   F_D(r) = -G_H'(r) / r = int_delta^inf exp(-r^2/(4t) - alpha^2 t) / (8 pi t^2) dt
 *          = (1/(2pi)) int_0^inf exp(-delta(alpha^2+k^2)) / (alpha^2+k^2) k^2 J1(k r)/r dk,
 *
 * tabulated the same way (J1 from the C library, k/2 at r = 0).  In the discrete formula the
 * dipole's Fourier coefficient is -i (k . s) exp(-i k . y): differentiating exp(ik.(x-y)) with
 * respect to the source point.  Pins for both live in the tests (closed forms, identities,
 * brute force); none of them re-types these formulas.
 */
#define _DEFAULT_SOURCE 1 /* j0() is POSIX, not ISO C */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ---------------------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1,1]: Newton iteration on the three-term Legendre recurrence.      */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ---------------------------------------------------------------------------------------- */
/* Hankel quadrature of G_H: nodes k_i and combined weights c_i with G_H(r) = sum c_i J0(k_i r) */
typedef struct {
    int n, kind; /* kind 0: G_H = sum c_i J0(k_i r); kind 1: F_D = sum c_i J1(k_i r) / r */
    double *k, *c;
} hankel_rule;

#define OR_GL_N 24

/* Panels on [0, k_c], k_c = sqrt(45/delta) (exp(-delta k_c^2) ~ 3e-20).  A panel starting at a
 * has length min(sqrt(a^2+alpha^2), 2pi/r_max, 1/sqrt(delta)): the first bound keeps the poles
 * of 1/(alpha^2+k^2) at +-i alpha well outside each panel's Bernstein ellipse, the second puts at
 * most one period of J0(k r) in a panel, the third resolves the Gaussian factor. */
static int hankel_build(double alpha, double delta, double rmax, int kind, hankel_rule *h)
{
    h->kind = kind;
    double xg[OR_GL_N], wg[OR_GL_N];
    gauss_legendre(OR_GL_N, xg, wg);
    double kc = sqrt(45.0 / delta);
    double cap = 1.0 / sqrt(delta);
    if (rmax > 0 && 2.0 * OR_PI / rmax < cap) cap = 2.0 * OR_PI / rmax;
    /* count panels */
    int np = 0;
    for (double a = 0.0; a < kc; ++np) {
        double L = sqrt(a * a + alpha * alpha);
        if (L > cap) L = cap;
        a += L;
    }
    h->n = np * OR_GL_N;
    h->k = (double *)malloc(sizeof(double) * h->n);
    h->c = (double *)malloc(sizeof(double) * h->n);
    if (!h->k || !h->c) return -1;
    int p = 0;
    for (double a = 0.0; a < kc; ++p) {
        double L = sqrt(a * a + alpha * alpha);
        if (L > cap) L = cap;
        for (int i = 0; i < OR_GL_N; ++i) {
            double k = a + 0.5 * L * (xg[i] + 1.0);
            double s = alpha * alpha + k * k;
            h->k[p * OR_GL_N + i] = k;
            h->c[p * OR_GL_N + i] =
                0.5 * L * wg[i] * exp(-delta * s) / s * k * (kind ? k : 1.0) / (2.0 * OR_PI);
        }
        a += L;
    }
    return 0;
}

static void hankel_free(hankel_rule *h)
{
    free(h->k);
    free(h->c);
}

static double hankel_eval(const hankel_rule *h, double r)
{
    /* Neumaier-compensated sum of c_i J0(k_i r), or of c_i J1(k_i r) / r (k_i / 2 at r = 0) */
    double s = 0.0, comp = 0.0;
    for (int i = 0; i < h->n; ++i) {
        double b;
        if (h->kind == 0) b = j0(h->k[i] * r);
        else b = r > 0.0 ? j1(h->k[i] * r) / r : 0.5 * h->k[i];
        double t = h->c[i] * b;
        double u = s + t;
        if (fabs(s) >= fabs(t)) comp += (s - u) + t;
        else comp += (t - u) + s;
        s = u;
    }
    return s + comp;
}

/* Direct Hankel-quadrature value of G_H (kind 0) or F_D (kind 1) at n radii (no table). */
int or_kernel_hankel(double alpha, double delta, int kind, int64_t n, const double *r, double *out)
{
    double rmax = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (r[i] > rmax) rmax = r[i];
    hankel_rule h;
    if (hankel_build(alpha, delta, rmax, kind, &h)) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) out[i] = hankel_eval(&h, r[i]);
    hankel_free(&h);
    return 0;
}

int or_gh_hankel(double alpha, double delta, int64_t n, const double *r, double *out)
{
    return or_kernel_hankel(alpha, delta, 0, n, r, out);
}

/* ---------------------------------------------------------------------------------------- */
/* Piecewise Chebyshev table of G_H (or F_D) on [0, r_max].                                             */
#define OR_CHEB_N 25 /* points (degree 24) */

typedef struct {
    double alpha, delta, rmax, g0;
    int npan;
    double *edge; /* npan+1 panel edges */
    double *coef; /* npan x OR_CHEB_N Chebyshev coefficients */
} or_table;

static void cheb_coeffs(const double *f, double *c)
{
    /* f sampled at x_j = cos(pi (j+1/2)/n); c_k = (2/n) sum_j f_j cos(k pi (j+1/2)/n) */
    const int n = OR_CHEB_N;
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += f[j] * cos(OR_PI * k * (j + 0.5) / n);
        c[k] = 2.0 * s / n;
    }
    c[0] *= 0.5;
}

static double cheb_clenshaw(const double *c, double x)
{
    double b1 = 0.0, b2 = 0.0;
    for (int k = OR_CHEB_N - 1; k >= 1; --k) {
        double b0 = 2.0 * x * b1 - b2 + c[k];
        b2 = b1;
        b1 = b0;
    }
    return x * b1 - b2 + c[0];
}

typedef struct {
    double a, b;
    double c[OR_CHEB_N];
} pan_t;

/* Adaptive bisection: accept a panel when its three highest coefficients are below
 * tol_rel * G_H(0), or when it is narrower than sqrt(delta)/256 (below that width G_H is a
 * low-degree polynomial and a larger tail is quadrature noise).  Initial panels: [0, s], then
 * geometric [s 2^i, s 2^{i+1}] (s = sqrt(delta)) up to r_max. */
void *or_table_create_kind(double alpha, double delta, double rmax, double tol_rel, int kind)
{
    if (!(alpha > 0) || !(delta > 0) || !(rmax > 0) || (kind != 0 && kind != 1)) return NULL;
    hankel_rule h;
    if (hankel_build(alpha, delta, rmax, kind, &h)) return NULL;
    double g0 = hankel_eval(&h, 0.0);
    double thr = tol_rel * g0;

    int cap = 64, n = 0;
    pan_t *todo = (pan_t *)malloc(sizeof(pan_t) * cap);
    double s = sqrt(delta);
    double a = 0.0, b = s < rmax ? s : rmax;
    for (;;) {
        if (n == cap) { cap *= 2; todo = (pan_t *)realloc(todo, sizeof(pan_t) * cap); }
        todo[n].a = a;
        todo[n].b = b;
        ++n;
        if (b >= rmax) break;
        a = b;
        b = 2.0 * b < rmax ? 2.0 * b : rmax;
    }
    /* iterate: evaluate all pending panels in parallel, split those not converged */
    int acc_cap = 256, nacc = 0;
    pan_t *acc = (pan_t *)malloc(sizeof(pan_t) * acc_cap);
    int depth = 0;
    const double min_width = s / 256.0;
    while (n > 0 && depth < 40) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int p = 0; p < n; ++p) {
            double f[OR_CHEB_N];
            for (int j = 0; j < OR_CHEB_N; ++j) {
                double x = cos(OR_PI * (j + 0.5) / OR_CHEB_N);
                double r = 0.5 * (todo[p].a + todo[p].b) + 0.5 * (todo[p].b - todo[p].a) * x;
                f[j] = hankel_eval(&h, r);
            }
            cheb_coeffs(f, todo[p].c);
        }
        int nn = 0;
        pan_t *next = (pan_t *)malloc(sizeof(pan_t) * (2 * n + 1));
        for (int p = 0; p < n; ++p) {
            double tail = fabs(todo[p].c[OR_CHEB_N - 1]);
            if (fabs(todo[p].c[OR_CHEB_N - 2]) > tail) tail = fabs(todo[p].c[OR_CHEB_N - 2]);
            if (fabs(todo[p].c[OR_CHEB_N - 3]) > tail) tail = fabs(todo[p].c[OR_CHEB_N - 3]);
            if (tail <= thr || depth == 39 || todo[p].b - todo[p].a <= min_width) {
                if (nacc == acc_cap) { acc_cap *= 2; acc = (pan_t *)realloc(acc, sizeof(pan_t) * acc_cap); }
                acc[nacc++] = todo[p];
            } else {
                double m = 0.5 * (todo[p].a + todo[p].b);
                next[nn].a = todo[p].a; next[nn].b = m; ++nn;
                next[nn].a = m; next[nn].b = todo[p].b; ++nn;
            }
        }
        free(todo);
        todo = next;
        n = nn;
        ++depth;
    }
    free(todo);
    hankel_free(&h);
    /* sort accepted panels by left edge (insertion sort; counts are small) */
    for (int i = 1; i < nacc; ++i) {
        pan_t t = acc[i];
        int j = i - 1;
        while (j >= 0 && acc[j].a > t.a) { acc[j + 1] = acc[j]; --j; }
        acc[j + 1] = t;
    }
    or_table *T = (or_table *)calloc(1, sizeof(or_table));
    T->alpha = alpha;
    T->delta = delta;
    T->rmax = rmax;
    T->g0 = g0;
    T->npan = nacc;
    T->edge = (double *)malloc(sizeof(double) * (nacc + 1));
    T->coef = (double *)malloc(sizeof(double) * nacc * OR_CHEB_N);
    for (int i = 0; i < nacc; ++i) {
        T->edge[i] = acc[i].a;
        memcpy(T->coef + (size_t)i * OR_CHEB_N, acc[i].c, sizeof(double) * OR_CHEB_N);
    }
    T->edge[nacc] = acc[nacc - 1].b;
    free(acc);
    return T;
}

void *or_table_create(double alpha, double delta, double rmax, double tol_rel)
{
    return or_table_create_kind(alpha, delta, rmax, tol_rel, 0);
}

void or_table_free(void *t)
{
    or_table *T = (or_table *)t;
    if (!T) return;
    free(T->edge);
    free(T->coef);
    free(T);
}

int or_table_npanels(const void *t) { return ((const or_table *)t)->npan; }
double or_table_g0(const void *t) { return ((const or_table *)t)->g0; }

static inline double table_eval(const or_table *T, double r)
{
    if (r >= T->edge[T->npan]) r = T->edge[T->npan]; /* callers keep r <= r_max */
    int lo = 0, hi = T->npan - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (T->edge[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    double a = T->edge[lo], b = T->edge[lo + 1];
    double x = (2.0 * r - a - b) / (b - a);
    return cheb_clenshaw(T->coef + (size_t)lo * OR_CHEB_N, x);
}

int or_table_eval(const void *t, int64_t n, const double *r, double *out)
{
    const or_table *T = (const or_table *)t;
    for (int64_t i = 0; i < n; ++i) {
        if (!(r[i] >= 0.0) || r[i] > T->rmax * (1.0 + 1e-12)) return -1;
        out[i] = table_eval(T, r[i]);
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Direct pair sum u_i = sum_j q_j G_H(|x_i - y_j|), Neumaier-compensated, sources in index   */
/* order; also s_i = sum_j |q_j| G_H(|x_i - y_j|) (the conditioning scale of u_i).             */
int or_direct_sum(const void *t, int64_t ns, const double *xs, const double *ys, const double *q,
                  int64_t nt, const double *xt, const double *yt, double *u, double *s_abs)
{
    const or_table *T = (const or_table *)t;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t i = 0; i < nt; ++i) {
        double sum = 0.0, comp = 0.0, sa = 0.0, ca = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            double dx = xt[i] - xs[j], dy = yt[i] - ys[j];
            double r = sqrt(dx * dx + dy * dy);
            if (r > T->rmax * (1.0 + 1e-12)) { bad = 1; continue; }
            double g = table_eval(T, r);
            double v = q[j] * g, nsum = sum + v;
            if (fabs(sum) >= fabs(v)) comp += (sum - nsum) + v;
            else comp += (v - nsum) + sum;
            sum = nsum;
            double va = fabs(q[j]) * g, na = sa + va;
            if (fabs(sa) >= fabs(va)) ca += (sa - na) + va;
            else ca += (va - na) + sa;
            sa = na;
        }
        u[i] = sum + comp;
        if (s_abs) s_abs[i] = sa + ca;
    }
    return bad ? -1 : 0;
}

/* Direct pair sum of the double layer: u_i = sum_d F_D(|x_i - y_d|) (x_i - y_d) . s_d with
 * s_d = (sx_d, sy_d) = mu_d w_d nu_d (t: a kind-1 table), Neumaier-compensated, sources in index
 * order; s_abs_i = sum_d F_D(r) r |s_d| (the conditioning scale of u_i). */
int or_direct_sum_dl(const void *t, int64_t nd, const double *xd, const double *yd,
                     const double *sx, const double *sy, int64_t nt, const double *xt,
                     const double *yt, double *u, double *s_abs)
{
    const or_table *T = (const or_table *)t;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t i = 0; i < nt; ++i) {
        double sum = 0.0, comp = 0.0, sa = 0.0, ca = 0.0;
        for (int64_t j = 0; j < nd; ++j) {
            double dx = xt[i] - xd[j], dy = yt[i] - yd[j];
            double r = sqrt(dx * dx + dy * dy);
            if (r > T->rmax * (1.0 + 1e-12)) { bad = 1; continue; }
            double f = table_eval(T, r);
            double v = f * (dx * sx[j] + dy * sy[j]), nsum = sum + v;
            if (fabs(sum) >= fabs(v)) comp += (sum - nsum) + v;
            else comp += (v - nsum) + sum;
            sum = nsum;
            double va = f * r * sqrt(sx[j] * sx[j] + sy[j] * sy[j]), na = sa + va;
            if (fabs(sa) >= fabs(va)) ca += (sa - na) + va;
            else ca += (va - na) + sa;
            sa = na;
        }
        u[i] = sum + comp;
        if (s_abs) s_abs[i] = sa + ca;
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Discrete formula of Section 5.2 on modes |m_x|,|m_y| <= M, Delta k = 2pi/P, coordinates     */
/* taken relative to (cx, cy) (a common shift; the result does not depend on it).              */
/* Charges q at (xs, ys) and dipoles s = (sx, sy) at (xd, yd) (nd may be 0); a dipole's
 * coefficient is -i (k . s) exp(-i k . y). */
int or_discrete_sum_dl(double alpha, double delta, double P, int64_t M, double cx, double cy,
                       int64_t ns, const double *xs, const double *ys, const double *q,
                       int64_t nd, const double *xd, const double *yd, const double *sx,
                       const double *sy, int64_t nt, const double *xt, const double *yt,
                       double *u)
{
    const int64_t nm = 2 * M + 1;
    const double dk = 2.0 * OR_PI / P;
    double complex *c = (double complex *)calloc((size_t)(nm * nm), sizeof(double complex));
    if (!c) return -1;
    /* c[mx][my] = sum_j q_j exp(-i dk (mx (x_j-cx) + my (y_j-cy))) */
#pragma omp parallel
    {
        double complex *cl = (double complex *)calloc((size_t)(nm * nm), sizeof(double complex));
        double complex *ex = (double complex *)malloc(sizeof(double complex) * nm);
        double complex *ey = (double complex *)malloc(sizeof(double complex) * nm);
#pragma omp for schedule(static)
        for (int64_t j = 0; j < ns; ++j) {
            for (int64_t m = -M; m <= M; ++m) {
                ex[m + M] = cexp(-I * dk * (double)m * (xs[j] - cx));
                ey[m + M] = cexp(-I * dk * (double)m * (ys[j] - cy));
            }
            for (int64_t a = 0; a < nm; ++a) {
                double complex qa = q[j] * ex[a];
                for (int64_t b = 0; b < nm; ++b) cl[a * nm + b] += qa * ey[b];
            }
        }
#pragma omp for schedule(static)
        for (int64_t j = 0; j < nd; ++j) {
            for (int64_t m = -M; m <= M; ++m) {
                ex[m + M] = cexp(-I * dk * (double)m * (xd[j] - cx));
                ey[m + M] = cexp(-I * dk * (double)m * (yd[j] - cy));
            }
            for (int64_t a = 0; a < nm; ++a) {
                const double kx = dk * (double)(a - M);
                for (int64_t b = 0; b < nm; ++b) {
                    const double ky = dk * (double)(b - M);
                    cl[a * nm + b] += -I * (kx * sx[j] + ky * sy[j]) * ex[a] * ey[b];
                }
            }
        }
#pragma omp critical
        for (int64_t i = 0; i < nm * nm; ++i) c[i] += cl[i];
        free(cl);
        free(ex);
        free(ey);
    }
    /* multiply by (dk/2pi)^2 * exp(-delta(alpha^2+k^2))/(alpha^2+k^2) */
    for (int64_t a = 0; a < nm; ++a)
        for (int64_t b = 0; b < nm; ++b) {
            double kx = dk * (double)(a - M), ky = dk * (double)(b - M);
            double s = alpha * alpha + kx * kx + ky * ky;
            c[a * nm + b] *= (dk / (2.0 * OR_PI)) * (dk / (2.0 * OR_PI)) * exp(-delta * s) / s;
        }
#pragma omp parallel
    {
        double complex *ex = (double complex *)malloc(sizeof(double complex) * nm);
        double complex *ey = (double complex *)malloc(sizeof(double complex) * nm);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < nt; ++i) {
            for (int64_t m = -M; m <= M; ++m) {
                ex[m + M] = cexp(I * dk * (double)m * (xt[i] - cx));
                ey[m + M] = cexp(I * dk * (double)m * (yt[i] - cy));
            }
            double complex acc = 0.0;
            for (int64_t a = 0; a < nm; ++a) {
                double complex row = 0.0;
                for (int64_t b = 0; b < nm; ++b) row += c[a * nm + b] * ey[b];
                acc += row * ex[a];
            }
            u[i] = creal(acc);
        }
        free(ex);
        free(ey);
    }
    free(c);
    return 0;
}

int or_discrete_sum(double alpha, double delta, double P, int64_t M, double cx, double cy,
                    int64_t ns, const double *xs, const double *ys, const double *q,
                    int64_t nt, const double *xt, const double *yt, double *u)
{
    return or_discrete_sum_dl(alpha, delta, P, M, cx, cy, ns, xs, ys, q, 0, NULL, NULL, NULL,
                              NULL, nt, xt, yt, u);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
