/*
 * yk_api.cu — host side of the C ABI declared in include/yk.h: parameter selection, device
 * buffers, host/device pointer handling and the launch sequence of one evaluation.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "yk_internal.h"

using yk::FftStages;

namespace {

thread_local std::string g_last_error;

yk_status fail(yk_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

yk_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(YK_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(YK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define YK_CU(call, what)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);                                      \
    } while (0)

constexpr double kPi = 3.14159265358979323846;

/* ------------------------------------------------------------------------------------------ */
/* special functions for the parameter rules                                                   */

/* exponential integral E1(x), x > 0: power series for x <= 1 (Abramowitz-Stegun 5.1.11),
 * continued fraction for x > 1 (A-S 5.1.22) evaluated by the modified Lentz method */
double expint_e1(double x)
{
    if (x <= 1.0) {
        const double euler = 0.57721566490153286061;
        double sum = 0.0, term = 1.0;
        for (int k = 1; k < 200; ++k) {
            term *= -x / k;
            const double add = -term / k;
            sum += add;
            if (std::fabs(add) < 1e-18 * std::fabs(sum)) break;
        }
        return -euler - std::log(x) + sum;
    }
    /* E1(x) = e^{-x} / (x + 1/(1 + 1/(x + 2/(1 + 2/(x + ...))))) in the even form
     * e^{-x} * 1/(x+1- 1^2/(x+3- 2^2/(x+5- ...))) */
    const double tiny = 1e-300;
    double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 10000; ++i) {
        const double an = -(double)i * i;
        b += 2.0;
        d = 1.0 / (an * d + b);
        c = b + an / c;
        const double del = c * d;
        h *= del;
        if (std::fabs(del - 1.0) < 1e-16) break;
    }
    return h * std::exp(-x);
}

/* modified Bessel function K_nu(x), x > 0, from K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
 * by the trapezoidal rule (step 1/16; the integrand is analytic in the strip |Im t| < pi/2, so the
 * error is of order exp(-pi^2 16)), in long double, up to where x cosh t exceeds 11000 */
double bessel_k(int nu, double x)
{
    const long double h = 1.0L / 16.0L, xl = x;
    long double sum = 0.5L * expl(-xl);
    for (int i = 1;; ++i) {
        const long double t = h * i, c = coshl(t);
        if (xl * c > 11000.0L) break;
        sum += expl(-xl * c) * coshl(nu * t);
    }
    return (double)(h * sum);
}

/* Gauss-Legendre nodes/weights on [-1, 1] (Newton on the Legendre recurrence) */
void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                const double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            const double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* G_H(r) = int_delta^inf exp(-r^2/(4t) - alpha^2 t) / (4 pi t) dt with t = delta e^s:
 * (1/4pi) int_0^S exp(-r^2 e^{-s}/(4 delta) - alpha^2 delta e^s) ds, composite Gauss-Legendre.
 * Used only to size the period (the decay length), so a few digits suffice. */
double gh_time_integral(double alpha, double delta, double r)
{
    const double a2d = alpha * alpha * delta;
    const double S = std::log(60.0 / a2d) + 2.0; /* alpha^2 delta e^S >= 60 */
    /* 16-point rule in fixed storage, built once (no heap use on this path) */
    struct Rule {
        double x[16], w[16];
        Rule() { gauss_legendre(16, x, w); }
    };
    static const Rule rule;
    const double *gx = rule.x, *gw = rule.w;
    const int npan = 400;
    const double L = (S > 1.0 ? S : 1.0) / npan;
    double sum = 0.0;
    for (int p = 0; p < npan; ++p)
        for (int i = 0; i < 16; ++i) {
            const double s = L * (p + 0.5 * (gx[i] + 1.0));
            sum += 0.5 * L * gw[i] *
                   std::exp(-r * r * std::exp(-s) / (4.0 * delta) - a2d * std::exp(s));
        }
    return sum / (4.0 * kPi);
}

/* smallest k with E1(delta (alpha^2 + k^2)) <= eps E1(delta alpha^2) (tail of the radial Fourier
 * integral relative to G_H(0); reading of eq. kmax relative to the size of G_H) */
double kmax_relative(double alpha, double delta, double eps)
{
    const double x0 = delta * alpha * alpha;
    const double target = eps * expint_e1(x0);
    double lo = x0, hi = x0 + 1.0;
    while (expint_e1(hi) > target) hi = x0 + 2.0 * (hi - x0);
    for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (expint_e1(mid) > target) lo = mid;
        else hi = mid;
    }
    const double k2 = hi / delta - alpha * alpha;
    return k2 > 0.0 ? std::sqrt(k2) : 0.0;
}

/* eq. kmax as printed: exp(-delta (alpha^2 + k^2)) <= eps, zero when delta alpha^2 >= ln(1/eps) */
double kmax_paper(double alpha, double delta, double eps)
{
    const double v = (std::log(1.0 / eps) - delta * alpha * alpha) / delta;
    return v > 0.0 ? std::sqrt(v) : 0.0;
}

/* eq. kmax_dlp as printed: k exp(-delta (alpha^2 + k^2)) <= eps beyond k (0 if it holds for all k) */
double kmax_dlp_paper(double alpha, double delta, double eps)
{
    auto f = [&](double k) { return k * std::exp(-delta * (alpha * alpha + k * k)); };
    const double kpk = 1.0 / std::sqrt(2.0 * delta); /* maximiser of k exp(-delta k^2) */
    if (f(kpk) <= eps) return 0.0;
    double lo = kpk, hi = 2.0 * kpk;
    while (f(hi) > eps) {
        lo = hi;
        hi *= 2.0;
    }
    for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (f(mid) > eps) lo = mid;
        else hi = mid;
    }
    return hi;
}

/* int_k^inf exp(-delta s^2) s^2 / (alpha^2 + s^2) ds (the common factor exp(-delta alpha^2)
 * dropped): composite 16-point Gauss-Legendre on panels no wider than 1/(4 sqrt(delta)) and half
 * the distance to the poles at +-i alpha, up to where exp(-delta s^2) has fallen by e^{-60} */
double dlp_tail(double alpha, double delta, double k)
{
    struct Rule {
        double x[16], w[16];
        Rule() { gauss_legendre(16, x, w); }
    };
    static const Rule rule;
    const double K = std::sqrt(k * k + 60.0 / delta), cap = 0.25 / std::sqrt(delta);
    double sum = 0.0;
    for (double a = k; a < K;) {
        double L = std::min(cap, 0.5 * std::sqrt(a * a + alpha * alpha));
        if (a + L > K) L = K - a;
        for (int i = 0; i < 16; ++i) {
            const double t = a + 0.5 * L * (rule.x[i] + 1.0), t2 = t * t;
            sum += 0.5 * L * rule.w[i] * std::exp(-delta * t2) * t2 / (alpha * alpha + t2);
        }
        a += L;
    }
    return sum;
}

/* reading of eq. kmax_dlp relative to the kernel's size: the radial integrand of -G_H' carries
 * one more factor of k than G_H's; its tail beyond k_max is at most eps times its whole integral */
double kmax_dlp_relative(double alpha, double delta, double eps)
{
    const double target = eps * dlp_tail(alpha, delta, 0.0);
    double lo = 0.0, hi = 1.0 / std::sqrt(delta);
    while (dlp_tail(alpha, delta, hi) > target) {
        lo = hi;
        hi *= 2.0;
    }
    for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (dlp_tail(alpha, delta, mid) > target) lo = mid;
        else hi = mid;
    }
    return hi;
}

/* decay length: smallest r with G_H(r') <= eps G_H(0) for all r' >= r (G_H decreases in r) */
double decay_length(double alpha, double delta, double eps)
{
    const double g0 = expint_e1(alpha * alpha * delta) / (4.0 * kPi);
    double lo = 0.0, hi = std::max(1.0 / alpha, std::sqrt(delta));
    while (gh_time_integral(alpha, delta, hi) > eps * g0) {
        lo = hi;
        hi *= 2.0;
    }
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (gh_time_integral(alpha, delta, mid) > eps * g0) lo = mid;
        else hi = mid;
    }
    return hi;
}

/* Fourier transform of the window: phi_hat(xi) = int_{-w/2}^{w/2} phi(z) cos(xi z) dz with
 * z = (w/2) sin(theta), which removes the square-root edge behaviour of phi */
double window_ft(double xi, int w, double beta)
{
    static thread_local std::vector<double> gx, gw;
    if (gx.empty()) {
        gx.resize(128);
        gw.resize(128);
        gauss_legendre(128, gx.data(), gw.data());
    }
    const double half = 0.5 * w;
    double sum = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
        const double th = 0.25 * kPi * (gx[i] + 1.0);
        sum += 0.25 * kPi * gw[i] * std::exp(beta * (std::cos(th) - 1.0)) *
               std::cos(xi * half * std::sin(th)) * half * std::cos(th);
    }
    return 2.0 * sum;
}

/* per-tap window polynomials: tap a covers z = u - w/2 + a, u in [0, 1); with x = 2u - 1 the
 * window there is interpolated at deg+1 Chebyshev points and the series converted to powers of
 * x, all in long double; mono[k * w + a] = coefficient of x^k for tap a.  With deriv, deg * w
 * more coefficients follow: those of phi'(z) = 2 dP_a/dx (z in cells), and *dmax receives a bound
 * on |phi'| sampled over every tap. */
void window_polys(int w, double beta, int deg, bool deriv, std::vector<long double> &mono_all,
                  double *dmax)
{
    const int m = deg + 1;
    const long double pi = 3.14159265358979323846264338327950288L;
    mono_all.assign((size_t)m * w + (deriv ? (size_t)deg * w : 0), 0.0L);
    for (int a = 0; a < w; ++a) {
        std::vector<long double> f(m), c(m, 0.0L), mono(m, 0.0L), t0(m, 0.0L), t1(m, 0.0L), t2(m);
        for (int j = 0; j < m; ++j) {
            const long double x = cosl(pi * (j + 0.5L) / m);
            const long double z = 0.5L * (x + 1.0L) - 0.5L * w + a;
            const long double v = (2.0L * z / w) * (2.0L * z / w);
            f[j] = v <= 1.0L ? expl(-(long double)beta * v / (1.0L + sqrtl(1.0L - v))) : 0.0L;
        }
        for (int k = 0; k < m; ++k) {
            long double sum = 0.0L;
            for (int j = 0; j < m; ++j) sum += f[j] * cosl(pi * k * (j + 0.5L) / m);
            c[k] = 2.0L * sum / m;
        }
        c[0] *= 0.5L;
        /* sum_k c_k T_k(x) in powers of x via T_{k+1} = 2x T_k - T_{k-1} */
        t0[0] = 1.0L;
        if (m > 1) t1[1] = 1.0L;
        for (int i = 0; i < m; ++i) mono[i] += c[0] * t0[i];
        for (int k = 1; k < m; ++k) {
            for (int i = 0; i < m; ++i) mono[i] += c[k] * t1[i];
            for (int i = 0; i < m; ++i) t2[i] = -t0[i] + (i > 0 ? 2.0L * t1[i - 1] : 0.0L);
            t0 = t1;
            t1 = t2;
        }
        for (int k = 0; k < m; ++k) mono_all[(size_t)k * w + a] = mono[k];
        if (deriv) {
            long double *dc = mono_all.data() + (size_t)m * w;
            for (int k = 0; k < deg; ++k) dc[(size_t)k * w + a] = 2.0L * (k + 1) * mono[k + 1];
            for (int sidx = 0; sidx <= 64; ++sidx) {
                const long double x = -1.0L + sidx / 32.0L;
                long double pd = dc[(size_t)(deg - 1) * w + a];
                for (int k = deg - 2; k >= 0; --k) pd = pd * x + dc[(size_t)k * w + a];
                if (fabsl(pd) > *dmax) *dmax = (double)fabsl(pd);
            }
        }
    }
}

/* window of width w at offset z (cells), long double */
long double es_phi_ld(long double z, int w, double beta)
{
    const long double v = (2.0L * z / w) * (2.0L * z / w);
    return v <= 1.0L ? expl(-(long double)beta * v / (1.0L + sqrtl(1.0L - v))) : 0.0L;
}

/* kWinPieces-piece window polynomials for the double-float window kernel: piece h of tap a covers
 * u in [h/P, (h+1)/P) (u = l0 - t + w/2, P = kWinPieces) with x = 2P u - 2h - 1 in [-1, 1); the
 * window there is interpolated at D+1 Chebyshev points and converted to powers of x in long double:
 * out[(h (D+1) + k) w + a].  With deriv, the coefficients of phi'(z) = 2P dP_h/dx follow:
 * out[P (D+1) w + (h D + k) w + a].  Returns the largest deviation from the window at 48 points of
 * every piece of the interior taps (the two edge taps carry the window's square-root edge, a
 * floor of ~5e-13 at w = 12 whatever the degree). */
using yk::kWinPieces;
long double window_pieces(int w, double beta, int D, bool deriv, std::vector<long double> &out)
{
    const int P = kWinPieces, m = D + 1;
    const long double pi = 3.14159265358979323846264338327950288L;
    out.assign((size_t)P * m * w + (deriv ? (size_t)P * D * w : 0), 0.0L);
    long double worst = 0.0L;
    for (int a = 0; a < w; ++a)
        for (int h = 0; h < P; ++h) {
            std::vector<long double> f(m), c(m, 0.0L), mono(m, 0.0L), t0(m, 0.0L), t1(m, 0.0L),
                t2(m);
            for (int j = 0; j < m; ++j) {
                const long double x = cosl(pi * (j + 0.5L) / m);
                const long double u = (x + 1.0L + 2.0L * h) / (2.0L * P);
                f[j] = es_phi_ld(u - 0.5L * w + a, w, beta);
            }
            for (int k = 0; k < m; ++k) {
                long double sum = 0.0L;
                for (int j = 0; j < m; ++j) sum += f[j] * cosl(pi * k * (j + 0.5L) / m);
                c[k] = 2.0L * sum / m;
            }
            c[0] *= 0.5L;
            t0[0] = 1.0L;
            if (m > 1) t1[1] = 1.0L;
            for (int i = 0; i < m; ++i) mono[i] += c[0] * t0[i];
            for (int k = 1; k < m; ++k) {
                for (int i = 0; i < m; ++i) mono[i] += c[k] * t1[i];
                for (int i = 0; i < m; ++i) t2[i] = -t0[i] + (i > 0 ? 2.0L * t1[i - 1] : 0.0L);
                t0 = t1;
                t1 = t2;
            }
            for (int k = 0; k < m; ++k) out[((size_t)h * m + k) * w + a] = mono[k];
            if (deriv)
                for (int k = 0; k < D; ++k)
                    out[(size_t)P * m * w + ((size_t)h * D + k) * w + a] =
                        2.0L * P * (k + 1) * mono[k + 1];
            if (a > 0 && a < w - 1)
                for (int sidx = 0; sidx < 48; ++sidx) {
                    const long double x = -1.0L + (sidx + 0.5L) / 24.0L;
                    long double pv = mono[D];
                    for (int k = D - 1; k >= 0; --k) pv = pv * x + mono[k];
                    const long double u = (x + 1.0L + 2.0L * h) / (2.0L * P);
                    worst = std::max(worst, fabsl(pv - es_phi_ld(u - 0.5L * w + a, w, beta)));
                }
        }
    return worst;
}

bool smooth5(int64_t n)
{
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

/* radices of an L-point transform: 4s, then a 2, then 3s, then 5s */
bool make_stages(int L, int n_tab, FftStages &st)
{
    std::memset(&st, 0, sizeof st);
    st.L = L;
    int m = L, s = 0;
    auto push = [&](int r) {
        if (s >= YK_MAX_STAGES) return false;
        st.r[s++] = r;
        m /= r;
        return true;
    };
    while (m % 4 == 0)
        if (!push(4)) return false;
    while (m % 2 == 0)
        if (!push(2)) return false;
    while (m % 3 == 0)
        if (!push(3)) return false;
    while (m % 5 == 0)
        if (!push(5)) return false;
    if (m != 1) return false;
    st.n = s;
    int B = L;
    for (int i = 0; i < s; ++i) {
        st.B[i] = B;
        st.tw_step[i] = n_tab / B;
        B /= st.r[i];
    }
    yk::fft_fill_magic(st);
    return true;
}

/* position of frequency m after the DIF stages: digits of m little-endian in r_1, r_2, ...,
 * each digit p_s placed at span_s = B_s / r_s */
void dif_positions(const FftStages &st, std::vector<int> &pos)
{
    pos.assign(st.L, 0);
    for (int m = 0; m < st.L; ++m) {
        int mm = m, p = 0;
        for (int s = 0; s < st.n; ++s) {
            const int d = mm % st.r[s];
            mm /= st.r[s];
            p += d * (st.B[s] / st.r[s]);
        }
        pos[m] = p;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* device memory                                                                               */

yk_status buf_alloc(yk_plan_t p, DevBuf &b, size_t bytes, const char *what)
{
    if (b.ptr && b.bytes >= bytes) return YK_OK;
    if (b.ptr) {
        if (p->dealloc) p->dealloc(b.ptr, (void *)p->stream, p->alloc_ctx);
        else cudaFree(b.ptr);
        p->bytes -= (int64_t)b.bytes;
        b.ptr = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) return YK_OK;
    void *ptr = nullptr;
    if (p->alloc) {
        ptr = p->alloc(bytes, (void *)p->stream, p->alloc_ctx);
        if (!ptr) return fail(YK_ERR_OOM, "allocator returned NULL for %s (%zu bytes)", what, bytes);
    } else {
        cudaError_t e = cudaMalloc(&ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? YK_ERR_OOM : YK_ERR_CUDA,
                        "cudaMalloc(%s, %zu bytes): %s", what, bytes, cudaGetErrorString(e));
        }
    }
    b.ptr = ptr;
    b.bytes = bytes;
    p->bytes += (int64_t)bytes;
    return YK_OK;
}

void buf_free(yk_plan_t p, DevBuf &b)
{
    if (!b.ptr) return;
    if (p->dealloc) p->dealloc(b.ptr, (void *)p->stream, p->alloc_ctx);
    else cudaFree(b.ptr);
    p->bytes -= (int64_t)b.bytes;
    b.ptr = nullptr;
    b.bytes = 0;
}

void free_all(yk_plan_t p)
{
    DevBuf *all[] = {&p->grid, &p->spec, &p->mult, &p->tw, &p->perm_h, &p->iperm_f, &p->win,
                     &p->win_df, &p->win_pc, &p->win32, &p->wnu, &p->win_src, &p->win_dip, &p->win_trg, &p->stage_d[0], &p->stage_d[1],
                     &p->stage_d[2], &p->stage_d[3], &p->stage_d[4], &p->stage_d[5],
                     &p->tile_cnt, &p->tile_ptr, &p->tile_cur, &p->tile_order, &p->part, &p->trg_cnt,
                     &p->trg_ptr,
                     &p->trg_cur, &p->err, &p->w_src, &p->src_t, &p->ent_t, &p->ent_j,
                     &p->trg_t, &p->trg_idx, &p->trg_tmp, &p->src_tap, &p->trg_tap,
                     &p->trg_hist, &p->stage_x, &p->stage_y,
                     &p->stage_w, &p->stage_u};
    for (DevBuf *b : all) buf_free(p, *b);
    for (int r = 0; r < yk_plan_s::kEventRing; ++r)
        for (int k = 0; k < 2 * YK_NUM_STAGES; ++k)
            if (p->events[r][k]) {
                cudaEventDestroy(p->events[r][k]);
                p->events[r][k] = nullptr;
            }
    p->profile = false;
}

template <typename T> T *P(DevBuf &b) { return static_cast<T *>(b.ptr); }

bool is_device_ptr(const void *ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

/* pageable host memory (not device, managed or page-locked): a call that reads it must finish its
 * copies before returning, and one that writes it must wait for the stream */
bool is_pageable_ptr(const void *ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered;
}

/* device view of n doubles: the pointer itself if it is device memory, else a staging copy */
yk_status to_device(yk_plan_t p, const double *src, int64_t n, DevBuf &stage,
                    const double **out, const char *what)
{
    *out = src;
    if (n == 0 || is_device_ptr(src)) return YK_OK;
    yk_status s = buf_alloc(p, stage, sizeof(double) * (size_t)n, what);
    if (s != YK_OK) return s;
    YK_CU(cudaMemcpyAsync(stage.ptr, src, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice,
                          p->stream),
          what);
    *out = P<double>(stage);
    return YK_OK;
}

yk::Geom geom_of(const yk_plan_s *p)
{
    yk::Geom g;
    g.ox = p->ox;
    g.oy = p->oy;
    g.inv_h = (double)p->n / p->period;
    g.beta = p->beta;
    g.c = 4.0 / ((double)p->w * p->w);
    g.n = (int)p->n;
    g.T = p->T;
    g.nt = p->nt;
    g.Ti = p->Ti;
    g.nti = p->nti;
    g.w = p->w;
    for (int k = 0; k < 4; ++k) g.box[k] = p->box[k];
    g.A = std::ldexp(g.inv_h, yk::kFixBits);
    g.Bx = -p->ox * g.A;
    g.By = -p->oy * g.A;
    g.n44 = (long long)p->n << yk::kFixBits;
    /* the same FMA and rounding as the device's fixed_coord (both IEEE, round to nearest even) */
    g.tbox[0] = std::llrint(std::fma(p->box[0], g.A, g.Bx));
    g.tbox[1] = std::llrint(std::fma(p->box[1], g.A, g.Bx));
    g.tbox[2] = std::llrint(std::fma(p->box[2], g.A, g.By));
    g.tbox[3] = std::llrint(std::fma(p->box[3], g.A, g.By));
    return g;
}

/* wait for the stream, fold the device error word into the sticky status */
yk_status sync_and_check(yk_plan_t p)
{
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        p->status = YK_ERR_CUDA;
        return cuda_fail(e, "stream synchronize");
    }
    if (p->err.ptr) {
        int h_err = 0;
        e = cudaMemcpy(&h_err, p->err.ptr, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            p->status = YK_ERR_CUDA;
            return cuda_fail(e, "error word");
        }
        if (h_err & yk::ERR_POINT_OUTSIDE) p->status = YK_ERR_ARG;
    }
    if (p->status == YK_ERR_ARG)
        return fail(YK_ERR_ARG, "a source or target lies outside the plan's box");
    if (p->status != YK_OK) return fail((yk_status)p->status, "plan is in an error state");
    return YK_OK;
}

/* bracket a stage with events when profiling */
inline void stage_begin(yk_plan_t p, int s)
{
    if (p->profile)
        cudaEventRecord(p->events[p->stage_runs[s] % yk_plan_s::kEventRing][2 * s], p->stream);
}
inline void stage_end(yk_plan_t p, int s)
{
    if (p->profile) {
        cudaEventRecord(p->events[p->stage_runs[s] % yk_plan_s::kEventRing][2 * s + 1], p->stream);
        ++p->stage_runs[s];
    }
}

yk_status plan_tables(yk_plan_t p)
{
    const int64_t n = p->n, M = p->M;
    const size_t nt2 = (size_t)p->nt * p->nt;
    yk_status s;
#define YK_TRY(x)                                                                               \
    do {                                                                                        \
        if ((s = (x)) != YK_OK) return s;                                                       \
    } while (0)
    const bool f32 = p->precision == YK_FP32C;
    const size_t rb = f32 ? sizeof(float) : sizeof(double);
    YK_TRY(buf_alloc(p, p->grid, rb * n * n, "grid"));
    YK_TRY(buf_alloc(p, p->spec, 2 * rb * (M + 1) * n, "spectrum"));
    YK_TRY(buf_alloc(p, p->mult, rb * (M + 1) * (2 * M + 1), "multiplier"));
    YK_TRY(buf_alloc(p, p->tw, 2 * rb * n, "twiddles"));
    YK_TRY(buf_alloc(p, p->perm_h, sizeof(int) * (n / 2), "permutation"));
    YK_TRY(buf_alloc(p, p->iperm_f, sizeof(int) * n, "permutation"));
    YK_TRY(buf_alloc(p, p->tile_cnt, sizeof(int) * nt2, "tile counts"));
    YK_TRY(buf_alloc(p, p->tile_ptr, sizeof(int) * (nt2 + 1), "tile offsets"));
    /* the source cursors double as the heavy-first ordering's 80-int scratch */
    YK_TRY(buf_alloc(p, p->tile_cur, sizeof(int) * (nt2 > 80 ? nt2 : 80), "tile cursors"));
    YK_TRY(buf_alloc(p, p->tile_order, sizeof(int) * nt2, "tile order"));
    const size_t nti2 = (size_t)p->nti * p->nti;
    YK_TRY(buf_alloc(p, p->trg_cnt, sizeof(int) * nti2, "tile counts"));
    YK_TRY(buf_alloc(p, p->trg_ptr, sizeof(int) * (nti2 + 1), "tile offsets"));
    YK_TRY(buf_alloc(p, p->trg_cur, sizeof(int) * nti2, "tile cursors"));
    if (p->fft_df || f32) { /* owner-tile spread: one padded tile of partial sums per tile */
        const size_t span = (size_t)p->T + p->w - 1;
        YK_TRY(buf_alloc(p, p->part, sizeof(double) * nt2 * span * span, "padded tiles"));
    }
#undef YK_TRY
    if (!make_stages((int)(n / 2), (int)n, p->st_half) || !make_stages((int)n, (int)n, p->st_full))
        return fail(YK_ERR_INTERNAL, "FFT stage plan failed for n = %lld", (long long)n);
    std::vector<int> pos_h, pos_f, ipos_f(n);
    dif_positions(p->st_half, pos_h);
    dif_positions(p->st_full, pos_f);
    for (int64_t m = 0; m < n; ++m) ipos_f[pos_f[m]] = (int)m;
    /* twiddles from long double, rounded once to the table's type (FP32C: float pairs; FP64 with
     * double-float FFT: hi/lo float pairs per component; FP64: doubles) */
    std::vector<double2> tw(f32 ? 0 : n);
    std::vector<float2> tw32(f32 ? n : 0);
    for (int64_t j = 0; j < n; ++j) {
        const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)j /
                              (long double)n;
        const long double c = cosl(a), sn = -sinl(a);
        if (f32) {
            tw32[j] = make_float2((float)c, (float)sn);
        } else if (p->fft_df) {
            float v[4];
            v[0] = (float)c;
            v[1] = (float)(c - (long double)v[0]);
            v[2] = (float)sn;
            v[3] = (float)(sn - (long double)v[2]);
            std::memcpy(&tw[j], v, sizeof v);
        } else {
            tw[j] = make_double2((double)c, (double)sn);
        }
    }
    std::vector<double> dfac(M + 1);
    for (int64_t m = 0; m <= M; ++m) {
        const double ph = window_ft(2.0 * kPi * (double)m / (double)n, p->w, p->beta);
        dfac[m] = 1.0 / (ph * ph);
    }
    if (!f32 || p->dlp) {
        /* windows as per-tap polynomials of degree w + 1 (the FP64 path always; FP32C for its
         * dipoles), followed by the derivative's coefficients when the plan takes dipoles */
        /* degree w - 1: interior taps to ~1e-13 of the peak at w = 12 (the two edge taps carry
         * the window's square-root edge, ~5e-13 at any degree), well inside eps = 10^(1-w) */
        p->wdeg = std::max(2, p->w - 1);
        std::vector<long double> mono;
        p->dmax = 0.0;
        window_polys(p->w, p->beta, p->wdeg, p->dlp != 0, mono, &p->dmax);
        p->dmax *= 1.0 + 1e-6;
        cudaError_t ew = cudaSuccess;
        if (!f32 && p->fft_df) {
            /* the double-float window kernel's kWinPieces-piece tables (degree kPieceDeg[w]) */
            std::vector<long double> pc;
            const int D = yk::kPieceDeg[p->w];
            p->pdeg = D;
            window_pieces(p->w, p->beta, D, p->dlp != 0, pc);
            std::vector<float2> pc_df(pc.size());
            for (size_t i = 0; i < pc.size(); ++i) {
                const float hi = (float)pc[i];
                pc_df[i] = make_float2(hi, (float)(pc[i] - (long double)hi));
            }
            if ((s = buf_alloc(p, p->win_pc, sizeof(float2) * pc_df.size(), "window")) != YK_OK)
                return s;
            ew = cudaMemcpy(p->win_pc.ptr, pc_df.data(), sizeof(float2) * pc_df.size(),
                            cudaMemcpyHostToDevice);
            if (ew != cudaSuccess) return cuda_fail(ew, "window table");
        }
        if (!f32) {
            std::vector<double> poly(mono.size());
            std::vector<float2> poly_df(mono.size());
            for (size_t i = 0; i < mono.size(); ++i) {
                poly[i] = (double)mono[i];
                const float hi = (float)mono[i];
                poly_df[i] = make_float2(hi, (float)(mono[i] - (long double)hi));
            }
            if ((s = buf_alloc(p, p->win, sizeof(double) * poly.size(), "window")) != YK_OK)
                return s;
            if ((s = buf_alloc(p, p->win_df, sizeof(float2) * poly_df.size(), "window")) != YK_OK)
                return s;
            ew = cudaMemcpy(p->win.ptr, poly.data(), sizeof(double) * poly.size(),
                            cudaMemcpyHostToDevice);
            if (ew == cudaSuccess)
                ew = cudaMemcpy(p->win_df.ptr, poly_df.data(), sizeof(float2) * poly_df.size(),
                                cudaMemcpyHostToDevice);
        } else {
            std::vector<float> poly32(mono.size());
            for (size_t i = 0; i < mono.size(); ++i) poly32[i] = (float)mono[i];
            if ((s = buf_alloc(p, p->win32, sizeof(float) * poly32.size(), "window")) != YK_OK)
                return s;
            ew = cudaMemcpy(p->win32.ptr, poly32.data(), sizeof(float) * poly32.size(),
                            cudaMemcpyHostToDevice);
        }
        if (ew != cudaSuccess) return cuda_fail(ew, "window table");
    }
    DevBuf d_dfac = {nullptr, 0};
    if ((s = buf_alloc(p, d_dfac, sizeof(double) * (M + 1), "deconvolution")) != YK_OK) return s;
    cudaError_t e = cudaMemcpyAsync(p->perm_h.ptr, pos_h.data(), sizeof(int) * (n / 2),
                                    cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->iperm_f.ptr, ipos_f.data(), sizeof(int) * n, cudaMemcpyHostToDevice,
                            p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->tw.ptr, f32 ? (const void *)tw32.data() : (const void *)tw.data(),
                            2 * rb * n, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_dfac.ptr, dfac.data(), sizeof(double) * (M + 1),
                            cudaMemcpyHostToDevice, p->stream);
    /* truncated kernel: its radial transform on a fine k table (spacing H with R1 H = 0.22, so
     * 10-point interpolation errs by ~1e-13 of the peak), up to the corner of the mode square */
    DevBuf d_tab = {nullptr, 0}, d_nodes = {nullptr, 0};
    const double dk = 2.0 * kPi / p->period;
    double H = 0.0;
    int ntab = 0;
    if (e == cudaSuccess && p->truncated) {
        H = 0.22 / p->r1;
        const double ktop = std::sqrt(2.0) * (double)M * dk;
        ntab = (int)std::ceil(ktop / H) + 12;
        /* transition quadrature: 16-point Gauss-Legendre panels no wider than 6 / ktop */
        const double sw = (p->r1 - p->r0) / 12.0;
        const int npan = (int)std::ceil((p->r1 - p->r0) * ktop / 6.0) + 2;
        double gx[16], gw[16];
        gauss_legendre(16, gx, gw);
        std::vector<double2> nodes((size_t)npan * 16);
        const double L = (p->r1 - p->r0) / npan;
        for (int a = 0; a < npan; ++a)
            for (int i = 0; i < 16; ++i) {
                const double r = p->r0 + L * (a + 0.5 * (gx[i] + 1.0));
                const double chi = 0.5 * std::erfc((r - p->r0 - 6.0 * sw) / sw);
                nodes[(size_t)a * 16 + i] =
                    make_double2(r, 0.5 * L * gw[i] * bessel_k(0, p->alpha * r) * chi * r);
            }
        if ((s = buf_alloc(p, d_tab, sizeof(double) * ntab, "kernel table")) != YK_OK ||
            (s = buf_alloc(p, d_nodes, sizeof(double2) * nodes.size(), "kernel table")) != YK_OK) {
            buf_free(p, d_dfac);
            buf_free(p, d_tab);
            return s;
        }
        e = cudaMemcpyAsync(d_nodes.ptr, nodes.data(), sizeof(double2) * nodes.size(),
                            cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess)
            e = yk::launch_trunc_table(P<double>(d_tab), ntab, H, p->alpha, p->delta, p->r0,
                                       bessel_k(0, p->alpha * p->r0),
                                       bessel_k(1, p->alpha * p->r0), P<double2>(d_nodes),
                                       (int)nodes.size(), p->stream);
    }
    const double *tab = p->truncated ? P<double>(d_tab) : nullptr;
    if (e == cudaSuccess) {
        if (f32)
            e = yk::launch_build_mult32(P<float>(p->mult), P<double>(d_dfac), (int)M, p->alpha,
                                        p->delta, dk, p->period, p->stream, tab, ntab, H);
        else if (p->fft_df)
            e = yk::launch_build_mult_df(p->mult.ptr, P<double>(d_dfac), (int)M, p->alpha,
                                         p->delta, dk, p->period, p->stream, tab, ntab, H);
        else
            e = yk::launch_build_mult(P<double>(p->mult), P<double>(d_dfac), (int)M, p->alpha,
                                      p->delta, dk, p->period, p->stream, tab, ntab, H);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    buf_free(p, d_dfac);
    buf_free(p, d_tab);
    buf_free(p, d_nodes);
    if (e != cudaSuccess) return cuda_fail(e, "plan tables");
    return YK_OK;
}

} /* namespace */

/* ------------------------------------------------------------------------------------------ */
/* evaluation descriptor for the batch kernel                                                  */

void yk_set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

void yk_gauss_legendre(int n, double *x, double *w) { gauss_legendre(n, x, w); }

bool yk_fill_inst(const yk_plan_s *pc, yk::Inst *d)
{
    yk_plan_s *p = const_cast<yk_plan_s *>(pc);
    if (p->zero || p->n_src + p->n_dip == 0 || p->n_trg == 0) return false;
    std::memset((void *)d, 0, sizeof *d);
    d->g = geom_of(p);
    d->sth = p->st_half;
    d->stf = p->st_full;
    d->n = (int)p->n;
    d->M = (int)p->M;
    d->f32 = p->precision == YK_FP32C;
    d->fft_df = p->fft_df;
    d->rows = yk::rows_per_item(d->n, d->f32, true);
    d->tile_ptr = P<int>(p->tile_ptr);
    d->order = P<int>(p->tile_order);
    d->ent_t = P<double2>(p->ent_t);
    d->ent_j = P<int>(p->ent_j);
    d->part = (p->fft_df || d->f32) ? p->part.ptr : nullptr;
    d->spread_warps = p->spread_warps;
    d->spread_batch = p->spread_batch;
    d->interp_threads = p->interp_threads;
    d->wq = P<double>(p->w_src);
    d->trg_ptr = P<int>(p->trg_ptr);
    d->trg_t = P<double2>(p->trg_t);
    d->trg_idx = P<int>(p->trg_idx);
    d->grid = p->grid.ptr;
    d->spec = p->spec.ptr;
    d->mult = p->mult.ptr;
    d->tw = p->tw.ptr;
    d->perm_h = P<int>(p->perm_h);
    d->iperm_f = P<int>(p->iperm_f);
    d->win = P<double>(p->win);
    d->win_df = P<float2>(p->win_df);
    d->wdeg = p->wdeg;
    d->n_chg = (int)p->n_src;
    d->dip = p->n_dip > 0 ? 1 : 0;
    d->wnu = P<double2>(p->wnu);
    d->win32 = P<float>(p->win32);
    d->dmax = p->dmax;
    d->win_src = P<float2>(p->win_src);
    d->win_dip = P<float2>(p->win_dip);
    d->win_trg = P<float2>(p->win_trg);
    d->win_trg_pitch = p->n_trg;
    for (int s = 0; s < yk::ST_COUNT; ++s) {
        d->items[s] = yk::stage_items(*d, s);
        d->smem[s] = yk::stage_smem(*d, s);
    }
    return true;
}

/* ------------------------------------------------------------------------------------------ */
/* ABI                                                                                         */

extern "C" {

void yk_opts_default(yk_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = YK_FP64;
    o->tol = 1e-10;
    o->eps_hist = 1e-6;
    o->box[0] = -1.5;
    o->box[1] = 1.5;
    o->box[2] = -1.5;
    o->box[3] = 1.5;
}

const char *yk_last_error(void) { return g_last_error.c_str(); }

/* parameter rules shared by yk_plan and yk_plan_params; fills the parameter fields of *p */
static yk_status choose_params(double alpha, const yk_opts *o, yk_plan_s *p)
{
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(YK_ERR_ARG, "alpha must be > 0");
    if (!(o->tol > 0.0 && o->tol < 1.0)) return fail(YK_ERR_ARG, "tol must lie in (0, 1)");
    if (o->precision != YK_FP64 && o->precision != YK_FP32C)
        return fail(YK_ERR_ARG, "precision must be YK_FP64 or YK_FP32C");
    if (!(o->box[1] > o->box[0] && o->box[3] > o->box[2]) || !std::isfinite(o->box[0]) ||
        !std::isfinite(o->box[1]) || !std::isfinite(o->box[2]) || !std::isfinite(o->box[3]))
        return fail(YK_ERR_ARG, "box must satisfy xmin < xmax and ymin < ymax");
    if (o->tile < 0) return fail(YK_ERR_ARG, "tile must be >= 0");
    /* the owner-tile spreads (FP32C, double-float FP64) keep per-warp padded copies of a tile in
     * shared memory and pack in-tile positions in 6 bits: their tile edge is at most 32 */
    if (o->tile > 32 && (o->precision == YK_FP32C || !o->fft_fp64))
        return fail(YK_ERR_ARG, "tile must be <= 32 (64 with fft_fp64)");
    if (o->kmax_rule != 0 && o->kmax_rule != 1) return fail(YK_ERR_ARG, "kmax_rule must be 0 or 1");
    if (o->spread_warps < 0 || o->spread_warps > 4)
        return fail(YK_ERR_ARG, "spread_warps must be 0 (default) or 1..4");
    if (o->spread_batch != 0 &&
        (o->precision == YK_FP32C ? (o->spread_batch != 8 && o->spread_batch != 16 && o->spread_batch != 32)
                                  : (o->spread_batch != 4 && o->spread_batch != 8 && o->spread_batch != 16)))
        return fail(YK_ERR_ARG, "spread_batch must be 0, 4, 8 or 16 (FP32C: 0, 8, 16 or 32)");
    if (o->interp_threads != 0 && o->interp_threads != 64 && o->interp_threads != 128 &&
        o->interp_threads != 256)
        return fail(YK_ERR_ARG, "interp_threads must be 0, 64, 128 or 256");
    if (o->interp_tile < 0 || o->interp_tile > 32 || (o->interp_tile > 0 && o->fft_fp64 &&
                                                       o->precision == YK_FP64))
        return fail(YK_ERR_ARG, "interp_tile must be 0 (default) or at most 32, and 0 with "
                                "fft_fp64");
    if ((o->alloc == nullptr) != (o->free == nullptr))
        return fail(YK_ERR_ARG, "give both alloc and free callbacks, or neither");
    double delta = o->delta;
    if (!(delta > 0.0)) {
        if (!(o->h_vol > 0.0)) return fail(YK_ERR_ARG, "give delta > 0 or h_vol > 0");
        const double eh = o->eps_hist > 0.0 ? o->eps_hist : 1e-6;
        if (!(eh < 1.0)) return fail(YK_ERR_ARG, "eps_hist must lie in (0, 1)");
        const double kp = 0.9 * kPi / o->h_vol; /* 0.9 k_Nyq (eq. k_nyq, Section 6.4) */
        delta = std::log(1.0 / eh) / (kp * kp + alpha * alpha);
    }
    p->alpha = alpha;
    p->delta = delta;
    p->tol = o->tol;
    p->eps = o->tol / 4.0;
    p->precision = o->precision;
    p->fft_df = (o->precision == YK_FP64 && !o->fft_fp64) ? 1 : 0;
    p->stream = (cudaStream_t)o->stream;
    p->alloc = o->alloc;
    p->dealloc = o->free;
    p->alloc_ctx = o->alloc_ctx;

    /* Fourier cutoff (eq. kmax) and period (decay length of G_H beyond the box span) */
    p->dlp = o->dlp ? 1 : 0;
    p->kmax = o->kmax > 0.0         ? o->kmax
              : o->kmax_rule == 1 ? kmax_paper(alpha, delta, p->eps)
                                  : kmax_relative(alpha, delta, p->eps);
    if (p->dlp && !(o->kmax > 0.0)) /* the double layer's cutoff (eq. kmax_dlp) is stricter */
        p->kmax = std::max(p->kmax, o->kmax_rule == 1 ? kmax_dlp_paper(alpha, delta, p->eps)
                                                      : kmax_dlp_relative(alpha, delta, p->eps));
    const double span = std::max(o->box[1] - o->box[0], o->box[3] - o->box[2]);
    if (o->truncate < 0 || o->truncate > 2) return fail(YK_ERR_ARG, "truncate must be 0, 1 or 2");
    p->truncated = 0;
    if (p->kmax > 0.0 && o->truncate != 1) {
        /* truncated kernel: chi = 1 up to the box diagonal D (no source-target pair is farther
         * apart), then 1/2 erfc((r - D - 6 s)/s) down to ~1e-17 at D + 12 s.  s = 20 / k_max keeps
         * the transform's tail beyond k_max at that of G_H.  Valid while G_H = K0(alpha r)/(2 pi)
         * beyond D (the local part there is below E1(D^2 / (4 delta)) / (4 pi)). */
        const double D = std::hypot(o->box[1] - o->box[0], o->box[3] - o->box[2]);
        const double s = 20.0 / p->kmax, r1 = D + 12.0 * s;
        const bool valid = D * D / (4.0 * delta) >= 50.0;
        const double p_plain = o->period > 0.0 ? o->period
                                               : span + decay_length(alpha, delta, p->eps);
        if (o->truncate == 2 && !valid)
            return fail(YK_ERR_ARG, "the truncated kernel needs box diagonal^2 / (4 delta) >= 50");
        if (valid && (o->truncate == 2 || (o->period <= 0.0 && span + r1 < p_plain))) {
            p->truncated = 1;
            p->r0 = D;
            p->r1 = r1;
            p->period = o->period > 0.0 ? o->period : span + r1;
            if (!(p->period >= span + r1))
                return fail(YK_ERR_ARG, "period %.17g is below span + truncation radius %.17g",
                            p->period, span + r1);
        } else {
            p->period = p_plain;
        }
    } else {
        p->period = o->period > 0.0 ? o->period : span + decay_length(alpha, delta, p->eps);
    }
    if (!(p->period > span))
        return fail(YK_ERR_ARG, "period %.17g must exceed the box span %.17g", p->period, span);
    for (int k = 0; k < 4; ++k) p->box[k] = o->box[k];
    const double cx = 0.5 * (o->box[0] + o->box[1]), cy = 0.5 * (o->box[2] + o->box[3]);
    p->ox = cx - 0.5 * p->period;
    p->oy = cy - 0.5 * p->period;
    p->zero = !(p->kmax > 0.0);
    p->M = p->zero ? 0 : (int64_t)std::ceil(p->kmax * p->period / (2.0 * kPi));

    /* window width (digits of eps), grid size (>= 2 (2M+1), 5-smooth, with a tile edge) */
    int w = (int)std::ceil(std::log10(1.0 / p->eps)) + 1;
    /* a dipole is spread with the window's gradient: its aliasing error is the charges' times up
     * to |k'| / |k| ~ 3 (alias k' of a kept mode k at two-fold oversampling), so a plan that takes
     * dipoles uses one more digit of window */
    if (p->dlp) ++w;
    w = std::min(16, std::max(2, w));
    p->w = w;
    p->beta = 2.30 * w;
    const int64_t nmin = std::max<int64_t>({2 * (2 * p->M + 1), 2 * (int64_t)w, 16});
    int64_t n = nmin + (nmin & 1);
    int T = 0;
    for (;; n += 2) {
        const int nmax = o->precision == YK_FP32C ? yk::kMaxGridF32 : yk::kMaxGridF64;
        if (n > nmax)
            return fail(YK_ERR_UNSUPPORTED,
                        "a grid of at least %lld points per axis is needed (the library supports "
                        "%d at this precision): raise delta or tol, or lower the period",
                        (long long)nmin, nmax);
        if (!smooth5(n)) continue;
        T = 0;
        if (o->tile > 0) {
            if (n % o->tile == 0 && o->tile >= w && n >= 2 * o->tile) T = o->tile;
        } else {
            /* default edge: the largest admissible divisor up to 20 (FP32C) or 24 (double-float
             * FP64), where the owner-tile spreads measured fastest on B300 (smaller padded copies:
             * more CTAs, and so more warps, per SM); the all-FP64 path up to 64; the autotuner
             * searches every edge up to 32 (64) */
            const int tmax = o->precision == YK_FP32C ? 20 : (!o->fft_fp64 ? 24 : 64);
            int pref = 0, sw = 0, sb = 0, it = 0, ti = 0;
            if (o->use_tuned)
                yk_tuned_shape(o->precision, w, n, o->n_src_hint, &pref, &sw, &sb, &it, &ti);
            const int tlim = pref > 0 ? (o->precision == YK_FP32C || !o->fft_fp64 ? 32 : 64) : tmax;
            for (int t = tlim; t >= w; --t)
                if (n % t == 0 && n >= 2 * t) {
                    /* largest admissible edge, or the one nearest the tuned edge */
                    if (!T || (pref > 0 && std::abs(t - pref) < std::abs(T - pref))) T = t;
                    if (!pref) break;
                }
            /* no admissible edge up to tmax (w close to it): the smallest one above */
            for (int t = tmax + 1; !T && t <= (o->precision == YK_FP32C || !o->fft_fp64 ? 32 : 64); ++t)
                if (n % t == 0 && n >= 2 * t) T = t;
        }
        if (T) break;
    }
    p->n = n;
    p->T = T;
    p->nt = (int)(n / T);
    p->h = p->period / (double)n;
    /* launch shape: the caller's, else the autotuner's (use_tuned), else the defaults */
    int tt = 0, sw = 0, sb = 0, it = 0, ti = 0;
    if (o->use_tuned) yk_tuned_shape(o->precision, w, n, o->n_src_hint, &tt, &sw, &sb, &it, &ti);
    /* the targets' tile: the interpolation reads a tile's halo once for all its targets, so it
     * gains from larger tiles where the owner-tile spread gains from smaller ones.  On those
     * paths it is chosen apart from T: the caller's edge, else the admissible divisor nearest
     * the tuned one, else the largest admissible divisor up to 32 (T itself when none is) */
    p->Ti = T;
    if (o->precision == YK_FP32C || !o->fft_fp64) {
        const int want = o->interp_tile > 0 ? o->interp_tile : ti;
        if (o->interp_tile > 0 && !(n % want == 0 && want >= w && n >= 2 * want))
            return fail(YK_ERR_ARG, "interp_tile %d does not divide the grid size %lld or is "
                                    "below the window width %d", want, (long long)n, w);
        int best = 0;
        for (int t = 32; t >= w; --t)
            if (n % t == 0 && n >= 2 * t) {
                if (!best || (want > 0 && std::abs(t - want) < std::abs(best - want))) best = t;
                if (!want) break;
            }
        if (best) p->Ti = best;
    }
    p->nti = (int)(n / p->Ti);
    p->spread_warps = o->spread_warps ? o->spread_warps : (sw ? sw : 4);
    p->spread_batch = o->spread_batch ? o->spread_batch
                                      : (sb ? sb : (o->precision == YK_FP32C ? 32 : 16));
    p->interp_threads = o->interp_threads ? o->interp_threads : (it ? it : 256);
    return YK_OK;
}

/* device bytes a plan holds for given point counts (plan tables plus resident layout) */
static int64_t predicted_bytes(const yk_plan_s *p, int64_t n_src, int64_t n_trg)
{
    if (p->zero) return (int64_t)sizeof(int);
    const int64_t n = p->n, M = p->M, nt2 = (int64_t)p->nt * p->nt,
                  nti2 = (int64_t)p->nti * p->nti;
    const int64_t r = p->precision == YK_FP32C ? 4 : 8; /* bytes of the real type */
    int64_t b = r * n * n + 2 * r * (M + 1) * n + r * (M + 1) * (2 * M + 1) + 2 * r * n +
                4 * (n / 2) + 4 * n + 4 * (4 * nt2 + 3 * nti2 + 2) + 4;
    if (p->precision == YK_FP64) b += 8 * (int64_t)(p->w + 2) * p->w * (p->dlp ? 2 : 1);
    else if (p->dlp) b += 4 * (int64_t)(2 * p->w + 3) * p->w;
    const bool owner = p->fft_df || p->precision == YK_FP32C;
    const int64_t epp = owner ? 1 : 4; /* entries per source */
    b += n_src * (8 + 16 + epp * (16 + 4)) + n_trg * (16 + 4 + 16);
    if (owner) b += 8 * nt2 * (int64_t)(p->T + p->w - 1) * (p->T + p->w - 1);
    if (p->fft_df) b += (n_src + n_trg) * 16 * (int64_t)p->w; /* per-point window values */
    return b;
}

extern "C" yk_status yk_plan_params(double alpha, const yk_opts *o, int64_t n_src, int64_t n_trg,
                                    yk_info *info)
{
    if (!info) return fail(YK_ERR_ARG, "info is NULL");
    yk_opts def;
    yk_opts_default(&def);
    if (!o) o = &def;
    yk_plan_s tmp;
    std::memset((void *)&tmp, 0, sizeof tmp);
    yk_status s = choose_params(alpha, o, &tmp);
    if (s != YK_OK) return s;
    tmp.bytes = predicted_bytes(&tmp, n_src, n_trg);
    return yk_plan_info(&tmp, info);
}

yk_status yk_plan(double alpha, const yk_opts *o, yk_plan_t *out)
{
    if (!out) return fail(YK_ERR_ARG, "yk_plan: out is NULL");
    *out = nullptr;
    yk_opts def;
    yk_opts_default(&def);
    if (!o) o = &def;
    yk_plan_s *p = new (std::nothrow) yk_plan_s();
    if (!p) return fail(YK_ERR_OOM, "host allocation of the plan failed");
    std::memset((void *)p, 0, sizeof *p);
    {
        yk_status s0 = choose_params(alpha, o, p);
        if (s0 != YK_OK) {
            delete p;
            return s0;
        }
    }
    yk_status s = YK_OK;
    if (o->profile) {
        for (int r = 0; r < yk_plan_s::kEventRing && s == YK_OK; ++r)
            for (int k = 0; k < 2 * YK_NUM_STAGES && s == YK_OK; ++k) {
                cudaError_t e = cudaEventCreate(&p->events[r][k]);
                if (e != cudaSuccess) s = cuda_fail(e, "event create");
            }
        p->profile = s == YK_OK;
    }
    if (s == YK_OK) s = buf_alloc(p, p->err, sizeof(int), "error word");
    if (s == YK_OK) {
        cudaError_t e = cudaMemsetAsync(p->err.ptr, 0, sizeof(int), p->stream);
        if (e != cudaSuccess) s = cuda_fail(e, "error word");
    }
    if (s == YK_OK && !p->zero) s = plan_tables(p);
    if (s != YK_OK) {
        free_all(p);
        delete p;
        return s;
    }
    *out = p;
    return YK_OK;
}

yk_status yk_plan_info(yk_plan_t p, yk_info *info)
{
    if (!p || !info) return fail(YK_ERR_ARG, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->alpha = p->alpha;
    info->delta = p->delta;
    info->tol = p->tol;
    info->eps = p->eps;
    info->kmax = p->kmax;
    info->period = p->period;
    info->origin[0] = p->ox;
    info->origin[1] = p->oy;
    info->h = p->h;
    info->n_modes = p->M;
    info->n_grid = p->zero ? 0 : p->n;
    info->w = p->w;
    info->beta = p->beta;
    info->tile = p->T;
    info->interp_tile = p->Ti;
    info->precision = p->precision;
    info->device_bytes = p->bytes;
    info->truncated = p->truncated;
    info->r_support = p->truncated ? p->r1 : 0.0;
    info->spread_warps = p->spread_warps;
    info->spread_batch = p->spread_batch;
    info->interp_threads = p->interp_threads;
    return YK_OK;
}

yk_status yk_set_points_dl(yk_plan_t p, int64_t n_src, const double *xs, const double *ys,
                           const double *w, int64_t n_dip, const double *xd, const double *yd,
                           const double *wd, const double *nx, const double *ny, int64_t n_trg,
                           const double *xt, const double *yt)
{
    if (!p) return fail(YK_ERR_ARG, "plan is NULL");
    if (n_src < 0 || n_trg < 0 || n_dip < 0) return fail(YK_ERR_ARG, "negative point count");
    if (n_src + n_dip > (1ll << 28) || n_trg > (1ll << 30))
        return fail(YK_ERR_UNSUPPORTED, "too many points for 32-bit entry indices");
    if ((n_src > 0 && (!xs || !ys || !w)) || (n_trg > 0 && (!xt || !yt)) ||
        (n_dip > 0 && (!xd || !yd || !wd || !nx || !ny)))
        return fail(YK_ERR_ARG, "NULL coordinate, weight or normal array");
    if (n_dip > 0 && !p->dlp)
        return fail(YK_ERR_ARG, "dipole sources need a plan created with opts.dlp");
    if (p->status != YK_OK) return fail((yk_status)p->status, "plan is in an error state");
    p->points_set = false;
    ++p->layout_version;
    p->n_src = n_src;
    p->n_dip = n_dip;
    p->n_trg = n_trg;
    if (p->zero) {
        p->points_set = true;
        return YK_OK;
    }
    yk_status s;
#define YK_TRY(x)                                                                               \
    do {                                                                                        \
        if ((s = (x)) != YK_OK) return s;                                                       \
    } while (0)
    const size_t ns = (size_t)n_src, nd = (size_t)n_dip, nt = (size_t)n_trg;
    YK_TRY(buf_alloc(p, p->w_src, sizeof(double) * ns, "weights"));
    YK_TRY(buf_alloc(p, p->src_t, sizeof(double2) * (ns + nd), "source coordinates"));
    /* entries: one per source for the owner-tile spread, else one per tile a window touches */
    const size_t epp = (p->fft_df || p->precision == YK_FP32C) ? 1 : 4;
    YK_TRY(buf_alloc(p, p->ent_t, sizeof(double2) * epp * (ns + nd), "entries"));
    YK_TRY(buf_alloc(p, p->ent_j, sizeof(int) * epp * (ns + nd), "entries"));
    YK_TRY(buf_alloc(p, p->trg_t, sizeof(double2) * nt, "targets"));
    YK_TRY(buf_alloc(p, p->trg_idx, sizeof(int) * nt, "targets"));
    YK_TRY(buf_alloc(p, p->trg_tmp, sizeof(double2) * nt, "targets"));
    if (nd > 0) YK_TRY(buf_alloc(p, p->wnu, sizeof(double2) * nd, "dipole weights"));
    const yk::Geom g = geom_of(p);
    const double *dx = nullptr, *dy = nullptr, *dw = nullptr;
    YK_TRY(to_device(p, xs, n_src, p->stage_x, &dx, "source x"));
    YK_TRY(to_device(p, ys, n_src, p->stage_y, &dy, "source y"));
    YK_TRY(to_device(p, w, n_src, p->stage_w, &dw, "weights"));
    const double *ddx = nullptr, *ddy = nullptr, *ddw = nullptr, *dnx = nullptr, *dny = nullptr;
    YK_TRY(to_device(p, xd, n_dip, p->stage_d[0], &ddx, "dipole x"));
    YK_TRY(to_device(p, yd, n_dip, p->stage_d[1], &ddy, "dipole y"));
    YK_TRY(to_device(p, wd, n_dip, p->stage_d[2], &ddw, "dipole weights"));
    YK_TRY(to_device(p, nx, n_dip, p->stage_d[3], &dnx, "dipole normals"));
    YK_TRY(to_device(p, ny, n_dip, p->stage_d[4], &dny, "dipole normals"));
    if (n_src > 0)
        YK_CU(cudaMemcpyAsync(p->w_src.ptr, dw, sizeof(double) * ns, cudaMemcpyDeviceToDevice,
                              p->stream),
              "weights");
    YK_CU(yk::launch_pack_wnu(n_dip, ddw, dnx, dny, P<double2>(p->wnu), p->stream),
          "dipole weights");
    /* the double-float and FP32C paths prepare points in fixed point (no FP64 rounding past
     * the grid coordinate); the all-FP64 path keeps FP64 grid coordinates */
    const bool prep = p->fft_df || p->precision == YK_FP32C;
    if (prep) {
        YK_TRY(buf_alloc(p, p->src_tap, sizeof(int2) * (ns + nd), "source taps"));
        YK_TRY(buf_alloc(p, p->trg_tap, sizeof(int4) * nt, "target taps"));
        const int64_t nch = yk::hist_chunks(n_trg, p->nti * p->nti);
        if (nch > 0)
            YK_TRY(buf_alloc(p, p->trg_hist, sizeof(int) * (size_t)nch * p->nti * p->nti,
                             "target histograms"));
    }
    stage_begin(p, YK_STAGE_BIN_SRC);
    if (prep)
        YK_CU(yk::launch_prep_sources(g, n_src, dx, dy, n_dip, ddx, ddy, P<int2>(p->src_tap),
                                      P<float4>(p->src_t), P<int>(p->tile_cnt),
                                      P<int>(p->tile_ptr), P<int>(p->tile_cur),
                                      P<double2>(p->ent_t), P<int>(p->ent_j), P<int>(p->err),
                                      p->stream, true),
              "bin sources");
    else
        YK_CU(yk::launch_bin_sources(g, n_src, dx, dy, n_dip, ddx, ddy, P<double2>(p->src_t),
                                     P<int>(p->tile_cnt), P<int>(p->tile_ptr),
                                     P<int>(p->tile_cur), P<double2>(p->ent_t), P<int>(p->ent_j),
                                     P<int>(p->err), p->stream),
              "bin sources");
    /* the cursors are free after the fill: they serve as the ordering's scratch */
    YK_CU(yk::launch_tile_order(P<int>(p->tile_ptr), p->nt * p->nt, P<int>(p->tile_order),
                                P<int>(p->tile_cur), p->stream),
          "tile order");
    if (p->fft_df) {
        /* double-float path: window values once per source (they depend on positions only),
         * in the order of the owner-tile entries (a dipole's entry slot stays unused: dipoles
         * keep their own records) */
        const size_t w = (size_t)p->w;
        YK_TRY(buf_alloc(p, p->win_src, sizeof(float2) * 2 * w * (ns + nd), "source windows"));
        YK_CU(yk::launch_frac_windows_df(g, n_src + n_dip, P<float4>(p->src_t),
                                         P<int>(p->tile_ptr) + (size_t)p->nt * p->nt,
                                         P<float2>(p->win_pc), p->pdeg, false,
                                         P<float2>(p->win_src), p->stream, 0, P<int>(p->ent_j),
                                         n_src),
              "source windows");
        if (nd > 0) {
            /* dipoles in their own order (a dipole outside the box has no entries, and its
             * record is never read) */
            YK_TRY(buf_alloc(p, p->win_dip, sizeof(float2) * 4 * w * nd, "dipole windows"));
            YK_CU(yk::launch_frac_windows_df(g, n_dip, P<float4>(p->src_t) + ns, nullptr,
                                             P<float2>(p->win_pc), p->pdeg, true,
                                             P<float2>(p->win_dip), p->stream),
                  "dipole windows");
        }
    }
    stage_end(p, YK_STAGE_BIN_SRC);
    /* the staging buffers are reused for the targets: order the copies after the source bins */
    const double *tx = nullptr, *ty = nullptr;
    YK_TRY(to_device(p, xt, n_trg, p->stage_x, &tx, "target x"));
    YK_TRY(to_device(p, yt, n_trg, p->stage_y, &ty, "target y"));
    stage_begin(p, YK_STAGE_BIN_TRG);
    if (prep)
        YK_CU(yk::launch_prep_targets(g, n_trg, tx, ty, P<int4>(p->trg_tap), P<float4>(p->trg_tmp),
                                      P<int>(p->trg_cnt), P<int>(p->trg_ptr), P<int>(p->trg_cur),
                                      P<double2>(p->trg_t), nullptr, P<int>(p->trg_idx),
                                      P<int>(p->err), p->stream,
                                      P<int>(p->trg_hist)),
              "bin targets");
    else
        YK_CU(yk::launch_bin_targets(g, n_trg, tx, ty, P<double2>(p->trg_tmp),
                                     P<int>(p->trg_cnt), P<int>(p->trg_ptr), P<int>(p->trg_cur),
                                     P<double2>(p->trg_t), P<int>(p->trg_idx), P<int>(p->err),
                                     p->stream),
              "bin targets");
    if (p->fft_df) {
        YK_TRY(buf_alloc(p, p->win_trg, sizeof(float2) * 2 * (size_t)p->w * nt, "target windows"));
        /* the window arguments are gathered in tile order from the preparation's copy in the
         * original order (trg_tmp) through the targets' indices: the binning then writes no
         * third per-target array at random slots */
        YK_CU(yk::launch_frac_windows_df(g, n_trg, P<float4>(p->trg_tmp),
                                         P<int>(p->trg_ptr) + (size_t)p->nti * p->nti,
                                         P<float2>(p->win_pc), p->pdeg, false,
                                         P<float2>(p->win_trg), p->stream, n_trg,
                                         P<int>(p->trg_idx), n_trg),
              "target windows");
    }
    stage_end(p, YK_STAGE_BIN_TRG);
#undef YK_TRY
    /* host inputs: return after the copies are consumed so the caller may reuse its arrays */
    /* pageable host inputs: return after the copies are consumed so the caller may reuse its
     * arrays (page-locked inputs are copied asynchronously, like device memory) */
    bool pageable = false;
    for (const double *a : {xs, ys, w})
        pageable = pageable || (n_src > 0 && is_pageable_ptr(a));
    for (const double *a : {xd, yd, wd, nx, ny})
        pageable = pageable || (n_dip > 0 && is_pageable_ptr(a));
    for (const double *a : {xt, yt})
        pageable = pageable || (n_trg > 0 && is_pageable_ptr(a));
    if (pageable) {
        s = sync_and_check(p);
        if (s != YK_OK) return s;
    }
    p->points_set = true;
    return YK_OK;
}

yk_status yk_set_points(yk_plan_t p, int64_t n_src, const double *xs, const double *ys,
                        const double *w, int64_t n_trg, const double *xt, const double *yt)
{
    return yk_set_points_dl(p, n_src, xs, ys, w, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                            n_trg, xt, yt);
}

yk_status yk_eval_longrange_dl(yk_plan_t p, const double *density, const double *mu, double *u)
{
    if (!p) return fail(YK_ERR_ARG, "plan is NULL");
    if (!p->points_set) return fail(YK_ERR_STATE, "yk_set_points has not been called");
    if (p->status != YK_OK) return fail((yk_status)p->status, "plan is in an error state");
    if ((p->n_src > 0 && !density) || (p->n_trg > 0 && !u))
        return fail(YK_ERR_ARG, "NULL density or output array");
    if (p->n_dip > 0 && !mu)
        return fail(YK_ERR_ARG, "the plan's points include dipoles: give their density mu "
                                "(yk_eval_longrange_dl)");
    const bool host_u = p->n_trg > 0 && !is_device_ptr(u);
    yk_status s;
    double *du = u;
    if (host_u) {
        if ((s = buf_alloc(p, p->stage_u, sizeof(double) * (size_t)p->n_trg, "output")) != YK_OK)
            return s;
        du = P<double>(p->stage_u);
    }
    if (p->n_trg > 0) {
        if (p->zero || p->n_src + p->n_dip == 0) {
            YK_CU(cudaMemsetAsync(du, 0, sizeof(double) * (size_t)p->n_trg, p->stream), "zero output");
        } else {
            const double *dd = nullptr, *dmu = nullptr;
            if ((s = to_device(p, density, p->n_src, p->stage_w, &dd, "density")) != YK_OK) return s;
            if ((s = to_device(p, mu, p->n_dip, p->stage_d[5], &dmu, "dipole density")) != YK_OK)
                return s;
            yk::Inst d;
            yk_fill_inst(p, &d);
            d.dens = dd;
            d.mu = dmu;
            d.u = du;
            static const char *names[yk::ST_COUNT] = {"spread", "row FFT", "column FFT",
                                                      "row inverse FFT", "interpolation"};
            for (int st = 0; st < yk::ST_COUNT; ++st) {
                stage_begin(p, YK_STAGE_SPREAD + st);
                YK_CU(yk::launch_stage(d, st, p->stream), names[st]);
                stage_end(p, YK_STAGE_SPREAD + st);
            }
        }
    }
    if (host_u) {
        YK_CU(cudaMemcpyAsync(u, du, sizeof(double) * (size_t)p->n_trg, cudaMemcpyDeviceToHost,
                              p->stream),
              "output copy");
        /* a page-locked output is written asynchronously: valid after yk_sync */
        if (is_pageable_ptr(u)) return sync_and_check(p);
    }
    if ((p->n_src > 0 && is_pageable_ptr(density)) || (p->n_dip > 0 && is_pageable_ptr(mu)))
        return sync_and_check(p);
    return YK_OK;
}

yk_status yk_eval_longrange(yk_plan_t p, const double *density, double *u)
{
    if (p && p->n_dip > 0)
        return fail(YK_ERR_ARG, "the plan's points include dipoles: use yk_eval_longrange_dl");
    return yk_eval_longrange_dl(p, density, nullptr, u);
}

yk_status yk_stage_times(yk_plan_t p, double *ms)
{
    if (!p || !ms) return fail(YK_ERR_ARG, "NULL argument");
    if (!p->profile) return fail(YK_ERR_STATE, "plan was created without opts.profile");
    YK_CU(cudaStreamSynchronize(p->stream), "stream synchronize");
    for (int s = 0; s < YK_NUM_STAGES; ++s) {
        ms[s] = -1.0;
        const int64_t runs = p->stage_runs[s];
        const int64_t k = runs < yk_plan_s::kEventRing ? runs : yk_plan_s::kEventRing;
        double sum = 0.0;
        int64_t used = 0;
        for (int64_t r = runs - k; r < runs; ++r) {
            float t = 0.0f;
            const int slot = (int)(r % yk_plan_s::kEventRing);
            if (cudaEventElapsedTime(&t, p->events[slot][2 * s], p->events[slot][2 * s + 1]) ==
                cudaSuccess) {
                sum += t;
                ++used;
            }
        }
        if (used) ms[s] = sum / (double)used;
        p->stage_runs[s] = 0;
    }
    return YK_OK;
}

yk_status yk_sync(yk_plan_t p)
{
    if (!p) return fail(YK_ERR_ARG, "plan is NULL");
    return sync_and_check(p);
}

yk_status yk_destroy(yk_plan_t p)
{
    if (!p) return YK_OK;
    cudaStreamSynchronize(p->stream);
    free_all(p);
    delete p;
    return YK_OK;
}

} /* extern "C" */
