/*
 * yk_local.cu — the local asymptotic parts S_{L,A}[sigma] and D_{L,A}[mu] (Section 2.1, eqs. sla,
 * dla; Section 4.1, the lemmas, eqs. slp_local1 and dlp_local1, through their delta*^2 terms),
 * V_L[f] (eq. vl, the Lemma for V_L) and the dyadic corrections, at targets near the boundary.
 *
 * The boundary arrives as panels of q Gauss-Legendre nodes in the panel parameter t in [-1, 1]
 * (Section 3.2): per panel the node coordinates and the density are turned into Legendre series,
 * so gamma(t), sigma(t) and their derivatives are available anywhere on the panel.  Per
 * target (one thread each): the panels within the locality radius r_loc = sqrt(d*)(12 + 2 alpha
 * sqrt(d*)) (remark on locality, Section 4.1) are listed by a cell grid; the panel with the nearest
 * node is refined by Newton on d/dt |x - gamma(t)|^2 = 0 (Section 3.2, closest point), moving to a
 * neighbouring panel when the root leaves [-1, 1]; at the closest point x0 the lemma's terms are
 * evaluated in FP64 with
 *   c1 = r / sqrt(d*), c2 = alpha sqrt(d*), rho = sign((x - x0) . nu0),
 *   kappa0 = curvature of the boundary graph in the (tangent, outward normal) frame,
 *   Z = 4 c2 exp(-c1^2/4 - c2^2) / sqrt(pi)  (the printed Z lacks the factor c2),
 *   sigma0'' = second arclength derivative of sigma at x0.
 * Targets farther than r_loc from the boundary get 0.
 *
 * The volume local part V_L[f] (Section 2.1, eq. vl; Lemma for V_L, eq. vp_local1, through its
 * delta*^2 term) reuses the same closest-point search: at the near targets the lemma in the frame
 * (tangent xi, inward normal eta) at x0, with f's derivatives at the target rotated into that
 * frame and kappa0 the boundary graph's second derivative there (positive where the domain is
 * convex); elsewhere the interior form (eq. vp_local3).
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "yk_internal.h"

namespace {

using yk::df32;
using yk::df_fast_two_sum;
using yk::df_mul_add;
using yk::df_two_sum;
using yk::operator+;
using yk::operator-;
using yk::operator*;

constexpr int kMaxQ = 32;      /* nodes per panel the library accepts */
constexpr int kMaxCells = 1 << 22;

/* (2n+1)/(n+1) and n/(n+1): the Legendre recurrence without divisions */
__constant__ double c_la[kMaxQ], c_lb[kMaxQ];
__constant__ float c_laf[kMaxQ], c_lbf[kMaxQ];

struct LocalGrid {
    double x0, y0, h; /* cell (i, j) covers [x0 + i h, x0 + (i+1) h) x [y0 + j h, ...) */
    int nx, ny;
};

/* Legendre series of the panel's x, y and sigma relative to their values at the panel's middle
 * node (ref), from the values at the Gauss-Legendre nodes: c_n = sum_k L[n][k] (f_k - f_ref) with
 * L[n][k] = (2n+1)/2 w_k P_n(t_k) (exact for the degree q-1 interpolant).  Relative to the panel,
 * the coefficients' rounding scales with the panel's extent, not with |x| ~ 1: on short panels the
 * t-derivatives (curvature) would otherwise lose most of their digits.  Also writes FP32 copies
 * (coordinates, the middle nodes, the x and y series) for the FP32 search phase. */
__global__ void k_panel_series(int64_t npan, int q, const double *__restrict__ xb,
                               const double *__restrict__ yb, const double *__restrict__ sg,
                               const double *__restrict__ L, double *__restrict__ cx,
                               double *__restrict__ cy, double *__restrict__ cs,
                               float *__restrict__ cxf, float *__restrict__ cyf,
                               float *__restrict__ xbf, float *__restrict__ ybf,
                               float *__restrict__ xmf, float *__restrict__ ymf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npan * q) return;
    const int64_t p = i / q;
    const int n = (int)(i - p * q);
    const int64_t m = p * q + q / 2; /* the reference node */
    const double xr = xb[m], yr = yb[m], sr = sg[m];
    double ax = 0.0, ay = 0.0, as = 0.0, mx = 0.0, my = 0.0, ms = 0.0;
    for (int k = 0; k < q; ++k) {
        const double lk = L[n * q + k];
        const double fx = xb[p * q + k] - xr, fy = yb[p * q + k] - yr, fs = sg[p * q + k] - sr;
        ax += lk * fx;
        ay += lk * fy;
        as += lk * fs;
        mx = fmax(mx, fabs(fx));
        my = fmax(my, fabs(fy));
        ms = fmax(ms, fabs(fs));
    }
    /* a coefficient below the sums' rounding (a few ulp of the values times q) is noise: on a
     * short panel the high coefficients are, and P_n'' (up to n^4/8) would amplify them into the
     * curvature; they are set to zero */
    const double noise = 8.0 * q * 1.1102230246251565e-16;
    cx[i] = (n >= 2 && fabs(ax) < noise * mx) ? 0.0 : ax;
    cy[i] = (n >= 2 && fabs(ay) < noise * my) ? 0.0 : ay;
    cs[i] = (n >= 2 && fabs(as) < noise * ms) ? 0.0 : as;
    cxf[i] = (float)cx[i];
    cyf[i] = (float)cy[i];
    xbf[i] = (float)xb[i];
    ybf[i] = (float)yb[i];
    if (n == q / 2) {
        xmf[p] = (float)xr;
        ymf[p] = (float)yr;
    }
}

/* the boundary's bounding box and longest panel chord, per CTA (grid-strided):
 * out[5 b + 0..4] = {xmin, xmax, ymin, ymax, hmax} over CTA b's share (reduced on the host) */
__global__ void __launch_bounds__(1024) k_extent(int64_t npan, int q, const double *__restrict__ xb,
                                                 const double *__restrict__ yb,
                                                 double *__restrict__ out)
{
    __shared__ double red[5][32];
    double v[5] = {1e300, -1e300, 1e300, -1e300, 0.0};
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                  stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = t0; k < npan * q; k += stride) {
        v[0] = fmin(v[0], xb[k]);
        v[1] = fmax(v[1], xb[k]);
        v[2] = fmin(v[2], yb[k]);
        v[3] = fmax(v[3], yb[k]);
    }
    for (int64_t p = t0; p < npan; p += stride)
        v[4] = fmax(v[4], hypot(xb[p * q + q - 1] - xb[p * q], yb[p * q + q - 1] - yb[p * q]));
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmin(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = fmax(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] = fmin(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
        v[3] = fmax(v[3], __shfl_xor_sync(0xffffffffu, v[3], o));
        v[4] = fmax(v[4], __shfl_xor_sync(0xffffffffu, v[4], o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0)
        for (int j = 0; j < 5; ++j) red[j][w] = v[j];
    __syncthreads();
    if (threadIdx.x < 5) {
        const int j = threadIdx.x;
        double a = red[j][0];
        for (int k = 1; k < nw; ++k) a = (j == 0 || j == 2) ? fmin(a, red[j][k]) : fmax(a, red[j][k]);
        out[5 * blockIdx.x + j] = a;
    }
}

/* the cells a panel's nodes, widened by r_loc, overlap (count, then fill) */
__device__ void panel_cells(const double *xb, const double *yb, int64_t p, int q, double rl,
                            const LocalGrid &G, int &i0, int &i1, int &j0, int &j1)
{
    double xmin = xb[p * q], xmax = xmin, ymin = yb[p * q], ymax = ymin;
    for (int k = 1; k < q; ++k) {
        xmin = fmin(xmin, xb[p * q + k]);
        xmax = fmax(xmax, xb[p * q + k]);
        ymin = fmin(ymin, yb[p * q + k]);
        ymax = fmax(ymax, yb[p * q + k]);
    }
    i0 = max(0, (int)floor((xmin - rl - G.x0) / G.h));
    i1 = min(G.nx - 1, (int)floor((xmax + rl - G.x0) / G.h));
    j0 = max(0, (int)floor((ymin - rl - G.y0) / G.h));
    j1 = min(G.ny - 1, (int)floor((ymax + rl - G.y0) / G.h));
}

__global__ void k_cell_count(int64_t npan, int q, const double *__restrict__ xb,
                             const double *__restrict__ yb, double rl, LocalGrid G,
                             int *__restrict__ cnt)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npan) return;
    int i0, i1, j0, j1;
    panel_cells(xb, yb, p, q, rl, G, i0, i1, j0, j1);
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) atomicAdd(&cnt[j * G.nx + i], 1);
}

__global__ void k_cell_fill(int64_t npan, int q, const double *__restrict__ xb,
                            const double *__restrict__ yb, double rl, LocalGrid G,
                            const int *__restrict__ ptr, int *__restrict__ cur,
                            int *__restrict__ list)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npan) return;
    int i0, i1, j0, j1;
    panel_cells(xb, yb, p, q, rl, G, i0, i1, j0, j1);
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) {
            const int c = j * G.nx + i;
            list[ptr[c] + atomicAdd(&cur[c], 1)] = (int)p;
        }
}

/* value and first two t-derivatives of NS Legendre series (coefficients c[s][0..q)) at t, sharing
 * the recurrences P_{n+1} = ((2n+1) t P_n - n P_{n-1}) / (n+1), P'_{n+1} = P'_{n-1} + (2n+1) P_n,
 * P''_{n+1} = P''_{n-1} + (2n+1) P'_n */
template <typename T, int NS>
__device__ __forceinline__ void legendre_eval(const T *const (&c)[NS], int q, T t, T (&f)[NS],
                                              T (&f1)[NS], T (&f2)[NS], const T *la, const T *lb)
{
    T p0 = 1, p1 = t, d0 = 0, d1 = 1, e0 = 0, e1 = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        f[s] = c[s][0] + c[s][1] * t;
        f1[s] = c[s][1];
        f2[s] = 0;
    }
    for (int n = 1; n + 1 < q; ++n) {
        const T k = (T)(2 * n + 1);
        const T p2 = la[n] * t * p1 - lb[n] * p0;
        const T d2 = d0 + k * p1;
        const T e2 = e0 + k * d1;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const T cn = c[s][n + 1];
            f[s] += cn * p2;
            f1[s] += cn * d2;
            f2[s] += cn * e2;
        }
        p0 = p1;
        p1 = p2;
        d0 = d1;
        d1 = d2;
        e0 = e1;
        e1 = e2;
    }
}

/* the lemma's expansion (eq. slp_local1) through its delta*^2 term; s0p, g3, g4 are sigma0',
 * gamma0''' and gamma0'''' in the tangent-line parameter */
__device__ double lemma_terms(double alpha, double dstar, double r, double rho, double kappa0,
                              double s0, double s0pp, double s0p, double g3, double g4)
{
    const double sd = sqrt(dstar), c1 = r / sd, c2 = alpha * sd;
    const double em = exp(-c1 * c2) * erfc(0.5 * c1 - c2);
    const double ep = exp(c1 * c2) * erfc(0.5 * c1 + c2);
    const double phm = em - ep, php = em + ep;
    const double Z = 4.0 * c2 * exp(-0.25 * c1 * c1 - c2 * c2) * 0.56418958354775628695; /* 1/sqrt(pi) */
    const double P0 = phm / c2, P1 = c1 * P0, P2 = c1 * P1;
    const double Q0 = (phm - Z) / (c2 * c2 * c2) + c1 * php / (c2 * c2);
    const double P3 = c1 * P2, Q1 = c1 * Q0, k = kappa0;
    return sd * s0 * 0.25 * P0 + dstar * rho * k * s0 * 0.125 * P1 +
           dstar * sd * (k * k * s0 / 32.0 * (Q0 + 3.0 * P2) + s0pp * 0.125 * Q0) +
           dstar * dstar * rho *
               (k * k * k * s0 / 64.0 * (5.0 * P3 - 3.0 * Q1) +
                (3.0 / 16.0 * k * s0pp + 0.125 * s0p * g3 + s0 * g4 / 32.0) * Q1);
}

/* cell of each target (-1 outside the grid) and the targets per cell */
__global__ void k_target_cells(int64_t nt, const double *__restrict__ xt,
                               const double *__restrict__ yt, LocalGrid G,
                               const int *__restrict__ pan_ptr, int *__restrict__ tcell,
                               int *__restrict__ tcnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int ci = (int)floor((xt[i] - G.x0) / G.h), cj = (int)floor((yt[i] - G.y0) / G.h);
    int c = -1;
    if (ci >= 0 && ci < G.nx && cj >= 0 && cj < G.ny) {
        c = cj * G.nx + ci;
        if (pan_ptr[c + 1] == pan_ptr[c]) c = -1; /* no panel within r_loc: u = 0 */
    }
    tcell[i] = c;
    if (c >= 0) atomicAdd(&tcnt[c], 1);
}

__global__ void k_target_fill(int64_t nt, const int *__restrict__ tcell,
                              const int *__restrict__ tptr, int *__restrict__ tcur,
                              int *__restrict__ order)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int c = tcell[i];
    if (c >= 0) order[tptr[c] + atomicAdd(&tcur[c], 1)] = (int)i;
}

/* the boundary as the target kernels see it */
struct PanelSet {
    int64_t npan;
    int q;
    const double *xb, *yb;            /* nodes (FP64) */
    const double *cx, *cy, *cs;       /* Legendre series relative to the middle nodes */
    const double *sref;               /* sigma at the nodes (its middle node is cs's reference) */
    const float *cxf, *cyf, *xbf, *ybf, *xmf, *ymf; /* FP32 copies for the search */
    const double *tq;                 /* Gauss-Legendre nodes */
    const int *ptr, *list;            /* panels listed per cell */
    const double *wide;               /* window fits of short panels (k_panel_wide), or NULL */
};

/* Closest boundary point of (x, y), the target's cell c listing at least one panel: panel p and
 * parameter t.  The search runs in FP32 (nearest middle node, nearest node of that panel and its
 * neighbours, Newton on f(t) = (gamma(t) - x) . gamma'(t) to ~1e-5 in t, moving to a neighbour
 * panel when the root leaves [-1, 1], at most twice); Newton then polishes t in FP64, with f
 * evaluated relative to the panel's reference node (quadratic: from ~1e-5 two steps reach the
 * rounding level).  Returns false if the cell lists no panel. */
__device__ bool closest_point(const PanelSet &P, double x, double y, int c, int64_t &pout,
                              double &tout)
{
    const int q = P.q, h = q / 2;
    const float xf = (float)x, yf = (float)y;
    float best = 3.0e38f;
    int64_t p = -1;
    for (int e = P.ptr[c]; e < P.ptr[c + 1]; ++e) {
        const int pp = P.list[e];
        const float dx = P.xmf[pp] - xf, dy = P.ymf[pp] - yf;
        const float d2 = dx * dx + dy * dy;
        if (d2 < best) {
            best = d2;
            p = pp;
        }
    }
    if (p < 0) return false;
    float t = 0.0f;
    {
        const int64_t p0 = p;
        best = 3.0e38f;
        for (int dp = -1; dp <= 1; ++dp) {
            int64_t pp = p0 + dp;
            pp = pp < 0 ? P.npan - 1 : (pp >= P.npan ? 0 : pp);
            for (int k = 0; k < q; ++k) {
                const float dx = P.xbf[pp * q + k] - xf, dy = P.ybf[pp * q + k] - yf;
                const float d2 = dx * dx + dy * dy;
                if (d2 < best) {
                    best = d2;
                    p = pp;
                    t = (float)P.tq[k];
                }
            }
        }
    }
    for (int hop = 0; hop < 3; ++hop) {
        const float ox = (float)(P.xb[p * q + h] - x), oy = (float)(P.yb[p * q + h] - y);
        const float *const cf[2] = {P.cxf + p * q, P.cyf + p * q};
        for (int it = 0; it < 10; ++it) {
            float g[2], g1[2], g2[2];
            legendre_eval<float, 2>(cf, q, t, g, g1, g2, c_laf, c_lbf);
            const float ex = g[0] + ox, ey = g[1] + oy;
            const float f = ex * g1[0] + ey * g1[1];
            const float fp = g1[0] * g1[0] + g1[1] * g1[1] + ex * g2[0] + ey * g2[1];
            float dt = f / fp;
            if (!(fabsf(dt) < 4.0f)) dt = dt > 0.0f ? 4.0f : -4.0f;
            t = fminf(fmaxf(t - dt, -3.0f), 3.0f);
            if (fabsf(dt) < 2e-5f) break;
        }
        if (t > 1.0f && hop < 2) {
            p = p + 1 < P.npan ? p + 1 : 0;
            t = -1.0f;
        } else if (t < -1.0f && hop < 2) {
            p = p > 0 ? p - 1 : P.npan - 1;
            t = 1.0f;
        } else {
            break;
        }
    }
    const double ox = P.xb[p * q + h] - x, oy = P.yb[p * q + h] - y;
    const double *const c2[2] = {P.cx + p * q, P.cy + p * q};
    double td = t;
    bool last = false;
    for (int it = 0; it < 8; ++it) {
        double g[2], g1[2], g2[2];
        legendre_eval<double, 2>(c2, q, td, g, g1, g2, c_la, c_lb);
        const double ex = g[0] + ox, ey = g[1] + oy;
        const double f = ex * g1[0] + ey * g1[1];
        const double fp = g1[0] * g1[0] + g1[1] * g1[1] + ex * g2[0] + ey * g2[1];
        double dt = f / fp;
        if (!(fabs(dt) < 4.0)) dt = dt > 0.0 ? 4.0 : -4.0;
        td = fmin(fmax(td - dt, -3.0), 3.0);
        /* quadratic convergence: after a step of size dt the error is ~ C dt^2 with
         * C = f'' / (2 f').  f' = |gamma'|^2 (1 - d kappa) shrinks for targets at distance d
         * near a concave stretch's radius of curvature 1 / |kappa|, which the locality radius
         * may approach, so C has no useful bound there: once |dt| < 1e-6, one more step is
         * taken, after which the error is ~ C (C 1e-12)^2, below 1e-16 for C up to 1e4 */
        if (last) break;
        last = fabs(dt) < 1e-6;
    }
    pout = p;
    tout = td;
    return true;
}

/* ----------------------------------------------------------------------------------------- */
/* the boundary's derivatives at the closest point on short panels                            */

/* Orders 2 to 4 of the curve's and the density's derivatives come from the panel's own
 * degree-(q-1) series, whose coefficients carry the node rounding (~1e-16 of |x|, not of the
 * panel's span): its k-th derivative amplifies that by ~(2/h)^k q^(2k) on a panel of length h,
 * ~1e-6 of the curvature and nothing usable of the fourth derivative on 1e-3-long panels.  A
 * panel shorter than the window W (0.006 of the boundary's extent) therefore also gets a
 * least-squares fit over the nodes of its 2k + 1 neighbouring panels (covering ~W) in the frame
 * of its middle node: the boundary graph eta(xi) and the density mu(xi), Legendre series of
 * degree kWideDeg in xi / S (S the largest |xi| of the window's nodes).  The kernels take the
 * derivatives of order >= 2 from it where it exists.  Layout per panel: k (0: no fit), S,
 * tangent (2), eta's coefficients, mu's coefficients. */
constexpr int kWideDeg = 8;
constexpr int kWideN = kWideDeg + 1;
constexpr int kWideStride = 4 + 2 * kWideN;

/* value and first four derivatives of NS Legendre series (coefficients c[s][0..n)) at t, with
 * P'''_{m+1} = P'''_{m-1} + (2m+1) P''_m and P''''_{m+1} = P''''_{m-1} + (2m+1) P'''_m as in
 * legendre_eval */
template <int NS>
__device__ __forceinline__ void legendre_eval4(const double *const (&c)[NS], int n, double t,
                                               double (&f)[5][NS])
{
    double p[5][2] = {{1.0, t}, {0.0, 1.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        f[0][s] = c[s][0] + c[s][1] * t;
        f[1][s] = c[s][1];
        f[2][s] = f[3][s] = f[4][s] = 0.0;
    }
    for (int m = 1; m + 1 < n; ++m) {
        const double k = (double)(2 * m + 1);
        double nx[5];
        nx[0] = c_la[m] * t * p[0][1] - c_lb[m] * p[0][0];
#pragma unroll
        for (int d = 1; d < 5; ++d) nx[d] = p[d][0] + k * p[d - 1][1];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const double cn = c[s][m + 1];
#pragma unroll
            for (int d = 0; d < 5; ++d) f[d][s] += cn * nx[d];
        }
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            p[d][0] = p[d][1];
            p[d][1] = nx[d];
        }
    }
}

/* derivatives in the tangent-line parameter xi of F(xi) = f(t(xi)) from the parameter
 * derivatives of f and of xi(t) = (gamma(t) - x0) . tangent (inverse-function chain rule):
 * out[k] = d^(k+1) F / dxi^(k+1), k = 0..3 */
__device__ __forceinline__ void tangent_line(const double (&xi)[4], const double (&f)[4],
                                             double (&out)[4])
{
    const double x1 = xi[0], x2 = xi[1], x3 = xi[2], x4 = xi[3];
    const double i1 = 1.0 / x1, i2 = i1 * i1;
    const double t1 = i1, t2 = -x2 * i2 * i1;
    const double t3 = (3.0 * x2 * x2 - x1 * x3) * i2 * i2 * i1;
    const double t4 = (-15.0 * x2 * x2 * x2 + 10.0 * x1 * x2 * x3 - x1 * x1 * x4) * i2 * i2 * i2 * i1;
    out[0] = f[0] * t1;
    out[1] = f[1] * t1 * t1 + f[0] * t2;
    out[2] = f[2] * t1 * t1 * t1 + 3.0 * f[1] * t1 * t2 + f[0] * t3;
    out[3] = f[3] * t1 * t1 * t1 * t1 + 6.0 * f[2] * t1 * t1 * t2 +
             f[1] * (3.0 * t2 * t2 + 4.0 * t1 * t3) + f[0] * t4;
}

/* Window fit, part 1: one warp per panel (k = 0 for panels at least W long).  The lanes stride
 * over the window's samples, each accumulating its share of the normal equations (the Gram
 * matrix's upper triangle and two right sides) in registers; the shares are summed through
 * shared memory (each lane adds up two of the kWideSys columns) and written to gram[p]. */
constexpr int kWideGram = kWideN * (kWideN + 1) / 2;
constexpr int kWideSys = kWideGram + 2 * kWideN; /* Gram entries, then the two right sides */
constexpr int kWideSamples = 64;

__global__ void __launch_bounds__(64) k_panel_wide(int64_t npan, int q,
                                                    const double *__restrict__ xb,
                                                    const double *__restrict__ yb,
                                                    const double *__restrict__ sg,
                                                    const double *__restrict__ tq, double W,
                                                    double *__restrict__ wide,
                                                    double *__restrict__ gram)
{
    __shared__ double sh[2][32][kWideSys + 1]; /* per warp; the odd row length spreads banks */
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
    if (p >= npan) return; /* warp-uniform; no block-wide barrier follows */
    double *o = wide + p * kWideStride;
    /* panel length from its end nodes' chord, scaled from the nodes' span to [-1, 1]; neighbours
     * on each side (a degenerate panel, h = 0, gives the cap) */
    const double h = hypot(xb[p * q + q - 1] - xb[p * q], yb[p * q + q - 1] - yb[p * q]) * 2.0 /
                     (tq[q - 1] - tq[0]);
    const double kk = fmin(h < W ? ceil(0.5 * (W / h - 1.0)) : 0.0, (double)(npan / 8));
    const int k = (int)kk;
    if (lane == 0) o[0] = (double)k;
    if (k <= 0) return;
    /* the frame: origin at the middle node, xi along the chord of the panel's end nodes (any
     * direction over which the short stretch is a graph serves: the derivatives at x0 are taken
     * in x0's own tangent-line parameter afterwards) */
    const int64_t m = p * q + q / 2;
    const double cxe = xb[p * q + q - 1] - xb[p * q], cye = yb[p * q + q - 1] - yb[p * q];
    const double ce = sqrt(cxe * cxe + cye * cye);
    const double tx = cxe / ce, ty = cye / ce;
    const double xm = xb[m], ym = yb[m], sm = sg[m];
    /* the window's nodes, or an even subsample of kWideSamples of them (the fit's noise grows
     * only as the square root of the thinning) */
    const int nn = (2 * k + 1) * q, ns = min(nn, kWideSamples);
    auto node = [&](int j) { /* j-th sample of the window, panel p - k first */
        const int jj = (int)(((int64_t)j * nn) / ns), jp = jj / q;
        int64_t pp = p - k + jp;
        pp += pp < 0 ? npan : (pp >= npan ? -npan : 0);
        return pp * q + (jj - jp * q);
    };
    /* the window spans a short, nearly straight stretch: its largest |xi| is at an end sample */
    double S = 0.0;
    if (lane < 2) {
        const int64_t v = node(lane ? ns - 1 : 0);
        S = fabs((xb[v] - xm) * tx + (yb[v] - ym) * ty);
    }
    S = fmax(__shfl_sync(0xffffffffu, S, 0), __shfl_sync(0xffffffffu, S, 1));
    double acc[kWideSys];
#pragma unroll
    for (int i = 0; i < kWideSys; ++i) acc[i] = 0.0;
    for (int j = lane; j < ns; j += 32) {
        const int64_t v = node(j);
        const double dx = xb[v] - xm, dy = yb[v] - ym;
        const double s = (dx * tx + dy * ty) / S, eta = dx * ty - dy * tx, mu = sg[v] - sm;
        double P[kWideN];
        P[0] = 1.0;
        P[1] = s;
#pragma unroll
        for (int n = 1; n + 1 < kWideN; ++n) P[n + 1] = c_la[n] * s * P[n] - c_lb[n] * P[n - 1];
        int a = 0;
#pragma unroll
        for (int i = 0; i < kWideN; ++i)
#pragma unroll
            for (int j2 = i; j2 < kWideN; ++j2) acc[a++] += P[i] * P[j2];
#pragma unroll
        for (int i = 0; i < kWideN; ++i) {
            acc[kWideGram + i] += P[i] * eta;
            acc[kWideGram + kWideN + i] += P[i] * mu;
        }
    }
#pragma unroll
    for (int i = 0; i < kWideSys; ++i) sh[wrp][lane][i] = acc[i];
    __syncwarp();
    for (int c = lane; c < kWideSys; c += 32) {
        double v = 0.0;
        for (int l = 0; l < 32; ++l) v += sh[wrp][l][c];
        gram[p * kWideSys + c] = v;
    }
    if (lane == 0) {
        o[1] = S;
        o[2] = tx;
        o[3] = ty;
    }
}

/* Window fit, part 2: one thread per panel solves its system by Cholesky (the factor in a
 * square array) and two triangular solves per right side, writing the series' coefficients */
__global__ void k_panel_wide_solve(int64_t npan, const double *__restrict__ gram,
                                   double *__restrict__ wide)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npan) return;
    double *o = wide + p * kWideStride;
    if (!(o[0] > 0.0)) return;
    const double *G = gram + p * kWideSys;
    double L[kWideN][kWideN], be[kWideN], bm[kWideN];
    {
        int a = 0;
        for (int i = 0; i < kWideN; ++i)
            for (int j2 = i; j2 < kWideN; ++j2) L[j2][i] = G[a++]; /* lower triangle holds A */
        for (int i = 0; i < kWideN; ++i) {
            be[i] = G[kWideGram + i];
            bm[i] = G[kWideGram + kWideN + i];
        }
    }
    for (int j = 0; j < kWideN; ++j) {
        double d = L[j][j];
        for (int l = 0; l < j; ++l) d -= L[j][l] * L[j][l];
        d = sqrt(fmax(d, 1e-300));
        L[j][j] = d;
        for (int i = j + 1; i < kWideN; ++i) {
            double v = L[i][j];
            for (int l = 0; l < j; ++l) v -= L[i][l] * L[j][l];
            L[i][j] = v / d;
        }
    }
    for (int i = 0; i < kWideN; ++i) {
        for (int l = 0; l < i; ++l) {
            be[i] -= L[i][l] * be[l];
            bm[i] -= L[i][l] * bm[l];
        }
        be[i] /= L[i][i];
        bm[i] /= L[i][i];
    }
    for (int i = kWideN - 1; i >= 0; --i) {
        for (int l = i + 1; l < kWideN; ++l) {
            be[i] -= L[l][i] * be[l];
            bm[i] -= L[l][i] * bm[l];
        }
        be[i] /= L[i][i];
        bm[i] /= L[i][i];
    }
    for (int i = 0; i < kWideN; ++i) {
        o[4 + i] = be[i];
        o[4 + kWideN + i] = bm[i];
    }
}

/* tangent-line derivatives at the point x0 = (middle node) + (dx0, dy0) of panel p from its
 * window fit: G[k] = d^(k+1) gamma / dxi^(k+1) of the boundary graph in the frame (tangent,
 * outward normal) at x0 (G[0] = 0, G[1] = kappa0), M[k] the density's; false where the panel
 * has no fit (its own series serves) */
__device__ bool wide_derivs(const PanelSet &P, int64_t p, double dx0, double dy0,
                            double (&G)[4], double (&M)[4])
{
    if (!P.wide) return false;
    const double *o = P.wide + p * kWideStride;
    if (!(o[0] > 0.0)) return false;
    const double S = o[1], tx = o[2], ty = o[3];
    const double s0 = (dx0 * tx + dy0 * ty) / S;
    const double *const c[2] = {o + 4, o + 4 + kWideN};
    double f[5][2];
    legendre_eval4<2>(c, kWideN, s0, f);
    /* the curve (xi, eta(xi)) of the middle node's frame with xi as its parameter: derivatives
     * (1, e1), (0, e_k); at x0 its unit tangent T = (1, e1)/n1 and outward normal (-e1, 1)/n1 */
    double e[5], mu[4];
    double sc = 1.0;
    for (int d = 1; d < 5; ++d) {
        sc /= S;
        e[d] = f[d][0] * sc;
        mu[d - 1] = f[d][1] * sc;
    }
    const double n1 = sqrt(1.0 + e[1] * e[1]);
    double xi[4], eta[4];
    xi[0] = n1;
    eta[0] = 0.0;
    for (int d = 2; d < 5; ++d) {
        xi[d - 1] = e[d] * e[1] / n1;
        eta[d - 1] = e[d] / n1;
    }
    tangent_line(xi, eta, G);
    tangent_line(xi, mu, M);
    return true;
}

/* S_{L,A}: one thread per near target, the targets grouped by cell (a warp scans one cell's
 * panel list) */
__global__ void __launch_bounds__(128) k_slp_local(int n_near, const int *__restrict__ order,
                                                   const int *__restrict__ tcell,
                                                   const double *__restrict__ xt,
                                                   const double *__restrict__ yt, PanelSet P,
                                                   double alpha, double dstar, double rl,
                                                   double *__restrict__ u)
{
    const int e0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (e0 >= n_near) return;
    const int i = order[e0];
    const double x = xt[i], y = yt[i];
    int64_t p;
    double td;
    if (!closest_point(P, x, y, tcell[i], p, td)) {
        u[i] = 0.0;
        return;
    }
    const int q = P.q, h = q / 2;
    const double *const c3[3] = {P.cx + p * q, P.cy + p * q, P.cs + p * q};
    double f[5][3];
    legendre_eval4<3>(c3, q, td, f);
    const double s = f[0][2] + P.sref[p * q + h];
    const double st = sqrt(f[1][0] * f[1][0] + f[1][1] * f[1][1]);
    const double tx = f[1][0] / st, ty = f[1][1] / st;
    const double nux = ty, nuy = -tx; /* outward (counter-clockwise) */
    const double dx = (x - P.xb[p * q + h]) - f[0][0], dy = (y - P.yb[p * q + h]) - f[0][1];
    const double r = sqrt(dx * dx + dy * dy);
    double val = 0.0;
    if (r < rl) {
        const double rho = dx * nux + dy * nuy >= 0.0 ? 1.0 : -1.0;
        /* tangent-line derivatives: kappa0 = gamma'', gamma''', gamma'''' of the boundary graph,
         * sigma0', sigma0'' (orders >= 2 from the window fit on short panels) */
        double xi[4], eta[4], mt[4], G[4], M[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            xi[d] = f[d + 1][0] * tx + f[d + 1][1] * ty;
            eta[d] = f[d + 1][0] * nux + f[d + 1][1] * nuy;
            mt[d] = f[d + 1][2];
        }
        tangent_line(xi, eta, G);
        tangent_line(xi, mt, M);
        double Gw[4], Mw[4];
        if (wide_derivs(P, p, f[0][0], f[0][1], Gw, Mw))
            for (int d = 1; d < 4; ++d) {
                G[d] = Gw[d];
                M[d] = Mw[d];
            }
        val = lemma_terms(alpha, dstar, r, rho, G[1], s, M[1], M[0], G[2], G[3]);
    }
    u[i] = val;
}

/* the double-layer lemma's expansion (eq. dlp_local1) through the delta*^2 term, with the sign
 * of the source-point normal derivative (the history part's convention: the printed expansion
 * is the negative of this), and with the gamma'''' part of the delta*^{3/2} bracket multiplying
 * 3 Q0 + P2 (expanding eq. dla gives that factor; the printed 3 Q0 - U3 belongs to the kappa0^3
 * part only, and both agree on the boundary) */
__device__ double dla_lemma_terms(double alpha, double dstar, double r, double rho, double k,
                                  double mu0, double mu1, double mu2, double mu4, double g3,
                                  double g4)
{
    const double sd = sqrt(dstar), c1 = r / sd, c2 = alpha * sd;
    const double em = exp(-c1 * c2) * erfc(0.5 * c1 - c2);
    const double ep = exp(c1 * c2) * erfc(0.5 * c1 + c2);
    const double phm = em - ep, php = em + ep;
    const double Z = 4.0 * c2 * exp(-0.25 * c1 * c1 - c2 * c2) * 0.56418958354775628695; /* 1/sqrt(pi) */
    const double P0 = phm / c2, P1 = c1 * P0, P2 = c1 * P1, P3 = c1 * P2;
    const double Q0 = (phm - Z) / (c2 * c2 * c2) + c1 * php / (c2 * c2), Q1 = c1 * Q0;
    const double U0 = php, U1 = c1 * U0, U2 = c1 * U1, U3 = c1 * U2, U4 = c1 * U3;
    const double k2 = k * k;
    const double t0 = rho * mu0 * 0.25 * U0;
    const double t1 = sd * k * mu0 * 0.125 * (P0 + U1);
    const double t2 = dstar * rho * (mu2 * 0.125 * P1 + 3.0 / 32.0 * k2 * mu0 * (P1 + U2));
    const double t3 = dstar * sd *
                      (5.0 / 64.0 * k2 * k * mu0 * (3.0 * Q0 - U3) -
                       mu0 * g4 / 32.0 * (3.0 * Q0 + P2) - 3.0 / 16.0 * k * mu2 * (Q0 + P2) -
                       mu1 * g3 * 0.125 * (2.0 * Q0 + P2));
    const double t4 = dstar * dstar * rho *
                      (35.0 / 512.0 * k2 * k2 * mu0 * (9.0 * Q1 + 2.0 * P3 - U4) -
                       mu4 / 32.0 * Q1 - 15.0 / 64.0 * k2 * mu2 * (Q1 + P3) -
                       5.0 / 16.0 * k * mu1 * g3 * (2.0 * Q1 + P3) -
                       (5.0 / 64.0 * k * mu0 * g4 + 5.0 / 96.0 * mu0 * g3 * g3) * (3.0 * Q1 + P3));
    return t0 + t1 + t2 - t3 - t4;
}

/* D_{L,A}: one thread per near target, as k_slp_local; the curve's and the density's first four
 * derivatives at the closest point come from the panel's Legendre series and are turned into
 * tangent-line derivatives (kappa0 = gamma'', gamma''', gamma'''' of the boundary graph in the
 * frame (tangent, outward normal); mu', mu'', mu'''').  A target within 1e-10 sqrt(delta*) of the
 * boundary is on it (rho = 0: the corollary's value, eq. dlp_local2); elsewhere rho = +-1 and the
 * value carries the layer's jump. */
__global__ void __launch_bounds__(128) k_dla_local(int n_near, const int *__restrict__ order,
                                                   const int *__restrict__ tcell,
                                                   const double *__restrict__ xt,
                                                   const double *__restrict__ yt, PanelSet P,
                                                   double alpha, double dstar, double rl,
                                                   double *__restrict__ u)
{
    const int e0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (e0 >= n_near) return;
    const int i = order[e0];
    const double x = xt[i], y = yt[i];
    int64_t p;
    double td;
    if (!closest_point(P, x, y, tcell[i], p, td)) {
        u[i] = 0.0;
        return;
    }
    const int q = P.q, h = q / 2;
    const double *const c3[3] = {P.cx + p * q, P.cy + p * q, P.cs + p * q};
    double f[5][3];
    legendre_eval4<3>(c3, q, td, f);
    const double st = sqrt(f[1][0] * f[1][0] + f[1][1] * f[1][1]);
    const double tx = f[1][0] / st, ty = f[1][1] / st;
    const double nux = ty, nuy = -tx; /* outward (counter-clockwise) */
    const double dx = (x - P.xb[p * q + h]) - f[0][0], dy = (y - P.yb[p * q + h]) - f[0][1];
    const double r = sqrt(dx * dx + dy * dy);
    double val = 0.0;
    if (r < rl) {
        double xi[4], eta[4], mt[4], G[4], M[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            xi[d] = f[d + 1][0] * tx + f[d + 1][1] * ty;
            eta[d] = f[d + 1][0] * nux + f[d + 1][1] * nuy;
            mt[d] = f[d + 1][2];
        }
        tangent_line(xi, eta, G);
        tangent_line(xi, mt, M);
        double Gw[4], Mw[4];
        if (wide_derivs(P, p, f[0][0], f[0][1], Gw, Mw)) /* short panel: orders >= 2 */
            for (int d = 1; d < 4; ++d) {
                G[d] = Gw[d];
                M[d] = Mw[d];
            }
        const double side = dx * nux + dy * nuy;
        const double rho = r <= 1e-10 * sqrt(dstar) ? 0.0 : (side >= 0.0 ? 1.0 : -1.0);
        const double mu0 = f[0][2] + P.sref[p * q + h];
        val = dla_lemma_terms(alpha, dstar, r, rho, G[1], mu0, M[0], M[1], M[3], G[2], G[3]);
    }
    u[i] = val;
}

/* V_L beyond the locality radius (corollary, eq. vp_local3): f and its Laplacian only */
__device__ __forceinline__ double vl_interior(double alpha, double dstar, double f, double lap)
{
    const double c2s = alpha * alpha * dstar, e2 = exp(-c2s);
    /* 1 - e^{-c} and 1 - (1 + c) e^{-c} without cancellation for small c */
    const double a1 = -expm1(-c2s);
    const double a2 = a1 - c2s * e2;
    return dstar * f / c2s * a1 + dstar * dstar * lap / (c2s * c2s) * a2;
}

/* The lemma's P1, Q0, W0, W1 for small c2.  The printed W0 = (4 - 4 e^{-c2^2} + 2 lambda -
 * Phi_+) / c2^2 has an O(c2^2) numerator made of O(1) terms, so in FP64 it loses ~1e-16 / c2^2.
 * Instead: g = e^{-c1 c2} erfc(c1/2 - c2) and h = e^{c1 c2} erfc(c1/2 + c2) satisfy
 * g' = -c1 g + G e^{-c2^2}, h' = c1 h - G e^{-c2^2} (d/dc2, G = 2 e^{-c1^2/4} / sqrt(pi)), so
 * Phi_+ = g + h and Phi_- = g - h have the Taylor coefficients p_n, m_n in c2 of
 *   (n+1) p_{n+1} = -c1 m_n,  (n+1) m_{n+1} = -c1 p_n + 2 G e_n,  p_0 = 2 erfc(c1/2), m_0 = 0,
 * e_n those of e^{-c2^2}.  Dividing the series by the powers of c2 term by term leaves sums with
 * no cancellation (the leading term of W0 is the remark's 4 - (2 + c1^2) E + c1 G). */
__device__ void lemma_small_c2(double c1, double c2, double &P1, double &Q0, double &W0,
                               double &W1)
{
    const double E = erfc(0.5 * c1), G = 1.1283791670955126 * exp(-0.25 * c1 * c1);
    double p = 2.0 * E, m = 0.0;   /* p_n, m_n */
    double en = 1.0;               /* e_n for even n */
    double c2n = 1.0;              /* c2^n */
    const double ic2 = 1.0 / c2, ic2s = ic2 * ic2;
    P1 = Q0 = W0 = W1 = 0.0;
    for (int n = 0; n < 90; ++n) {
        const bool even = (n & 1) == 0;
        const double e_n = even ? en : 0.0;
        if (even && n >= 2) {
            const double w0n = (2.0 * E - 4.0) * e_n - p; /* W0's coefficient of c2^{n-2} */
            W0 += w0n * c2n * ic2s;
            Q0 += (c1 * p - G * 2.0 * e_n) * c2n * ic2s;
            W1 += (4.0 * E - 8.0) * e_n * c2n * ic2s;
            if (n >= 4) W1 += 2.0 * w0n * c2n * ic2s * ic2s;
        }
        if (!even) {
            P1 += c1 * m * c2n * ic2;
            if (n >= 3) {
                Q0 += m * c2n * ic2s * ic2;
                W1 -= c1 * m * c2n * ic2s * ic2;
            }
        }
        /* next coefficients */
        const double pn1 = -c1 * m / (n + 1), mn1 = (-c1 * p + 2.0 * G * e_n) / (n + 1);
        p = pn1;
        m = mn1;
        if (even) en = -en / (n / 2 + 1); /* e_{n+2} = -e_n / (n/2 + 1) */
        c2n *= c2;
        if (n >= 12 && fabs(p) * c2n < 1e-19 * c2 * c2 && fabs(m) * c2n < 1e-19 * c2 * c2 &&
            fabs(en) * c2n < 1e-19 * c2 * c2)
            break;
    }
}

/* V_L by the lemma (eq. vp_local1) through the delta*^2 term */
__device__ double vl_lemma_terms(double alpha, double dstar, double r, double kappa0, double f,
                                 double f_eta, double f_etaeta, double f_xixi)
{
    const double sd = sqrt(dstar), c1 = r / sd, c2 = alpha * sd;
    double P1, Q0, W0, W1;
    if (c2 < 0.5) {
        lemma_small_c2(c1, c2, P1, Q0, W0, W1);
    } else {
        const double em = exp(-c1 * c2) * erfc(0.5 * c1 - c2);
        const double ep = exp(c1 * c2) * erfc(0.5 * c1 + c2);
        const double phm = em - ep, php = em + ep;
        const double Z = 4.0 * c2 * exp(-0.25 * c1 * c1 - c2 * c2) * 0.56418958354775628695;
        P1 = c1 * phm / c2;
        Q0 = (phm - Z) / (c2 * c2 * c2) + c1 * php / (c2 * c2);
        const double e2 = exp(-c2 * c2), lam = e2 * erfc(0.5 * c1);
        W0 = (4.0 - 4.0 * e2 + 2.0 * lam - php) / (c2 * c2);
        W1 = (2.0 * W0 - P1 + 4.0 * (lam - 2.0 * e2)) / (c2 * c2);
    }
    const double Q1 = c1 * Q0;
    return dstar * f * 0.25 * W0 + dstar * sd * (2.0 * f_eta - f * kappa0) * 0.125 * Q0 +
           dstar * dstar *
               ((f_eta * kappa0 * 0.125 - 3.0 * f * kappa0 * kappa0 / 32.0 - f_etaeta * 0.125) * Q1 +
                (f_etaeta + f_xixi) * 0.125 * W1);
}

/* every target: eq. vp_local3 (the near targets are overwritten by k_vp_local) */
__global__ void k_vp_interior(int64_t nt, const double *__restrict__ fd, double alpha, double dstar,
                              double *__restrict__ u)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    u[i] = vl_interior(alpha, dstar, fd[i], fd[3 * nt + i] + fd[5 * nt + i]);
}

/* V_L at the near targets: closest point, then the lemma in the frame (tangent xi, inward normal
 * eta) at x0; a target found outside the domain (on the outward side, beyond rounding) gets NaN
 * and is counted */
__global__ void __launch_bounds__(128) k_vp_local(int n_near, const int *__restrict__ order,
                                                  const int *__restrict__ tcell,
                                                  const double *__restrict__ xt,
                                                  const double *__restrict__ yt, int64_t nt,
                                                  const double *__restrict__ fd, PanelSet P,
                                                  double alpha, double dstar, double rl,
                                                  double *__restrict__ u, int *__restrict__ nout)
{
    const int e0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (e0 >= n_near) return;
    const int i = order[e0];
    const double x = xt[i], y = yt[i];
    int64_t p;
    double td;
    if (!closest_point(P, x, y, tcell[i], p, td)) return; /* keeps the interior value */
    const int q = P.q, h = q / 2;
    const double *const c2[2] = {P.cx + p * q, P.cy + p * q};
    double g[2], g1[2], g2[2];
    legendre_eval<double, 2>(c2, q, td, g, g1, g2, c_la, c_lb);
    const double st = sqrt(g1[0] * g1[0] + g1[1] * g1[1]);
    const double tx = g1[0] / st, ty = g1[1] / st; /* tangent xi */
    const double ex = -ty, ey = tx;                 /* inward normal eta (counter-clockwise) */
    const double dx = (x - P.xb[p * q + h]) - g[0], dy = (y - P.yb[p * q + h]) - g[1];
    const double r = sqrt(dx * dx + dy * dy);
    if (!(r < rl)) return;                          /* keeps the interior value */
    if (dx * ex + dy * ey < 0.0 && r > 1e-8 * sqrt(dstar)) {
        u[i] = nan("");
        atomicAdd(nout, 1);
        return;
    }
    double kappa0 = (g1[0] * g2[1] - g1[1] * g2[0]) / (st * st * st);
    double Gw[4], Mw[4];
    if (wide_derivs(P, p, g[0], g[1], Gw, Mw)) kappa0 = -Gw[1]; /* short panel: the window fit */
    const double f = fd[i], fx = fd[nt + i], fy = fd[2 * nt + i];
    const double fxx = fd[3 * nt + i], fxy = fd[4 * nt + i], fyy = fd[5 * nt + i];
    const double f_eta = fx * ex + fy * ey;
    const double f_etaeta = fxx * ex * ex + 2.0 * fxy * ex * ey + fyy * ey * ey;
    const double f_xixi = fxx * tx * tx + 2.0 * fxy * tx * ty + fyy * ty * ty;
    u[i] = vl_lemma_terms(alpha, dstar, r, kappa0, f, f_eta, f_etaeta, f_xixi);
}

/* ----------------------------------------------------------------------------------------- */
/* dyadic corrections S_{L,D}^{(j)} (eqs. slp_dyad, sld): per level j the panels are resampled on
 * m_j sub-panels of the same Gauss-Legendre rule (from the panel's Legendre series, i.e. the
 * interpolation of the paper's bisection), the nodes binned in cells of edge R_j, and every near
 * target sums K_j(|x - x'|) sigma ds over the nodes within R_j, K_j from a table */

constexpr int kDyDeg = 8;          /* degree of the table's pieces */
constexpr double kDyPiece = 0.5;   /* their width in rho = r^2 / (4 delta_j) */

struct DyLevel {
    df32 inv4d;        /* 1 / (kDyPiece 4 delta_j): the piece coordinate */
    float R2f;         /* FP32 screen radius^2: R_j widened past the FP32 distance error */
    float R2;          /* R_j^2 (K_j is below 1e-16 of its peak beyond R_j) */
    int npc;           /* table pieces */
    const float2 *tab; /* npc x (kDyDeg + 1) monomial coefficients in z = 2 (rho' - k) - 1, as
                          double-float pairs */
    const float *Xf, *Yf; /* the sorted nodes' coordinates: high words (also the FP32 screen) */
    const float *Xl, *Yl; /* and low words */
    LocalGrid G;       /* cells of edge >= R_j */
    const int *ptr;    /* nodes per cell */
    const float2 *Q;   /* density |gamma'| w of the sorted nodes, double-float */
    const float2 *NX, *NY; /* outward unit normals (double layer, double-float), else NULL */
};

/* node (p, s, k): parameter -1 + (2 s + 1 + t_k) / m of panel p */
__global__ void k_dy_nodes(int64_t npan, int q, int m, PanelSet P, const double *__restrict__ wq,
                           double *__restrict__ X, double *__restrict__ Y, double *__restrict__ Q,
                           double *__restrict__ NX, double *__restrict__ NY)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)m * q;
    if (i >= npan * per) return;
    const int64_t p = i / per;
    const int rem = (int)(i - p * per), sb = rem / q, k = rem - sb * q;
    const double t = -1.0 + (2.0 * sb + 1.0 + P.tq[k]) / m;
    const double *const c3[3] = {P.cx + p * q, P.cy + p * q, P.cs + p * q};
    double g[3], g1[3], g2[3];
    legendre_eval<double, 3>(c3, q, t, g, g1, g2, c_la, c_lb);
    const int h = q / 2;
    X[i] = P.xb[p * q + h] + g[0];
    Y[i] = P.yb[p * q + h] + g[1];
    const double sp = sqrt(g1[0] * g1[0] + g1[1] * g1[1]);
    Q[i] = (P.sref[p * q + h] + g[2]) * sp * wq[k] / m;
    if (NX) { /* outward normal of the counter-clockwise boundary */
        NX[i] = g1[1] / sp;
        NY[i] = -g1[0] / sp;
    }
}

__device__ __forceinline__ int pt_cell(double x, double y, const LocalGrid &G)
{
    int ci = (int)floor((x - G.x0) / G.h), cj = (int)floor((y - G.y0) / G.h);
    ci = min(max(ci, 0), G.nx - 1);
    cj = min(max(cj, 0), G.ny - 1);
    return cj * G.nx + ci;
}

__global__ void k_pt_count(int64_t n, const double *__restrict__ X, const double *__restrict__ Y,
                           LocalGrid G, int *__restrict__ cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[pt_cell(X[i], Y[i], G)], 1);
}

/* the nodes sorted by cell, as double-float pairs (the high words of the coordinates double as
 * the FP32 screen) */
__device__ __forceinline__ float2 df_pair(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

__global__ void k_pt_fill(int64_t n, const double *__restrict__ X, const double *__restrict__ Y,
                          const double *__restrict__ Q, const double *__restrict__ NX,
                          const double *__restrict__ NY, LocalGrid G, const int *__restrict__ ptr,
                          int *__restrict__ cur, float *__restrict__ Xf, float *__restrict__ Xl,
                          float *__restrict__ Yf, float *__restrict__ Yl, float2 *__restrict__ Qs,
                          float2 *__restrict__ NXs, float2 *__restrict__ NYs)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = pt_cell(X[i], Y[i], G);
    const int e = ptr[c] + atomicAdd(&cur[c], 1);
    const float2 x = df_pair(X[i]), y = df_pair(Y[i]);
    Xf[e] = x.x;
    Xl[e] = x.y;
    Yf[e] = y.x;
    Yl[e] = y.y;
    Qs[e] = df_pair(Q[i]);
    if (NX) {
        NXs[e] = df_pair(NX[i]);
        NYs[e] = df_pair(NY[i]);
    }
}

/* per near target of a level: its cell in the level's grid and its coordinates as FP32 pairs,
 * computed once (one thread per target) instead of by every lane of the target's warp */
__global__ void k_dy_targets(int n_near, const int *__restrict__ order,
                             const double *__restrict__ xt, const double *__restrict__ yt,
                             LocalGrid G, int2 *__restrict__ cell, float4 *__restrict__ xy)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_near) return;
    const int i = order[w];
    const double x = xt[i], y = yt[i];
    const double fx = floor((x - G.x0) / G.h), fy = floor((y - G.y0) / G.h);
    /* outside the cells' reach: no node lies within R_j (marked by an x cell below -1) */
    const bool in = fx >= -1.0 && fx <= G.nx && fy >= -1.0 && fy <= G.ny;
    cell[w] = in ? make_int2((int)fx, (int)fy) : make_int2(-2, -2);
    const float2 px = df_pair(x), py = df_pair(y);
    xy[w] = make_float4(px.x, px.y, py.x, py.y);
}

/* u_i += S_{L,D}^{(j)} at the near targets: one warp per target (the targets grouped by cell),
 * the lanes striding over the nodes of the 3 x 3 cells around it (sorted by cell, so the loads are
 * contiguous), each node screened in FP32 and, within R_j, its term q K_j(r) evaluated in
 * double-float arithmetic (distance, table piece, Horner, accumulation: B300 runs FP32 pairs much
 * faster than FP64); lane sums combined by shuffles in a fixed order */
__global__ void __launch_bounds__(256) k_dyadic_level(int n_near, const int *__restrict__ order,
                                                      const int2 *__restrict__ tcell,
                                                      const float4 *__restrict__ txy, DyLevel L,
                                                      double *__restrict__ u)
{
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= n_near) return; /* whole warps leave together */
    const int2 tc = tcell[w];
    if (tc.x < -1) return; /* no node within R_j */
    const int i = order[w];
    const float4 p4 = txy[w];
    const df32 xd(p4.x, p4.y), yd(p4.z, p4.w);
    const float xf = xd.hi, yf = yd.hi;
    const LocalGrid &G = L.G;
    const int ci = tc.x, cj = tc.y;
    df32 acc(0.0f, 0.0f);
    for (int dj = -1; dj <= 1; ++dj) {
        const int cy = cj + dj;
        if (cy < 0 || cy >= G.ny) continue;
        /* the three cells of a row are contiguous in the sorted order */
        const int c0 = cy * G.nx + max(ci - 1, 0), c1 = cy * G.nx + min(ci + 1, G.nx - 1);
        if (ci + 1 < 0 || ci - 1 >= G.nx) continue;
        for (int e = L.ptr[c0] + lane; e < L.ptr[c1 + 1]; e += 32) {
            const float xh = L.Xf[e], yh = L.Yf[e];
            const float dxf = xh - xf, dyf = yh - yf;
            if (!(dxf * dxf + dyf * dyf < L.R2f)) continue; /* FP32 screen */
            const df32 dx = df32(xh, L.Xl[e]) - xd, dy = df32(yh, L.Yl[e]) - yd;
            const df32 r2 = df_mul_add(dx * dx, dy, dy);
            if (!(r2.hi < L.R2)) continue;
            const df32 rho = r2 * L.inv4d;
            const int k = max(0, min((int)rho.hi, L.npc - 1));
            /* z = 2 (rho - k) - 1: rho.hi - k is exact, the rest by one two-sum */
            const df32 zs = df_two_sum(YK_FMUL(2.0f, YK_FSUB(rho.hi, (float)k)), -1.0f);
            const df32 z = df_fast_two_sum(zs.hi, YK_FADD(zs.lo, YK_FMUL(2.0f, rho.lo)));
            const float2 *a = L.tab + k * (kDyDeg + 1);
            df32 f(a[kDyDeg].x, a[kDyDeg].y);
#pragma unroll
            for (int n = kDyDeg - 1; n >= 0; --n) f = df_mul_add(df32(a[n].x, a[n].y), f, z);
            const float2 qv = L.Q[e];
            df32 qe(qv.x, qv.y);
            if (L.NX) { /* double layer: nu' . (x - x') = -(nu'_x dx + nu'_y dy) */
                const float2 nx = L.NX[e], ny = L.NY[e];
                qe = -(qe * df_mul_add(df32(nx.x, nx.y) * dx, df32(ny.x, ny.y), dy));
            }
            acc = df_mul_add(acc, qe, f);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const df32 v(__shfl_xor_sync(0xffffffffu, acc.hi, o),
                     __shfl_xor_sync(0xffffffffu, acc.lo, o));
        acc = acc + v;
    }
    if (lane == 0) u[i] += acc.to_double();
}

/* K_j on the pieces [k, k + 1] kDyPiece of rho = r^2 / (4 delta_j):
 * K_j = (1/4 pi) int_0^{ln 4} exp(-rho e^{-u} - alpha^2 delta_j e^u) du (t = delta_j e^u), by
 * 3 x 48 Gauss-Legendre nodes in u; each piece interpolated at its kDyDeg + 1 Chebyshev points
 * and written as a polynomial in z = 2 (rho / kDyPiece - k) - 1 (degree 8 on width 0.5: within
 * ~1e-16 of the piece's values, the fastest component being e^{-rho}) */
void dyadic_table_build(double c, int npc, double dj, bool dl, std::vector<double> &tab)
{
    constexpr int NG = 48, NP = 3, D = kDyDeg;
    static const struct Rule {
        double x[NG], w[NG];
        Rule() { yk_gauss_legendre(NG, x, w); }
    } rule; /* initialised once, thread-safely */
    const double *gx = rule.x, *gw = rule.w;
    const double L4 = std::log(4.0);
    auto K = [&](double rho) {
        double acc = 0.0;
        for (int p = 0; p < NP; ++p) {
            const double a = L4 * p / NP, b = L4 * (p + 1) / NP;
            for (int n = 0; n < NG; ++n) {
                const double uu = 0.5 * (b - a) * gx[n] + 0.5 * (a + b);
                const double wgt = dl ? std::exp(-uu) : 1.0; /* dt / t^2 = e^{-u} du / delta_j */
                acc += 0.5 * (b - a) * gw[n] * wgt *
                       std::exp(-rho * std::exp(-uu) - c * std::exp(uu));
            }
        }
        return dl ? acc / (8.0 * M_PI * dj) : acc / (4.0 * M_PI);
    };
    /* Chebyshev T_n as monomials in z */
    double T[D + 1][D + 1] = {};
    T[0][0] = 1.0;
    T[1][1] = 1.0;
    for (int n = 2; n <= D; ++n)
        for (int k = 0; k <= n; ++k)
            T[n][k] = (k > 0 ? 2.0 * T[n - 1][k - 1] : 0.0) - T[n - 2][k];
    tab.assign((size_t)npc * (D + 1), 0.0);
    double f[D + 1], zc[D + 1];
    for (int i = 0; i <= D; ++i) zc[i] = std::cos(M_PI * (i + 0.5) / (D + 1));
    for (int k = 0; k < npc; ++k) {
        for (int i = 0; i <= D; ++i) f[i] = K(kDyPiece * (k + 0.5 * (zc[i] + 1.0)));
        for (int n = 0; n <= D; ++n) {
            double an = 0.0;
            for (int i = 0; i <= D; ++i) an += f[i] * std::cos(n * M_PI * (i + 0.5) / (D + 1));
            an *= 2.0 / (D + 1);
            if (n == 0) an *= 0.5;
            for (int m = 0; m <= n; ++m) tab[(size_t)k * (D + 1) + m] += an * T[n][m];
        }
    }
}

/* tables are reused across calls with the same (alpha^2 delta_j, pieces) (a Rothe march or a
 * bench repeats them); a small mutex-guarded cache, oldest entry dropped beyond 32 */
void dyadic_table(double c, int npc, double dj, bool dl, std::vector<double> &tab)
{
    struct Entry {
        double c, dj;
        int npc;
        bool dl;
        std::vector<double> tab;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &en : cache)
            if (en.c == c && en.npc == npc && en.dl == dl && (!dl || en.dj == dj)) {
                tab = en.tab;
                return;
            }
    }
    dyadic_table_build(c, npc, dj, dl, tab);
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() >= 32) cache.erase(cache.begin());
    cache.push_back({c, dj, npc, dl, tab});
}

bool is_dev(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

yk_status lfail(yk_status s, const char *msg)
{
    yk_set_last_error(msg);
    return s;
}

/* S_{L,A} (vol false: sigma) or V_L (vol true: fd): shared set-up (extent, panel
 * series, cell lists, near targets grouped by cell), then the part's kernels */
yk_status run_local(const char *name, bool vol, int J, bool dl, double alpha, double delta_star, int64_t n_panels, int q,
                    const double *xb, const double *yb, const double *sigma, int64_t n_trg,
                    const double *xt, const double *yt, const double *fd, double *u, void *stream)
{
    char msg[160];
    auto fail = [&](yk_status code, const char *what) {
        std::snprintf(msg, sizeof msg, "%s: %s", name, what);
        return lfail(code, msg);
    };
    if (!(alpha > 0.0) || !(delta_star > 0.0) || !std::isfinite(alpha) || !std::isfinite(delta_star))
        return fail(YK_ERR_ARG, "alpha and delta_star must be > 0");
    if (n_panels < 1 || q < 2 || q > kMaxQ || n_trg < 0)
        return fail(YK_ERR_ARG, "need n_panels >= 1, 2 <= q <= 32, n_trg >= 0");
    if (n_panels * q > (1ll << 30) || n_trg > (1ll << 31) - 1)
        return fail(YK_ERR_UNSUPPORTED, "too many nodes or targets");
    if (!is_dev(xb) || !is_dev(yb) || (!vol && !is_dev(sigma)) ||
        (n_trg > 0 && (!is_dev(xt) || !is_dev(yt) || !is_dev(u) || (vol && !is_dev(fd)))))
        return fail(YK_ERR_ARG, "every array must be device memory");
    if (n_trg == 0) return YK_OK;
    if (vol) sigma = xb; /* the density series is not used; any node array serves */
    cudaStream_t st = (cudaStream_t)stream;
    const double sd = std::sqrt(delta_star), rl = sd * (12.0 + 2.0 * alpha * sd);

    /* host: Gauss-Legendre nodes; the boundary's extent comes from one device-to-host copy */
    /* host tables: the nodes t_k, then L[n][k] = (2n+1)/2 w_k P_n(t_k) (the projection onto the
     * Legendre series), and the recurrence ratios */
    std::vector<double> tq(q), wq(q), tab(q + q * q);
    yk_gauss_legendre(q, tq.data(), wq.data());
    for (int k = 0; k < q; ++k) {
        tab[k] = tq[k];
        double p0 = 1.0, p1 = tq[k];
        for (int n = 0; n < q; ++n) {
            const double pn = n == 0 ? 1.0 : (n == 1 ? tq[k] : 0.0);
            double v = pn;
            if (n >= 2) {
                const double p2 = ((2.0 * n - 1.0) * tq[k] * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
                v = p2;
            }
            tab[q + n * q + k] = 0.5 * (2.0 * n + 1.0) * wq[k] * v;
        }
    }
    {
        double la[kMaxQ], lb[kMaxQ];
        float laf[kMaxQ], lbf[kMaxQ];
        for (int n = 0; n < kMaxQ; ++n) {
            la[n] = (2.0 * n + 1.0) / (n + 1.0);
            lb[n] = (double)n / (n + 1.0);
            laf[n] = (float)la[n];
            lbf[n] = (float)lb[n];
        }
        cudaError_t ec = cudaMemcpyToSymbolAsync(c_la, la, sizeof la, 0, cudaMemcpyHostToDevice, st);
        if (ec == cudaSuccess)
            ec = cudaMemcpyToSymbolAsync(c_lb, lb, sizeof lb, 0, cudaMemcpyHostToDevice, st);
        if (ec == cudaSuccess)
            ec = cudaMemcpyToSymbolAsync(c_laf, laf, sizeof laf, 0, cudaMemcpyHostToDevice, st);
        if (ec == cudaSuccess)
            ec = cudaMemcpyToSymbolAsync(c_lbf, lbf, sizeof lbf, 0, cudaMemcpyHostToDevice, st);
        if (ec != cudaSuccess) return fail(YK_ERR_CUDA, "constant table copy failed");
    }
    const int64_t nb = n_panels * q;
    const int nblk = (int)std::min<int64_t>(148, (nb + 1023) / 1024);
    double *d_ext = nullptr;
    std::vector<double> part(5 * nblk);
    cudaError_t e = cudaMallocAsync(&d_ext, sizeof(double) * part.size(), st);
    if (e == cudaSuccess) {
        k_extent<<<nblk, 1024, 0, st>>>(n_panels, q, xb, yb, d_ext);
        e = cudaMemcpyAsync(part.data(), d_ext, sizeof(double) * part.size(),
                            cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(d_ext, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(YK_ERR_CUDA, "boundary extent failed");
    double ext[5] = {part[0], part[1], part[2], part[3], part[4]};
    for (int b = 1; b < nblk; ++b) {
        ext[0] = std::fmin(ext[0], part[5 * b]);
        ext[1] = std::fmax(ext[1], part[5 * b + 1]);
        ext[2] = std::fmin(ext[2], part[5 * b + 2]);
        ext[3] = std::fmax(ext[3], part[5 * b + 3]);
        ext[4] = std::fmax(ext[4], part[5 * b + 4]);
    }
    const double xmin = ext[0], xmax = ext[1], ymin = ext[2], ymax = ext[3], hmax = ext[4];
    if (!std::isfinite(xmin + xmax + ymin + ymax + hmax))
        return fail(YK_ERR_ARG, "non-finite boundary node");
    /* cells of edge >= r_loc + panel size, so every panel within r_loc of a target is listed in
     * the target's cell */
    LocalGrid G;
    G.h = rl + hmax;
    G.x0 = xmin - rl;
    G.y0 = ymin - rl;
    G.nx = (int)std::ceil((xmax + rl - G.x0) / G.h) + 1;
    G.ny = (int)std::ceil((ymax + rl - G.y0) / G.h) + 1;
    while ((int64_t)G.nx * G.ny > kMaxCells) {
        G.h *= 2.0;
        G.nx = (int)std::ceil((xmax + rl - G.x0) / G.h) + 1;
        G.ny = (int)std::ceil((ymax + rl - G.y0) / G.h) + 1;
    }
    const int ncell = G.nx * G.ny;

    /* scratch: Legendre series, cell lists */
    double *d_tq = nullptr, *d_c = nullptr;
    float *d_cf = nullptr;
    int *d_cnt = nullptr, *d_ptr = nullptr, *d_cur = nullptr, *d_list = nullptr;
    int *d_tcell = nullptr, *d_tcnt = nullptr, *d_tptr = nullptr, *d_order = nullptr;
    int *d_nout = nullptr;
    double *d_wide = nullptr, *d_wgram = nullptr;
    /* scratch is stream-ordered (no device-wide synchronisation on free) */
    auto cleanup = [&]() {
        for (void *b : {(void *)d_tq, (void *)d_c, (void *)d_cf, (void *)d_cnt, (void *)d_ptr,
                        (void *)d_cur, (void *)d_list, (void *)d_tcell, (void *)d_tcnt,
                        (void *)d_tptr, (void *)d_order, (void *)d_nout, (void *)d_wide,
                        (void *)d_wgram})
            if (b) cudaFreeAsync(b, st);
        cudaStreamSynchronize(st);
    };
    e = cudaMallocAsync(&d_tq, sizeof(double) * tab.size(), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_c, sizeof(double) * 3 * nb, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_cf, sizeof(float) * (4 * nb + 2 * n_panels), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_cnt, sizeof(int) * ncell, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_ptr, sizeof(int) * (ncell + 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_cur, sizeof(int) * ncell, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_nout, sizeof(int), st);
    if (e == cudaSuccess && J == 0)
        e = cudaMallocAsync(&d_wide, sizeof(double) * kWideStride * n_panels, st);
    if (e == cudaSuccess && J == 0)
        e = cudaMallocAsync(&d_wgram, sizeof(double) * kWideSys * n_panels, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_nout, 0, sizeof(int), st);
    if (e != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(YK_ERR_OOM, "scratch allocation failed");
    }
    e = cudaMemcpyAsync(d_tq, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st);
    double *cx = d_c, *cy = d_c + nb, *cs = d_c + 2 * nb;
    float *cxf = d_cf, *cyf = d_cf + nb, *xbf = d_cf + 2 * nb, *ybf = d_cf + 3 * nb;
    float *xmf = d_cf + 4 * nb, *ymf = d_cf + 4 * nb + n_panels;
    if (e == cudaSuccess) {
        k_panel_series<<<(int)((nb + 255) / 256), 256, 0, st>>>(
            n_panels, q, xb, yb, sigma, d_tq + q, cx, cy, cs, cxf, cyf, xbf, ybf, xmf, ymf);
        if (J == 0) /* window fits of panels shorter than 0.006 of the boundary's extent */
        {
            k_panel_wide<<<(int)((n_panels + 1) / 2), 64, 0, st>>>(
                n_panels, q, xb, yb, sigma, d_tq,
                0.006 * std::fmax(xmax - xmin, ymax - ymin), d_wide, d_wgram);
            k_panel_wide_solve<<<(int)((n_panels + 127) / 128), 128, 0, st>>>(n_panels, d_wgram,
                                                                              d_wide);
        }
        e = cudaMemsetAsync(d_cnt, 0, sizeof(int) * ncell, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cur, 0, sizeof(int) * ncell, st);
    const int pb = (int)((n_panels + 255) / 256);
    if (e == cudaSuccess) {
        k_cell_count<<<pb, 256, 0, st>>>(n_panels, q, xb, yb, rl, G, d_cnt);
        e = yk::launch_scan(d_cnt, d_ptr, ncell, d_cur, st);
    }
    int total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, d_ptr + ncell, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_list, sizeof(int) * (total > 0 ? total : 1), st);
    if (e == cudaSuccess) {
        k_cell_fill<<<pb, 256, 0, st>>>(n_panels, q, xb, yb, rl, G, d_ptr, d_cur, d_list);
        e = cudaGetLastError();
    }
    /* the targets in cells that list panels, grouped by cell */
    if (e == cudaSuccess) e = cudaMallocAsync(&d_tcell, sizeof(int) * n_trg, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_tcnt, sizeof(int) * ncell, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_tptr, sizeof(int) * (ncell + 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_order, sizeof(int) * n_trg, st);
    const int tb = (int)((n_trg + 255) / 256);
    if (e == cudaSuccess) {
        if (vol) {
            k_vp_interior<<<tb, 256, 0, st>>>(n_trg, fd, alpha, delta_star, u);
            e = cudaGetLastError();
        } else {
            e = cudaMemsetAsync(u, 0, sizeof(double) * n_trg, st);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_tcnt, 0, sizeof(int) * ncell, st);
    if (e == cudaSuccess) {
        k_target_cells<<<tb, 256, 0, st>>>(n_trg, xt, yt, G, d_ptr, d_tcell, d_tcnt);
        e = yk::launch_scan(d_tcnt, d_tptr, ncell, d_cur, st);
    }
    /* d_cur still holds the panel cursors: zero it for the target cursors */
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cur, 0, sizeof(int) * ncell, st);
    int n_near = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&n_near, d_tptr + ncell, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) {
        k_target_fill<<<tb, 256, 0, st>>>(n_trg, d_tcell, d_tptr, d_cur, d_order);
        e = cudaStreamSynchronize(st);
    }
    PanelSet P;
    P.npan = n_panels;
    P.q = q;
    P.xb = xb;
    P.yb = yb;
    P.cx = cx;
    P.cy = cy;
    P.cs = cs;
    P.sref = sigma;
    P.cxf = cxf;
    P.cyf = cyf;
    P.xbf = xbf;
    P.ybf = ybf;
    P.xmf = xmf;
    P.ymf = ymf;
    P.tq = d_tq;
    P.ptr = d_ptr;
    P.list = d_list;
    P.wide = d_wide;
    if (e == cudaSuccess && n_near > 0) {
        const int nb2 = (n_near + 127) / 128;
        if (vol)
            k_vp_local<<<nb2, 128, 0, st>>>(n_near, d_order, d_tcell, xt, yt, n_trg, fd, P, alpha,
                                            delta_star, rl, u, d_nout);
        else if (J == 0 && dl)
            k_dla_local<<<nb2, 128, 0, st>>>(n_near, d_order, d_tcell, xt, yt, P, alpha,
                                             delta_star, rl, u);
        else if (J == 0)
            k_slp_local<<<nb2, 128, 0, st>>>(n_near, d_order, d_tcell, xt, yt, P, alpha,
                                             delta_star, rl, u);
        e = cudaGetLastError();
    }
    /* dyadic levels: delta_star is delta here, so the set-up's near targets are those within the
     * level-1 radius */
    bool dy_oom = false;
    for (int j = 1; j <= J && e == cudaSuccess && n_near > 0; ++j) {
        const double dj = delta_star / std::pow(4.0, j), dj1 = 4.0 * dj;
        const double R = std::sqrt(dj1) * (12.0 + 2.0 * alpha * std::sqrt(dj1));
        const int npc = (int)std::ceil(R * R / (4.0 * dj) / kDyPiece) + 1;
        std::vector<double> tab;
        dyadic_table(alpha * alpha * dj, npc, dj, dl, tab);
        /* sub-panels no longer than 3 sqrt(delta_j) (chords at most 1.5 x shorter than arcs) */
        const int m = std::max(1, (int)std::ceil(1.5 * hmax / (3.0 * std::sqrt(dj))));
        const int64_t nn = n_panels * m * q;
        if (nn > (1ll << 31) - 1) {
            e = cudaErrorMemoryAllocation;
            dy_oom = true;
            break;
        }
        DyLevel L;
        L.inv4d = df32(1.0 / (kDyPiece * 4.0 * dj));
        L.R2 = (float)(R * R);
        {
            /* screen radius: R plus the FP32 rounding of the coordinates (< 2^-24 |x| each, three
             * roundings per difference) with room to spare */
            const double amax = std::max(std::max(std::fabs(xmin), std::fabs(xmax)),
                                         std::max(std::fabs(ymin), std::fabs(ymax))) + 2.0 * R;
            const double Rs = R * 1.0005 + 5e-7 * amax;
            L.R2f = (float)(Rs * Rs);
        }
        L.npc = npc;
        L.G.h = R;
        L.G.x0 = xmin - 2.0 * R;
        L.G.y0 = ymin - 2.0 * R;
        L.G.nx = (int)std::ceil((xmax + 2.0 * R - L.G.x0) / L.G.h) + 1;
        L.G.ny = (int)std::ceil((ymax + 2.0 * R - L.G.y0) / L.G.h) + 1;
        while ((int64_t)L.G.nx * L.G.ny > kMaxCells) {
            L.G.h *= 2.0;
            L.G.nx = (int)std::ceil((xmax + 2.0 * R - L.G.x0) / L.G.h) + 1;
            L.G.ny = (int)std::ceil((ymax + 2.0 * R - L.G.y0) / L.G.h) + 1;
        }
        const int nc = L.G.nx * L.G.ny;
        /* the table as double-float pairs */
        std::vector<float2> tab2(tab.size());
        for (size_t k = 0; k < tab.size(); ++k) {
            const float h = (float)tab[k];
            tab2[k] = make_float2(h, (float)(tab[k] - (double)h));
        }
        float2 *d_tab = nullptr;
        double *d_nodes = nullptr, *d_wq = nullptr;
        int *d_c = nullptr; /* cnt | ptr | cur */
        int2 *d_tcell = nullptr;
        float4 *d_txy = nullptr;
        e = cudaMallocAsync(&d_tab, sizeof(float2) * tab2.size(), st);
        if (e == cudaSuccess) e = cudaMallocAsync(&d_tcell, sizeof(int2) * (size_t)n_near, st);
        if (e == cudaSuccess) e = cudaMallocAsync(&d_txy, sizeof(float4) * (size_t)n_near, st);
        /* X Y Q (NX NY) per node in FP64, then the sorted Q (NX NY) as FP32 pairs */
        const int nu = dl ? 5 : 3, nsrt = dl ? 3 : 1;
        float *d_f = nullptr; /* the sorted X, Y: high words, low words */
        if (e == cudaSuccess) e = cudaMallocAsync(&d_nodes, sizeof(double) * (nu + nsrt) * nn, st);
        if (e == cudaSuccess) e = cudaMallocAsync(&d_f, sizeof(float) * 4 * nn, st);
        if (e == cudaSuccess) e = cudaMallocAsync(&d_wq, sizeof(double) * q, st);
        if (e == cudaSuccess) e = cudaMallocAsync(&d_c, sizeof(int) * (3 * (size_t)nc + 1), st);
        if (e != cudaSuccess) dy_oom = true;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_tab, tab2.data(), sizeof(float2) * tab2.size(),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_wq, wq.data(), sizeof(double) * q, cudaMemcpyHostToDevice, st);
        int *cnt = d_c, *cptr = d_c + nc, *ccur = d_c + 2 * nc + 1;
        double *X = d_nodes, *Y = d_nodes + nn, *Qn = d_nodes + 2 * nn;
        double *NX = dl ? d_nodes + 3 * nn : nullptr, *NY = dl ? d_nodes + 4 * nn : nullptr;
        float2 *Qs = reinterpret_cast<float2 *>(d_nodes + nu * nn);
        float2 *NXs = dl ? Qs + nn : nullptr, *NYs = dl ? Qs + 2 * nn : nullptr;
        const int gb = (int)((nn + 255) / 256);
        if (e == cudaSuccess) {
            k_dy_nodes<<<gb, 256, 0, st>>>(n_panels, q, m, P, d_wq, X, Y, Qn, NX, NY);
            e = cudaMemsetAsync(cnt, 0, sizeof(int) * nc, st);
        }
        if (e == cudaSuccess) {
            k_pt_count<<<gb, 256, 0, st>>>(nn, X, Y, L.G, cnt);
            e = yk::launch_scan(cnt, cptr, nc, ccur, st);
        }
        /* the scan used the cursors as scratch: zero them for the fill */
        if (e == cudaSuccess) e = cudaMemsetAsync(ccur, 0, sizeof(int) * nc, st);
        if (e == cudaSuccess) {
            k_pt_fill<<<gb, 256, 0, st>>>(nn, X, Y, Qn, NX, NY, L.G, cptr, ccur, d_f, d_f + nn,
                                          d_f + 2 * nn, d_f + 3 * nn, Qs, NXs, NYs);
            L.Xf = d_f;
            L.Xl = d_f + nn;
            L.Yf = d_f + 2 * nn;
            L.Yl = d_f + 3 * nn;
            L.tab = d_tab;
            L.ptr = cptr;
            L.Q = Qs;
            L.NX = NXs;
            L.NY = NYs;
            k_dy_targets<<<(n_near + 255) / 256, 256, 0, st>>>(n_near, d_order, xt, yt, L.G,
                                                                d_tcell, d_txy);
            k_dyadic_level<<<(int)(((int64_t)n_near * 32 + 255) / 256), 256, 0, st>>>(
                n_near, d_order, d_tcell, d_txy, L, u);
            e = cudaGetLastError();
        }
        for (void *b : {(void *)d_tcell, (void *)d_txy})
            if (b) cudaFreeAsync(b, st);
        for (void *b : {(void *)d_tab, (void *)d_nodes, (void *)d_wq, (void *)d_c, (void *)d_f})
            if (b) cudaFreeAsync(b, st);
    }
    int n_out = 0;
    if (e == cudaSuccess && vol)
        e = cudaMemcpyAsync(&n_out, d_nout, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return dy_oom ? fail(YK_ERR_OOM, "dyadic level scratch allocation failed")
                      : fail(YK_ERR_CUDA, "a CUDA call failed");
    }
    if (n_out > 0) {
        std::snprintf(msg, sizeof msg, "%s: %d targets within the locality radius lie outside the "
                      "domain (u = NaN there)", name, n_out);
        return lfail(YK_ERR_ARG, msg);
    }
    return YK_OK;
}

} /* namespace */

extern "C" YK_API yk_status yk_slp_local(double alpha, double delta_star, int64_t n_panels, int q,
                                         const double *xb, const double *yb, const double *sigma,
                                         int64_t n_trg, const double *xt, const double *yt,
                                         double *u, void *stream)
{
    if (!sigma) return lfail(YK_ERR_ARG, "yk_slp_local: sigma is NULL");
    return run_local("yk_slp_local", false, 0, false, alpha, delta_star, n_panels, q, xb, yb, sigma, n_trg, xt, yt,
                     nullptr, u, stream);
}

extern "C" YK_API yk_status yk_dlp_local(double alpha, double delta_star, int64_t n_panels, int q,
                                         const double *xb, const double *yb, const double *mu,
                                         int64_t n_trg, const double *xt, const double *yt,
                                         double *u, void *stream)
{
    if (!mu) return lfail(YK_ERR_ARG, "yk_dlp_local: mu is NULL");
    return run_local("yk_dlp_local", false, 0, true, alpha, delta_star, n_panels, q, xb, yb, mu,
                     n_trg, xt, yt, nullptr, u, stream);
}

extern "C" YK_API yk_status yk_vp_local(double alpha, double delta_star, int64_t n_panels, int q,
                                        const double *xb, const double *yb, int64_t n_trg,
                                        const double *xt, const double *yt, const double *fd,
                                        double *u, void *stream)
{
    if (n_trg > 0 && !fd) return lfail(YK_ERR_ARG, "yk_vp_local: fd is NULL");
    return run_local("yk_vp_local", true, 0, false, alpha, delta_star, n_panels, q, xb, yb, nullptr, n_trg,
                     xt, yt, fd, u, stream);
}

extern "C" YK_API yk_status yk_slp_dyadic(double alpha, double delta, int J, int64_t n_panels,
                                          int q, const double *xb, const double *yb,
                                          const double *sigma, int64_t n_trg, const double *xt,
                                          const double *yt, double *u, void *stream)
{
    if (!sigma) return lfail(YK_ERR_ARG, "yk_slp_dyadic: sigma is NULL");
    if (J < 1 || J > 10) return lfail(YK_ERR_ARG, "yk_slp_dyadic: need 1 <= J <= 10");
    return run_local("yk_slp_dyadic", false, J, false, alpha, delta, n_panels, q, xb, yb, sigma, n_trg,
                     xt, yt, nullptr, u, stream);
}

extern "C" YK_API yk_status yk_dlp_dyadic(double alpha, double delta, int J, int64_t n_panels,
                                          int q, const double *xb, const double *yb,
                                          const double *mu, int64_t n_trg, const double *xt,
                                          const double *yt, double *u, void *stream)
{
    if (!mu) return lfail(YK_ERR_ARG, "yk_dlp_dyadic: mu is NULL");
    if (J < 1 || J > 10) return lfail(YK_ERR_ARG, "yk_dlp_dyadic: need 1 <= J <= 10");
    return run_local("yk_dlp_dyadic", false, J, true, alpha, delta, n_panels, q, xb, yb, mu, n_trg,
                     xt, yt, nullptr, u, stream);
}
