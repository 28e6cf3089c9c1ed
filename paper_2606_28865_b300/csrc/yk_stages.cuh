/*
 * yk_stages.cuh — device bodies of the evaluation stages, one work item each (a spread tile, a
 * block of grid rows, a grid column, an interpolation tile).  Called by the per-stage kernels of
 * yk_kernels.cu (one CTA per item) and by the persistent batch kernel of yk_batch.cu (CTAs pull
 * items of many instances from a queue).  Every function is entered by all threads of the CTA
 * and uses `sm` (dynamic shared memory of at least stage_smem() bytes).
 */
#ifndef YK_STAGES_CUH
#define YK_STAGES_CUH

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "yk_internal.h"

namespace yk {

/* complex of double-floats as stored in memory (spectrum, twiddles) */
struct __align__(16) dfc {
    df32 x, y;
};

/* storage and conversions per arithmetic type R: FP64 path (double), FP32C path (float), and the
 * FP64 path's FFT in double-float (df32: arithmetic in FP32 pairs, grid stored in FP64) */
template <typename R> struct Tr;
template <> struct Tr<double> {
    using G = double;   /* grid value */
    using G2 = double2; /* two grid values (a packed complex) */
    using C2 = double2; /* stored complex */
    static __device__ __forceinline__ cpx<double> from_g2(double2 v) { return mk<double>(v.x, v.y); }
    static __device__ __forceinline__ double2 to_g2(cpx<double> z) { return make_double2(z.re, z.im); }
    static __device__ __forceinline__ cpx<double> from_c2(double2 v) { return mk<double>(v.x, v.y); }
    static __device__ __forceinline__ double2 to_c2(cpx<double> z) { return make_double2(z.re, z.im); }
    static __device__ __forceinline__ double2 zero_c2() { return make_double2(0.0, 0.0); }
};
template <> struct Tr<float> {
    using G = float;
    using G2 = float2;
    using C2 = float2;
    static __device__ __forceinline__ cpx<float> from_g2(float2 v) { return mk<float>(v.x, v.y); }
    static __device__ __forceinline__ float2 to_g2(cpx<float> z) { return make_float2(z.re, z.im); }
    static __device__ __forceinline__ cpx<float> from_c2(float2 v) { return mk<float>(v.x, v.y); }
    static __device__ __forceinline__ float2 to_c2(cpx<float> z) { return make_float2(z.re, z.im); }
    static __device__ __forceinline__ float2 zero_c2() { return make_float2(0.0f, 0.0f); }
};
template <> struct Tr<df32> {
    using G = df32; /* the FP64 path's grid holds FP32 pairs in its 8-byte cells */
    using G2 = dfc;
    using C2 = dfc;
    static __device__ __forceinline__ cpx<df32> from_g2(dfc v) { return mk<df32>(v.x, v.y); }
    static __device__ __forceinline__ dfc to_g2(cpx<df32> z)
    {
        dfc r;
        r.x = z.re;
        r.y = z.im;
        return r;
    }
    static __device__ __forceinline__ cpx<df32> from_c2(dfc v) { return mk<df32>(v.x, v.y); }
    static __device__ __forceinline__ dfc to_c2(cpx<df32> z)
    {
        dfc r;
        r.x = z.re;
        r.y = z.im;
        return r;
    }
    static __device__ __forceinline__ dfc zero_c2()
    {
        dfc r;
        r.x = df32(0.0f, 0.0f);
        r.y = df32(0.0f, 0.0f);
        return r;
    }
};

constexpr double kMagic = 6755399441055744.0; /* 1.5 * 2^52: fma(a, b, kMagic) rounds a*b to an integer */
constexpr int kSpreadBatch = 16;              /* sources a warp of the double-float owner-tile
                                                 spread takes at a time */

__device__ __forceinline__ double block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    v = red[0];
    __syncthreads();
    return v;
}

/* FP64 window values of the w taps of a point at grid coordinate t (first tap l0): by Horner on
 * the per-tap polynomials staged in shared memory (cw, (deg+1) x W), or by the formula */
template <int W>
__device__ __forceinline__ void windows64(double *f, int l0, double t, const double *cw, int deg,
                                          const Geom &g)
{
    if (cw) {
        const double x = 2.0 * (((double)l0 - t) + 0.5 * W) - 1.0;
#pragma unroll
        for (int a = 0; a < W; ++a) f[a] = cw[deg * W + a];
        for (int k = deg - 1; k >= 0; --k) {
#pragma unroll
            for (int a = 0; a < W; ++a) f[a] = fma(f[a], x, cw[k * W + a]);
        }
    } else {
#pragma unroll
        for (int a = 0; a < W; ++a) f[a] = es_window<double>((double)(l0 + a) - t, g.beta, g.c);
    }
}

/* double-float window values of the w taps at x = 2u - 1 (u = l0 - t + w/2), Horner on the
 * per-tap polynomials cw ((deg+1) x W double-float coefficients in shared memory) */
template <int W>
__device__ __forceinline__ df32 window_df(const df32 *cw, int deg, int a, df32 x)
{
    df32 p = cw[deg * W + a];
    for (int k = deg - 1; k >= 0; --k) p = p * x + cw[k * W + a];
    return p;
}

__device__ __forceinline__ df32 window_arg_df(int l0, double t, int W)
{
    return df32(2.0 * (((double)l0 - t) + 0.5 * W) - 1.0);
}

/* window coefficients, followed by the derivative's when the evaluation has dipoles */
__device__ __forceinline__ int window_coeffs(const Inst &d)
{
    return (d.wdeg + 1) * d.g.w + (d.dip ? d.wdeg * d.g.w : 0);
}

/* copy the first m double-float window coefficients into shared memory (the spread takes the
 * derivative's too, the interpolation the window's only) */
__device__ __forceinline__ df32 *stage_window_df(const Inst &d, df32 *dst, int m)
{
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float2 c = d.win_df[i];
        dst[i] = df32(c.x, c.y);
    }
    return dst;
}

/* copy the window polynomials into shared memory (NULL when the formula is used) */
__device__ __forceinline__ const double *stage_window(const Inst &d, double *dst, int m)
{
    if (!d.win) return nullptr;
    for (int i = threadIdx.x; i < m; i += blockDim.x) dst[i] = d.win[i];
    return dst;
}

/* FP32 Horner on per-tap polynomials (FP32C dipoles): x = 2u - 1 as for windows64 */
template <int W> __device__ __forceinline__ float window32(const float *cw, int deg, int a, float x)
{
    float p = cw[deg * W + a];
    for (int k = deg - 1; k >= 0; --k) p = fmaf(p, x, cw[k * W + a]);
    return p;
}

/* ----------------------------------------------------------------------------------------- */
/* spread (type 1, Section 5.2 eq. disrete_sigma_hat): one output tile per item                */

/* FP64: 64-bit fixed point.  Per-tile scale 2^k: every product |q| phi phi <= max|q| stays below
 * 2^51 (so one fma with 1.5 * 2^52 rounds it to an integer) and the sum of all of them below
 * 2^62; integer sums are exact, so the tile does not depend on the order of its entries. */
template <int W> __device__ void st_spread64(const Inst &d, int item, unsigned char *sm)
{
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(sm); /* T x T */
    __shared__ double red[32];
    __shared__ int s_k;
    const Geom &g = d.g;
    const int T = g.T, tile = d.order ? d.order[item] : item;
    const int tyi = tile / g.nt, txi = tile - tyi * g.nt;
    const int X0 = txi * T, Y0 = tyi * T;
    const double *__restrict__ wq = d.wq;
    const double *__restrict__ dens = d.dens;
    double *__restrict__ grid = static_cast<double *>(d.grid);
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) acc[i] = 0ull;
    const double *cw = stage_window(d, reinterpret_cast<double *>(acc + T * T), window_coeffs(d));
    const int beg = d.tile_ptr[tile], end = d.tile_ptr[tile + 1];
    double mq = 0.0;
    for (int e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const int j = d.ent_j[e];
        if (!d.dip || j < d.n_chg) {
            mq = fmax(mq, fabs(wq[j] * dens[j]));
        } else { /* a dipole's taps are at most (|s_x| + |s_y|) max|phi'| */
            const double2 wn = d.wnu[j - d.n_chg];
            mq = fmax(mq, fabs(d.mu[j - d.n_chg] * g.inv_h) * (fabs(wn.x) + fabs(wn.y)) * d.dmax);
        }
    }
    mq = block_max(mq, red);
    if (threadIdx.x == 0) {
        int e2 = 0;
        if (mq > 0.0) frexp(mq, &e2);
        const int cbits = 32 - __clz(end - beg);
        s_k = min(51, 62 - cbits) - e2;
    }
    __syncthreads();
    const int kexp = s_k;
    const long long magic_bits = __double_as_longlong(kMagic);
    if (mq > 0.0) {
        for (int e = beg + threadIdx.x; e < end; e += blockDim.x) {
            const double2 t = d.ent_t[e];
            const int j = d.ent_j[e];
            const int lx = first_tap<W>(t.x), ly = first_tap<W>(t.y);
            double fx[W], fy[W];
            windows64<W>(fx, lx, t.x, cw, d.wdeg, g);
            windows64<W>(fy, ly, t.y, cw, d.wdeg, g);
            int dx0 = (lx - X0) % g.n;
            if (dx0 < 0) dx0 += g.n;
            int dy0 = (ly - Y0) % g.n;
            if (dy0 < 0) dy0 += g.n;
            if (d.dip && j >= d.n_chg) {
                /* dipole: taps s_x phi'(X - t_x) phi(Y - t_y) + s_y phi(X - t_x) phi'(Y - t_y),
                 * s = -mu w nu / h (the gradient of the window in the source point) */
                const double2 wn = d.wnu[j - d.n_chg];
                const double m = ldexp(-d.mu[j - d.n_chg] * g.inv_h, kexp);
                const double sx = m * wn.x, sy = m * wn.y;
                double gx[W], gy[W];
                windows64<W>(gx, lx, t.x, cw + (d.wdeg + 1) * W, d.wdeg - 1, g);
                windows64<W>(gy, ly, t.y, cw + (d.wdeg + 1) * W, d.wdeg - 1, g);
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    int yy = dy0 + c;
                    if (yy >= g.n) yy -= g.n;
                    if (yy < T) {
                        const double ay = sx * fy[c], cy = sy * gy[c];
#pragma unroll
                        for (int a = 0; a < W; ++a) {
                            int xx = dx0 + a;
                            if (xx >= g.n) xx -= g.n;
                            if (xx < T) {
                                const double v = fma(cy, fx[a], ay * gx[a]);
                                const long long iv = __double_as_longlong(v + kMagic) - magic_bits;
                                atomicAdd(&acc[yy * T + xx], (unsigned long long)iv);
                            }
                        }
                    }
                }
                continue;
            }
            const double qs = ldexp(wq[j] * dens[j], kexp);
#pragma unroll
            for (int c = 0; c < W; ++c) {
                int yy = dy0 + c;
                if (yy >= g.n) yy -= g.n;
                if (yy < T) {
                    const double qy = qs * fy[c];
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        int xx = dx0 + a;
                        if (xx >= g.n) xx -= g.n;
                        if (xx < T) {
                            const long long iv =
                                __double_as_longlong(fma(qy, fx[a], kMagic)) - magic_bits;
                            atomicAdd(&acc[yy * T + xx], (unsigned long long)iv);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
        const int r = i / T, c = i - r * T;
        grid[(size_t)(Y0 + r) * g.n + X0 + c] =
            mq > 0.0 ? ldexp((double)(long long)acc[i], -kexp) : 0.0;
    }
    __syncthreads(); /* shared memory is reused by the next item */
}

/* Owner-tile spread (double-float and FP32C paths).  Every source was binned once, to the tile
 * of its first tap (lx, ly); its w x w window then lies in that tile's padded region of
 * P = T + w - 1 cells per axis, so a tile accumulates whole windows with no in-tile test and writes
 * a padded tile of P^2 partial sums.  A grid cell is covered by the padded regions of at most four
 * tiles (its own and the tiles one step down and to the left, since P < 2T); the row FFT adds them
 * in a fixed order when it loads the grid (fold_cell), so the result stays deterministic and no
 * global atomics are used.
 *
 * A CTA takes one tile.  Each of its first kOwnerCopies warps owns a private padded copy of the
 * tile in shared memory and walks every kOwnerCopies-th batch of the tile's sources one source at a
 * time, one lane per tap, so the cells a warp updates together are distinct.  The copy's pitch is
 * P rounded up to a value congruent to w mod 16: tap t = c w + a of a window then lands in 8-byte
 * bank slot (base + t) mod 16, so 16 consecutive taps (a half-warp of 64-bit accesses) hit 16
 * distinct slots.  The copies are summed in warp order when the padded tile is written. */
constexpr int kOwnerCopies = 4;

__host__ __device__ constexpr int owner_span(int T, int W) { return T + W - 1; }
__host__ __device__ constexpr int owner_pitch(int T, int W)
{
    return owner_span(T, W) + ((((W - owner_span(T, W)) % 16) + 16) % 16);
}
__host__ __device__ constexpr int owner_copy_cells(int T, int W)
{
    return owner_span(T, W) * owner_pitch(T, W);
}

/* the copies of the walk in a CTA of nthreads: the plan's warps per spread CTA (<= kOwnerCopies);
 * the batch kernel's larger CTAs leave their other warps idle during the walk */
__host__ __device__ inline int owner_copies(int nthreads, int spread_warps)
{
    return nthreads / 32 < spread_warps ? nthreads / 32 : spread_warps;
}

/* window values kept per source in the owner-tile spread's batch buffer: charges only, 2w values
 * stored by the coalesced commit (consecutive 16-byte chunks, no bank conflicts); with dipoles,
 * 4w values plus one (an odd stride: the per-source commit of 16 sources hits 16 distinct 8-byte
 * bank slots) */
__host__ __device__ constexpr int owner_batch_stride(int W, bool dip) { return dip ? 4 * W + 1 : 2 * W; }

template <int W, bool DIP>
__device__ void st_spread_owner_df(const Inst &d, int item, unsigned char *sm)
{
    constexpr int EB = kSpreadBatch;      /* the largest batch (register arrays are sized for it) */
    constexpr int NI = (W * W + 31) / 32; /* taps per lane per source */
    constexpr int SW = owner_batch_stride(W, DIP);
    const Geom &g = d.g;
    const int T = g.T, P = owner_span(T, W), PP = owner_pitch(T, W), TS = P * PP;
    const int NC = owner_copies(blockDim.x, d.spread_warps);
    const int eb = d.spread_batch;        /* sources per batch: 4, 8 or 16 */
    df32 *acc = reinterpret_cast<df32 *>(sm);                        /* [NC][TS] */
    df32 *wbuf = acc + NC * TS;                                      /* [NC][eb][SW] */
    df32 *qbuf = wbuf + NC * eb * SW;                                /* [NC][eb] */
    int *obuf = reinterpret_cast<int *>(qbuf + NC * eb);             /* [NC][eb] */
    const int tile = d.order ? d.order[item] : item;
    const int beg = d.tile_ptr[tile], end = d.tile_ptr[tile + 1];
    if (beg == end) return; /* nothing to write: the fold skips empty tiles */
    for (int i = threadIdx.x; i < NC * TS; i += blockDim.x) acc[i] = df32(0.0f, 0.0f);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < NC) {
        df32 *mine = acc + warp * TS;
        df32 *wb = wbuf + warp * eb * SW;
        df32 *qb = qbuf + warp * eb;
        int *ob = obuf + warp * eb;
        /* this lane's taps (c, a) = (t / W, t % W), t = i * 32 + lane; tv false past the last
         * tap (the last round's idle lanes load and store nothing) */
        int toff[NI], tc[NI], ta[NI];
        bool tv[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int t = i * 32 + lane;
            tv[i] = t < W * W;
            tc[i] = tv[i] ? t / W : 0;
            ta[i] = tv[i] ? t - (t / W) * W : 0;
            toff[i] = tc[i] * PP + ta[i];
        }
        const float2 *__restrict__ ws = d.win_src;
        const float2 *__restrict__ wd = d.win_dip;
        const int4 *__restrict__ ent = reinterpret_cast<const int4 *>(d.ent_t);
        const int stride = NC * eb;
        /* Software pipeline over batches of eb sources: the inputs of the next batch (window
         * values, weight and density) are loaded into registers before the current batch is
         * walked and stored to shared memory after it, so the walk hides their latency; the entry
         * records (tap offset, source index) are loaded one batch earlier still, since the weight
         * and density loads depend on the source index.
         * Charges only: the batch's window records are one contiguous block (entry order), read
         * as 16-byte chunks, chunk g = r * 32 + lane of the block in round r; lane s < eb holds
         * source s's record, weight and density.  With dipoles: two lanes per source (half 0 the
         * y-parts, half 1 the x-parts), since a dipole's record lies elsewhere. */
        constexpr int NCH = DIP ? 1 : (EB * W + 31) / 32;  /* chunks per lane (charges only) */
        constexpr int NV = DIP ? W : 1;                     /* float2 per lane (with dipoles) */
        float4 ch[NCH];
        float2 v1[NV], v2[NV];
        double pa = 0.0, pb = 0.0;
        double2 pw = make_double2(0.0, 0.0);
        const int slot = DIP ? (lane & (EB - 1)) : lane, half = DIP ? lane / EB : 0;
        auto record = [&](int e) {
            return (slot < eb && e < end) ? ent[e] : make_int4(0, -1, 0, 0);
        };
        auto fetch = [&](int bb, int4 r) {
            if (!DIP) {
                const float4 *src = reinterpret_cast<const float4 *>(ws + (size_t)bb * 2 * W);
                const int nch = min(eb, end - bb) * W;
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const int gi = k * 32 + lane;
                    if (gi < nch) ch[k] = src[gi];
                }
                if (r.y >= 0) {
                    pa = d.wq[r.y];
                    pb = d.dens[r.y];
                }
                return;
            }
            if (r.y < 0) return;
            const int j = r.y;
            if (j < d.n_chg) {
                /* half 0: phi_y (times q = w sigma at commit); half 1: phi_x */
                const float2 *src = ws + (size_t)(bb + slot) * 2 * W + half * W;
#pragma unroll
                for (int a = 0; a < NV; ++a) v1[a] = src[a];
                if (half == 0) {
                    pa = d.wq[j];
                    pb = d.dens[j];
                }
            } else {
                /* dipole: half 0 phi_y, phi'_y (times s_x, s_y at commit); half 1 phi'_x, phi_x */
                const int jd = j - d.n_chg;
                const float2 *src = wd + (size_t)jd * 4 * W;
                const float2 *s1 = src + (half ? 3 * W : 0), *s2 = src + (half ? W : 2 * W);
#pragma unroll
                for (int a = 0; a < NV; ++a) {
                    v1[a] = s1[a];
                    v2[a] = s2[a];
                }
                if (half == 0) {
                    pa = d.mu[jd];
                    pw = d.wnu[jd];
                }
            }
        };
        auto commit = [&](int bb, int4 r) {
            if (!DIP) {
                if (r.y >= 0) {
                    qb[slot] = df32(pa * pb);
                    ob[slot] = r.x;
                }
                __syncwarp();
                const int nch = min(eb, end - bb) * W;
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const int gi = k * 32 + lane;
                    if (gi < nch) {
                        /* values 2p, 2p + 1 of source s; the first W are phi_y, scaled by q */
                        const int s = gi / W, p2 = 2 * (gi - s * W);
                        const df32 q = qb[s];
                        df32 x0(ch[k].x, ch[k].y), x1(ch[k].z, ch[k].w);
                        if (p2 < W) x0 = q * x0;
                        if (p2 + 1 < W) x1 = q * x1;
                        wb[s * SW + p2] = x0;
                        wb[s * SW + p2 + 1] = x1;
                    }
                }
                return;
            }
            if (r.y < 0) return;
            df32 *wl = wb + slot * SW;
            const bool dipole = r.y >= d.n_chg;
            if (!dipole) {
                const df32 f = half ? df32(1.0f, 0.0f) : df32(pa * pb);
#pragma unroll
                for (int a = 0; a < NV; ++a) wl[half * W + a] = f * df32(v1[a].x, v1[a].y);
            } else {
                /* taps s_x phi'(X - t_x) phi(Y - t_y) + s_y phi(X - t_x) phi'(Y - t_y),
                 * s = -mu w nu / h (the gradient of the window in the source point) */
                const double m = -pa * g.inv_h;
                const df32 f1 = half ? df32(1.0f, 0.0f) : df32(m * pw.x);
                const df32 f2 = half ? df32(1.0f, 0.0f) : df32(m * pw.y);
#pragma unroll
                for (int a = 0; a < NV; ++a) {
                    wl[half * W + a] = f1 * df32(v1[a].x, v1[a].y);
                    wl[(2 + half) * W + a] = f2 * df32(v2[a].x, v2[a].y);
                }
            }
            if (half == 0) ob[slot] = r.x | (dipole ? 1 << 30 : 0);
        };
        int b0 = beg + warp * eb;
        int4 rc = record(b0 + slot);
        int4 rn = record(b0 + stride + slot);
        fetch(b0, rc);
        for (; b0 < end; b0 += stride) {
            commit(b0, rc);
            __syncwarp();
            rc = rn;
            if (b0 + stride < end) fetch(b0 + stride, rc);
            rn = record(b0 + 2 * stride + slot);
            const int cnt = min(eb, end - b0);
            for (int k = 0; k < cnt; ++k) {
                const int v = ob[k];
                const int base = v & 0x3fffffff;
                const df32 *wk = wb + k * SW;
                df32 cur[NI];
#pragma unroll
                for (int i = 0; i < NI; ++i)
                    if (tv[i]) cur[i] = mine[base + toff[i]];
                if (!DIP || !(v >> 30)) {
#pragma unroll
                    for (int i = 0; i < NI; ++i)
                        cur[i] = df_mul_add_lazy(cur[i], wk[tc[i]], wk[W + ta[i]]);
                } else { /* warp-uniform: one source at a time */
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        cur[i] = df_mul_add_lazy(cur[i], wk[tc[i]], wk[W + ta[i]]);
                        cur[i] = df_mul_add_lazy(cur[i], wk[2 * W + tc[i]], wk[3 * W + ta[i]]);
                    }
                }
#pragma unroll
                for (int i = 0; i < NI; ++i)
                    if (tv[i]) mine[base + toff[i]] = cur[i];
                __syncwarp(); /* the next source may touch the same cells through other lanes */
            }
            __syncwarp(); /* the window buffers are refilled by the next batch */
        }
    }
    __syncthreads();
    /* padded tile = sum of the copies in warp order, normalised (the cells were accumulated
     * unnormalised by df_mul_add_lazy) */
    df32 *__restrict__ out = static_cast<df32 *>(d.part) + (size_t)tile * P * P;
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
        const int r = i / P, c = i - r * P;
        const int ci = r * PP + c;
        df32 sum = acc[ci];
        for (int w = 1; w < NC; ++w) sum = sum + acc[w * TS + ci];
        out[i] = df_fast_two_sum(sum.hi, sum.lo);
    }
    __syncthreads(); /* shared memory is reused by the next item */
}

/* FP32C owner-tile spread: FP32 window values (computed here from the source's FP32 offsets) and
 * products, each cell a compensated pair (hi, lo) updated by two-sum; one lane per source
 * evaluates its windows, then the warp walks the batch one source at a time with one lane per
 * tap as above.  The copies are summed in warp order into a normalised pair per cell. */
template <int W, bool DIP>
__device__ void st_spread_owner32(const Inst &d, int item, unsigned char *sm)
{
    constexpr int NI = (W * W + 31) / 32;
    constexpr int SW = (DIP ? 4 * W : 2 * W) + 1; /* odd stride: the lanes' stores hit distinct banks */
    const Geom &g = d.g;
    const int T = g.T, P = owner_span(T, W), PP = owner_pitch(T, W), TS = P * PP;
    const int NC = owner_copies(blockDim.x, d.spread_warps);
    const int EB = d.spread_batch;  /* sources per batch (one lane each): 8, 16 or 32 */
    float2 *acc = reinterpret_cast<float2 *>(sm);                        /* [NC][TS] */
    float *wbuf = reinterpret_cast<float *>(acc + NC * TS);              /* [NC][EB][SW] */
    int *obuf = reinterpret_cast<int *>(wbuf + NC * EB * SW);            /* [NC][EB] */
    float *cw32 = reinterpret_cast<float *>(obuf + NC * EB);             /* dipole polynomials */
    const int tile = d.order ? d.order[item] : item;
    const int beg = d.tile_ptr[tile], end = d.tile_ptr[tile + 1];
    if (beg == end) return; /* nothing to write: the fold skips empty tiles */
    if (DIP)
        for (int i = threadIdx.x; i < window_coeffs(d); i += blockDim.x) cw32[i] = d.win32[i];
    for (int i = threadIdx.x; i < NC * TS; i += blockDim.x) acc[i] = make_float2(0.0f, 0.0f);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < NC) {
        float2 *mine = acc + warp * TS;
        float *wb = wbuf + warp * EB * SW;
        int *ob = obuf + warp * EB;
        int toff[NI], tc[NI], ta[NI];
        bool tv[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int t = i * 32 + lane;
            tv[i] = t < W * W;
            tc[i] = tv[i] ? t / W : 0;
            ta[i] = tv[i] ? t - (t / W) * W : 0;
            toff[i] = tc[i] * PP + ta[i];
        }
        const int4 *__restrict__ ent = reinterpret_cast<const int4 *>(d.ent_t);
        const float beta = (float)g.beta, cwin = (float)g.c;
        const int D = d.wdeg;
        for (int b0 = beg + warp * EB; b0 < end; b0 += NC * EB) {
            const int e = b0 + lane;
            if (lane < EB && e < end) {
                const int4 r = ent[e];
                const int j = r.y;
                const float sx = __int_as_float(r.z), sy = __int_as_float(r.w);
                float *wl = wb + lane * SW;
                int flag = 0;
                if (!DIP || j < d.n_chg) {
                    const float q = (float)(d.wq[j] * d.dens[j]);
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        wl[a] = q * es_window32(sy + (float)a, beta, cwin);
                        wl[W + a] = es_window32(sx + (float)a, beta, cwin);
                    }
                } else {
                    /* dipole: s = -mu w nu / h; window and derivative from the FP32 polynomials */
                    const double2 wn = d.wnu[j - d.n_chg];
                    const double m = -d.mu[j - d.n_chg] * g.inv_h;
                    const float gx = (float)(m * wn.x), gy = (float)(m * wn.y);
                    const float xx = 2.0f * sx + (float)(W - 1), xy = 2.0f * sy + (float)(W - 1);
                    const float *cwd = cw32 + (D + 1) * W;
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        wl[a] = gx * window32<W>(cw32, D, a, xy);
                        wl[W + a] = window32<W>(cwd, D - 1, a, xx);
                        if (DIP) {
                            wl[2 * W + a] = gy * window32<W>(cwd, D - 1, a, xy);
                            wl[3 * W + a] = window32<W>(cw32, D, a, xx);
                        }
                    }
                    flag = 1 << 30;
                }
                ob[lane] = r.x | flag;
            }
            __syncwarp();
            const int cnt = min(EB, end - b0);
            for (int k = 0; k < cnt; ++k) {
                const int v = ob[k];
                const int base = v & 0x3fffffff;
                const bool dipk = DIP && (v >> 30); /* warp-uniform: one source at a time */
                const float *wk = wb + k * SW;
                float2 cell[NI];
#pragma unroll
                for (int i = 0; i < NI; ++i)
                    if (tv[i]) cell[i] = mine[base + toff[i]];
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                    float val = wk[tc[i]] * wk[W + ta[i]];
                    if (dipk) val = fmaf(wk[2 * W + tc[i]], wk[3 * W + ta[i]], val);
                    const float s2 = __fadd_rn(cell[i].x, val);
                    const float bp = __fsub_rn(s2, cell[i].x);
                    const float err =
                        __fadd_rn(__fsub_rn(cell[i].x, __fsub_rn(s2, bp)), __fsub_rn(val, bp));
                    cell[i] = make_float2(s2, __fadd_rn(cell[i].y, err));
                }
#pragma unroll
                for (int i = 0; i < NI; ++i)
                    if (tv[i]) mine[base + toff[i]] = cell[i];
                __syncwarp(); /* the next source may touch the same cells through other lanes */
            }
            __syncwarp(); /* the window buffers are refilled by the next batch */
        }
    }
    __syncthreads();
    /* padded tile = the copies' pairs summed in warp order (two-sum of the high words, low words
     * added), written as a normalised pair */
    float2 *__restrict__ out = static_cast<float2 *>(d.part) + (size_t)tile * P * P;
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
        const int r = i / P, c = i - r * P;
        const int ci = r * PP + c;
        float hi = acc[ci].x, lo = acc[ci].y;
        for (int w = 1; w < NC; ++w) {
            const float2 q = acc[w * TS + ci];
            const df32 t = df_two_sum(hi, q.x);
            hi = t.hi;
            lo = __fadd_rn(lo, __fadd_rn(t.lo, q.y));
        }
        const df32 n2 = df_two_sum(hi, lo);
        out[i] = make_float2(n2.hi, n2.lo);
    }
    __syncthreads(); /* shared memory is reused by the next item */
}

/* one grid cell (x, y) of the owner-tile spread's output: the padded partials of the tiles whose
 * padded region covers it, added in a fixed order (far neighbours first); empty tiles were not
 * written and are skipped.  ty, ly = y / T, y % T of the cell's row. */
template <typename P2, typename ADD>
__device__ __forceinline__ void fold_terms(const Inst &d, int ty, int ly, int x, float invT,
                                           const P2 *__restrict__ part, ADD add)
{
    const Geom &g = d.g;
    const int T = g.T, nt = g.nt, P = owner_span(T, g.w), PPc = P * P;
    const int tx = min(nt - 1, (int)(((float)x + 0.5f) * invT)), lx = x - tx * T;
    const int *__restrict__ tp = d.tile_ptr;
    const int tyb = ty == 0 ? nt - 1 : ty - 1, txb = tx == 0 ? nt - 1 : tx - 1;
    const bool hy = ly < g.w - 1, hx = lx < g.w - 1; /* also in the padded region below / left */
    if (hy && hx) {
        const int t = tyb * nt + txb;
        if (tp[t + 1] > tp[t]) add(part[(size_t)t * PPc + (ly + T) * P + lx + T]);
    }
    if (hy) {
        const int t = tyb * nt + tx;
        if (tp[t + 1] > tp[t]) add(part[(size_t)t * PPc + (ly + T) * P + lx]);
    }
    if (hx) {
        const int t = ty * nt + txb;
        if (tp[t + 1] > tp[t]) add(part[(size_t)t * PPc + ly * P + lx + T]);
    }
    const int t = ty * nt + tx;
    if (tp[t + 1] > tp[t]) add(part[(size_t)t * PPc + ly * P + lx]);
}

__device__ __forceinline__ df32 fold_cell_df(const Inst &d, int ty, int ly, int x, float invT)
{
    df32 s(0.0f, 0.0f);
    fold_terms<df32>(d, ty, ly, x, invT, static_cast<const df32 *>(d.part),
                     [&](df32 v) { s = s + v; });
    return s;
}

/* ----------------------------------------------------------------------------------------- */
/* FFT passes (mixed-radix DIF in shared memory, see yk_core.h)                               */

/* floor(x / d) with the stage's multiplier (d = 1 when m == 0) */
__device__ __forceinline__ int fdiv(int x, unsigned m) { return m ? (int)__umulhi((unsigned)x, m) : x; }

/* the arithmetic of the butterflies: double-float stages compute in the lazily normalised form
 * (df32l) and normalise once per stored value; FP32 and FP64 stages compute in their own type */
template <typename R> struct FftArith {
    using C = R;
    static __device__ __forceinline__ C in(R v) { return v; }
    static __device__ __forceinline__ R out(C v) { return v; }
};
template <> struct FftArith<df32> {
    using C = df32l;
    static __device__ __forceinline__ C in(df32 v) { return df32l(v); }
    static __device__ __forceinline__ df32 out(df32l v) { return df_norm(v); }
};

/* one DIF stage with a compile-time radix: every butterfly of nrows rows (row stride rowlen) */
template <int RADIX, bool INV, typename R, typename TW>
__device__ __forceinline__ void fft_stage(cpx<R> *x, const FftStages &st, int s, const TW *tw,
                                          int nrows, int rowlen)
{
    using A = FftArith<R>;
    using C = typename A::C;
    const int B = st.B[s], span = B / RADIX, nb = st.L / RADIX, step = st.tw_step[s];
    const unsigned msp = st.span_m[s], mnb = st.nb_m[s];
    auto ld = [](cpx<R> z) { return mk<C>(A::in(z.re), A::in(z.im)); };
    auto sto = [](cpx<C> z) { return mk<R>(A::out(z.re), A::out(z.im)); };
    for (int i = threadIdx.x; i < nrows * nb; i += blockDim.x) {
        const int row = fdiv(i, mnb), t = i - row * nb;
        const int b = fdiv(t, msp), k = t - b * span;
        cpx<R> *xr = x + (size_t)row * rowlen + b * B + k;
        cpx<C> v[RADIX];
        if (!INV) {
#pragma unroll
            for (int q = 0; q < RADIX; ++q) v[q] = ld(xr[q * span]);
            if (RADIX == 2) dft2<-1>(v);
            else if (RADIX == 3) dft3<-1>(v);
            else if (RADIX == 4) dft4<-1>(v);
            else dft5<-1>(v);
            xr[0] = sto(v[0]);
#pragma unroll
            for (int p = 1; p < RADIX; ++p) {
                const TW w = tw[p * k * step];
                xr[p * span] = sto(mul(v[p], mk<C>((C)w.x, (C)w.y)));
            }
        } else {
            v[0] = ld(xr[0]);
#pragma unroll
            for (int p = 1; p < RADIX; ++p) {
                const TW w = tw[p * k * step];
                v[p] = mulc(ld(xr[p * span]), mk<C>((C)w.x, (C)w.y));
            }
            if (RADIX == 2) dft2<+1>(v);
            else if (RADIX == 3) dft3<+1>(v);
            else if (RADIX == 4) dft4<+1>(v);
            else dft5<+1>(v);
#pragma unroll
            for (int q = 0; q < RADIX; ++q) xr[q * span] = sto(v[q]);
        }
    }
    __syncthreads();
}

template <bool INV, typename R, typename TW>
__device__ __forceinline__ void fft_stage_any(cpx<R> *x, const FftStages &st, int s, const TW *tw,
                                              int nrows, int rowlen)
{
    switch (st.r[s]) {
    case 2: fft_stage<2, INV, R>(x, st, s, tw, nrows, rowlen); break;
    case 3: fft_stage<3, INV, R>(x, st, s, tw, nrows, rowlen); break;
    case 4: fft_stage<4, INV, R>(x, st, s, tw, nrows, rowlen); break;
    default: fft_stage<5, INV, R>(x, st, s, tw, nrows, rowlen); break;
    }
}

template <typename R, typename TW>
__device__ __forceinline__ void fft_fwd(cpx<R> *x, const FftStages &st, const TW *tw, int nrows,
                                        int rowlen)
{
    for (int s = 0; s < st.n; ++s) fft_stage_any<false, R>(x, st, s, tw, nrows, rowlen);
}

template <typename R, typename TW>
__device__ __forceinline__ void fft_inv(cpx<R> *x, const FftStages &st, const TW *tw, int nrows,
                                        int rowlen)
{
    for (int s = st.n - 1; s >= 0; --s) fft_stage_any<true, R>(x, st, s, tw, nrows, rowlen);
}

/* rows y0 .. y0 + nr - 1 of the grid from the owner-tile spread's padded partials, as packed
 * complex values x[r L + l] = grid[y][2l] + i grid[y][2l + 1] */
template <typename R> __device__ void load_folded_rows(const Inst &d, cpx<R> *x, int y0, int nr);

template <>
__device__ __forceinline__ void load_folded_rows<df32>(const Inst &d, cpx<df32> *x, int y0, int nr)
{
    const int L = d.n >> 1, T = d.g.T;
    const float invT = 1.0f / (float)T;
    for (int i = threadIdx.x; i < nr * L; i += blockDim.x) {
        const int r = i / L, l = i - r * L, y = y0 + r;
        const int ty = y / T, ly = y - ty * T;
        x[i] = mk<df32>(fold_cell_df(d, ty, ly, 2 * l, invT), fold_cell_df(d, ty, ly, 2 * l + 1, invT));
    }
}

/* FP32C: the partials are compensated pairs; a cell's (up to four) pairs are summed by two-sum
 * of the high words with the low words added, then rounded to one FP32 value */
__device__ __forceinline__ float fold_cell32(const Inst &d, int ty, int ly, int x, float invT)
{
    float hi = 0.0f, lo = 0.0f;
    fold_terms<float2>(d, ty, ly, x, invT, static_cast<const float2 *>(d.part), [&](float2 v) {
        const df32 t = df_two_sum(hi, v.x);
        hi = t.hi;
        lo = __fadd_rn(lo, __fadd_rn(t.lo, v.y));
    });
    return __fadd_rn(hi, lo);
}

template <>
__device__ __forceinline__ void load_folded_rows<float>(const Inst &d, cpx<float> *x, int y0, int nr)
{
    const int L = d.n >> 1, T = d.g.T;
    const float invT = 1.0f / (float)T;
    for (int i = threadIdx.x; i < nr * L; i += blockDim.x) {
        const int r = i / L, l = i - r * L, y = y0 + r;
        const int ty = y / T, ly = y - ty * T;
        x[i] = mk<float>(fold_cell32(d, ty, ly, 2 * l, invT), fold_cell32(d, ty, ly, 2 * l + 1, invT));
    }
}
template <> __device__ __forceinline__ void load_folded_rows<double>(const Inst &, cpx<double> *, int, int) {}

/* rows [item*rows, ...): real-to-complex FFT, keep m_x <= M, store transposed spec[m_x*n + y] */
template <typename R> __device__ void st_row_fwd(const Inst &d, int item, unsigned char *sm)
{
    using T = Tr<R>;
    using C2 = typename T::C2;
    using G2 = typename T::G2;
    cpx<R> *x = reinterpret_cast<cpx<R> *>(sm);
    const int n = d.n, M = d.M, L = n >> 1;
    const typename T::G *__restrict__ grid = static_cast<const typename T::G *>(d.grid);
    C2 *__restrict__ spec = static_cast<C2 *>(d.spec);
    const C2 *__restrict__ tw = static_cast<const C2 *>(d.tw);
    const int y0 = item * d.rows;
    const int nr = min(d.rows, n - y0);
    if (d.part) {
        /* owner-tile spread: fold the padded tile partials into the rows as they are loaded */
        load_folded_rows<R>(d, x, y0, nr);
    } else {
        for (int i = threadIdx.x; i < nr * L; i += blockDim.x) {
            const int r = i / L, l = i - r * L;
            x[i] = T::from_g2(reinterpret_cast<const G2 *>(grid + (size_t)(y0 + r) * n)[l]);
        }
    }
    __syncthreads();
    fft_fwd<R>(x, d.sth, tw, nr, L);
    for (int i = threadIdx.x; i < nr * (M + 1); i += blockDim.x) {
        const int m = i / nr, r = i - m * nr;
        const cpx<R> Zm = x[r * L + d.perm_h[m]];
        const cpx<R> Zc = x[r * L + d.perm_h[m == 0 ? 0 : L - m]];
        spec[(size_t)m * n + y0 + r] = T::to_c2(r2c_post<R>(Zm, Zc, T::from_c2(tw[m])));
    }
    __syncthreads();
}

/* column m_x = item: FFT along y, multiply by the symbol (eq. sh_fourier), zero |m_y| > M,
 * inverse FFT along y, in place */
template <typename R> __device__ void st_columns(const Inst &d, int item, unsigned char *sm)
{
    using T = Tr<R>;
    using C2 = typename T::C2;
    cpx<R> *x = reinterpret_cast<cpx<R> *>(sm);
    const int n = d.n, M = d.M, kx = item;
    const C2 *__restrict__ tw = static_cast<const C2 *>(d.tw);
    C2 *col = static_cast<C2 *>(d.spec) + (size_t)kx * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = T::from_c2(col[i]);
    __syncthreads();
    fft_fwd<R>(x, d.stf, tw, 1, n);
    const R *mrow = static_cast<const R *>(d.mult) + (size_t)kx * (2 * M + 1);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int m = d.iperm_f[i];
        const int my = m <= (n >> 1) ? m : m - n;
        if (my >= -M && my <= M) x[i] = scale(x[i], mrow[my + M]);
        else x[i] = T::from_c2(T::zero_c2());
    }
    __syncthreads();
    fft_inv<R>(x, d.stf, tw, 1, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = T::to_c2(x[i]);
    __syncthreads();
}

/* rows [item*rows, ...): gather m_x <= M, complex-to-real inverse FFT, write the real rows */
template <typename R> __device__ void st_row_inv(const Inst &d, int item, unsigned char *sm)
{
    using T = Tr<R>;
    using C2 = typename T::C2;
    using G2 = typename T::G2;
    cpx<R> *x = reinterpret_cast<cpx<R> *>(sm);
    const int n = d.n, M = d.M, L = n >> 1;
    const C2 *__restrict__ spec = static_cast<const C2 *>(d.spec);
    const C2 *__restrict__ tw = static_cast<const C2 *>(d.tw);
    typename T::G *__restrict__ grid = static_cast<typename T::G *>(d.grid);
    const int y0 = item * d.rows;
    const int nr = min(d.rows, n - y0);
    for (int i = threadIdx.x; i < nr * L; i += blockDim.x) {
        const int m = i / nr, r = i - m * nr;
        const int mc = L - m; /* in (0, L]; X[L] is zero because M < L */
        const C2 a = m <= M ? spec[(size_t)m * n + y0 + r] : T::zero_c2();
        const C2 b = mc <= M ? spec[(size_t)mc * n + y0 + r] : T::zero_c2();
        x[r * L + d.perm_h[m]] = c2r_pre<R>(T::from_c2(a), T::from_c2(b), T::from_c2(tw[m]));
    }
    __syncthreads();
    fft_inv<R>(x, d.sth, tw, nr, L);
    for (int i = threadIdx.x; i < nr * L; i += blockDim.x) {
        const int r = i / L, l = i - r * L;
        reinterpret_cast<G2 *>(grid + (size_t)(y0 + r) * n)[l] = T::to_g2(x[i]);
    }
    __syncthreads();
}

/* ----------------------------------------------------------------------------------------- */
/* interpolation (type 2): one target tile per item                                           */

template <typename R>
__device__ __forceinline__ void stage_halo(R *sg, const R *__restrict__ grid, const Geom &g,
                                           int X0, int Y0, int P)
{
    /* rows by warp, columns by lane (coalesced row reads, no division).  The halo reaches at most
     * W past the tile and n >= 2T >= 2W, so X0 + c and Y0 + r lie in (-n, 2n): one conditional
     * add or subtract wraps them onto the periodic grid.  Needs blockDim.x % 32 == 0. */
    if (P > g.n) { /* a halo wider than the grid: plain modulo (not reached with n >= 2T) */
        for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
            const int r = i / P, c = i - r * P;
            int gy = (Y0 + r) % g.n, gx = (X0 + c) % g.n;
            gy += gy < 0 ? g.n : 0;
            gx += gx < 0 ? g.n : 0;
            sg[i] = grid[(size_t)gy * g.n + gx];
        }
        return;
    }
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < P; r += nw) {
        int gy = Y0 + r;
        gy += gy < 0 ? g.n : (gy >= g.n ? -g.n : 0);
        const R *__restrict__ row = grid + (size_t)gy * g.n;
        for (int c = lane; c < P; c += 32) {
            int gx = X0 + c;
            gx += gx < 0 ? g.n : (gx >= g.n ? -g.n : 0);
            sg[r * P + c] = row[gx];
        }
    }
}

template <int W> __device__ void st_interp64(const Inst &d, int item, unsigned char *sm)
{
    double *sg = reinterpret_cast<double *>(sm);
    const Geom &g = d.g;
    const int T = g.Ti, P = T + W, lo = W / 2;
    const int tyi = item / g.nti, txi = item - tyi * g.nti;
    const int beg = d.trg_ptr[item], end = d.trg_ptr[item + 1];
    if (beg == end) return; /* uniform across the CTA */
    const int X0 = txi * T - lo, Y0 = tyi * T - lo;
    stage_halo<double>(sg, static_cast<const double *>(d.grid), g, X0, Y0, P);
    const double *cw = stage_window(d, sg + P * P, (d.wdeg + 1) * W);
    __syncthreads();
    for (int e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const double2 t = d.trg_t[e];
        const int lx = first_tap<W>(t.x), ly = first_tap<W>(t.y);
        double fx[W], fy[W];
        windows64<W>(fx, lx, t.x, cw, d.wdeg, g);
        windows64<W>(fy, ly, t.y, cw, d.wdeg, g);
        const double *base = sg + (ly - Y0) * P + (lx - X0);
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < W; ++c) {
            double row = 0.0;
#pragma unroll
            for (int a = 0; a < W; ++a) row = fma(fx[a], base[c * P + a], row);
            acc = fma(fy[c], row, acc);
        }
        d.u[d.trg_idx[e]] = acc;
    }
    __syncthreads();
}

/* the FP32 halo four times, with a row pitch PP that is a multiple of 4: copy k holds cell
 * (X0 + c + k, Y0 + r) at r PP + c, so that any four neighbouring cells of a row are one aligned
 * 16-byte load from copy (column mod 4).  Rows by warp, columns by lane, as stage_halo. */
__device__ __forceinline__ void stage_halo_quad32(float *s, const float *__restrict__ grid,
                                                  const Geom &g, int X0, int Y0, int P, int PP)
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5, CP = P * PP;
    for (int r = threadIdx.x >> 5; r < P; r += nw) {
        int gy = Y0 + r;
        if (P > g.n) { /* a halo wider than the grid: plain modulo (not reached with n >= 2T) */
            gy %= g.n;
            gy += gy < 0 ? g.n : 0;
        } else {
            gy += gy < 0 ? g.n : (gy >= g.n ? -g.n : 0);
        }
        const float *__restrict__ row = grid + (size_t)gy * g.n;
        for (int c = lane; c < P; c += 32) {
            int gx = X0 + c;
            if (P > g.n) {
                gx %= g.n;
                gx += gx < 0 ? g.n : 0;
            } else {
                gx += gx < 0 ? g.n : (gx >= g.n ? -g.n : 0);
            }
            const float v = row[gx];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c >= k) s[k * CP + r * PP + c - k] = v;
        }
    }
}

/* row pitch of the four-copy FP32 halo: P rounded up to a multiple of 4 (16-byte aligned rows) */
__host__ __device__ constexpr int halo_quad_pitch(int P) { return (P + 3) & ~3; }

/* FP32C: FP32 window values and row sums, rows combined in FP64.  The taps of a row are read
 * four cells at a time (16-byte loads from the four-copy halo): a quarter of the load
 * instructions, and a quarter-warp's 16-byte reads collide on fewer banks than a warp's 4-byte
 * reads (the targets of a warp tap random cells). */
template <int W> __device__ void st_interp32(const Inst &d, int item, unsigned char *sm)
{
    float *sg = reinterpret_cast<float *>(sm);
    const Geom &g = d.g;
    const int T = g.Ti, P = T + W, lo = W / 2, PP = halo_quad_pitch(P), CP = P * PP;
    const int tyi = item / g.nti, txi = item - tyi * g.nti;
    const int beg = d.trg_ptr[item], end = d.trg_ptr[item + 1];
    if (beg == end) return;
    const int X0 = txi * T - lo, Y0 = tyi * T - lo;
    stage_halo_quad32(sg, static_cast<const float *>(d.grid), g, X0, Y0, P, PP);
    __syncthreads();
    const int4 *__restrict__ trg = reinterpret_cast<const int4 *>(d.trg_t);
    const float beta = (float)g.beta, cw = (float)g.c;
    for (int e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const int4 r = trg[e];
        const float sx = __int_as_float(r.z), sy = __int_as_float(r.w);
        float fx[W], fy[W];
#pragma unroll
        for (int a = 0; a < W; ++a) {
            fx[a] = es_window32(sx + (float)a, beta, cw);
            fy[a] = es_window32(sy + (float)a, beta, cw);
        }
        /* cells cx .. cx + W - 1 of a row (0 <= cx <= T): copy (cx mod 4) from column cx - k */
        const int cx = r.x - X0, cy = r.y - Y0, k = cx & 3;
        const float *base = sg + k * CP + cy * PP + (cx - k);
        /* FP32 row sums combined in double-float (the exact product of the FP32 weight and row
         * sum added by two-sum): the final accumulation keeps ~48 bits, on the FP32 pipe */
        df32 acc(0.0f, 0.0f);
#pragma unroll
        for (int cc = 0; cc < W; ++cc) {
            const float4 *q = reinterpret_cast<const float4 *>(base + cc * PP);
            float row = 0.0f;
#pragma unroll
            for (int a = 0; a + 3 < W; a += 4) {
                const float4 v = q[a >> 2];
                row = fmaf(fx[a], v.x, row);
                row = fmaf(fx[a + 1], v.y, row);
                row = fmaf(fx[a + 2], v.z, row);
                row = fmaf(fx[a + 3], v.w, row);
            }
#pragma unroll
            for (int a = W & ~3; a < W; ++a) row = fmaf(fx[a], base[cc * PP + a], row);
            acc = df_mul_add(acc, df32(fy[cc], 0.0f), df32(row, 0.0f));
        }
        d.u[d.trg_idx[e]] = acc.to_double();
    }
    __syncthreads();
}

/* the double-float halo twice, with an even row pitch PP: copy 0 holds cell (X0 + c, Y0 + r) at
 * r PP + c and copy 1 the cell to its right (X0 + c + 1) at the same place, so that any two
 * neighbouring cells of a row are one aligned 16-byte load from one of the copies (copy 0 from an
 * even column, copy 1 from an odd one).  Rows by warp, columns by lane, as stage_halo. */
__device__ __forceinline__ void stage_halo_pair_df(df32 *s0, df32 *s1, const df32 *__restrict__ grid,
                                                   const Geom &g, int X0, int Y0, int P, int PP)
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < P; r += nw) {
        int gy = Y0 + r;
        if (P > g.n) { /* a halo wider than the grid: plain modulo (not reached with n >= 2T) */
            gy %= g.n;
            gy += gy < 0 ? g.n : 0;
        } else {
            gy += gy < 0 ? g.n : (gy >= g.n ? -g.n : 0);
        }
        const df32 *__restrict__ row = grid + (size_t)gy * g.n;
        for (int c = lane; c < P; c += 32) {
            int gx = X0 + c;
            if (P > g.n) {
                gx %= g.n;
                gx += gx < 0 ? g.n : 0;
            } else {
                gx += gx < 0 ? g.n : (gx >= g.n ? -g.n : 0);
            }
            const df32 v = row[gx];
            s0[r * PP + c] = v;
            if (c > 0) s1[r * PP + c - 1] = v;
        }
    }
}

/* row pitch of the paired halo: P rounded up to even (16-byte aligned rows) */
__host__ __device__ constexpr int halo_pair_pitch(int P) { return (P + 1) & ~1; }

/* FP64 path, double-float arithmetic: windows and tap sums in FP32 pairs, one conversion to
 * double per target.  The taps of a row are read two cells at a time (16-byte loads from the
 * paired halo): half the load instructions of one 8-byte load per cell, and a quarter-warp's
 * 16-byte reads collide on fewer banks than a half-warp's 8-byte reads (the targets of a warp tap
 * random cells). */
template <int W> __device__ void st_interp_df(const Inst &d, int item, unsigned char *sm)
{
    const Geom &g = d.g;
    const int T = g.Ti, P = T + W, lo = W / 2, PP = halo_pair_pitch(P);
    df32 *s0 = reinterpret_cast<df32 *>(sm);
    df32 *s1 = s0 + P * PP;
    const int tyi = item / g.nti, txi = item - tyi * g.nti;
    const int beg = d.trg_ptr[item], end = d.trg_ptr[item + 1];
    if (beg == end) return;
    const int X0 = txi * T - lo, Y0 = tyi * T - lo;
    stage_halo_pair_df(s0, s1, static_cast<const df32 *>(d.grid), g, X0, Y0, P, PP);
    __syncthreads();
    const int4 *__restrict__ trg = reinterpret_cast<const int4 *>(d.trg_t);
    for (int e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const int4 r = trg[e]; /* first taps (lx, ly), from the fixed-point preparation */
        const int cx = r.x - X0, cy = r.y - Y0; /* 0 <= cx, cy <= T */
        /* window values of this target, computed at yk_set_points: planes [phi_y taps | phi_x
         * taps], value k at k * pitch + e (consecutive threads read consecutive targets) */
        const float2 *wv = d.win_trg + e;
        const int64_t pw = d.win_trg_pitch;
        df32 fx[W];
#pragma unroll
        for (int a = 0; a < W; ++a) {
            const float2 v = wv[(W + a) * pw];
            fx[a] = df32(v.x, v.y);
        }
        /* cells cx .. cx + W - 1 of a row: from copy 0 at cx (even) or copy 1 at cx - 1 (odd) */
        const df32 *base = ((cx & 1) ? s1 + (cx - 1) : s0 + cx) + cy * PP;
        df32 acc(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < W; ++c) {
            /* row sum of W products with the unnormalised multiply-add (exact two-sum of the
             * high words, low words gathered), renormalised once by a full two-sum */
            const float4 *q = reinterpret_cast<const float4 *>(base + c * PP);
            df32 row(0.0f, 0.0f);
#pragma unroll
            for (int a = 0; a + 1 < W; a += 2) {
                const float4 v = q[a >> 1];
                row = df_mul_add_lazy(row, fx[a], df32(v.x, v.y));
                row = df_mul_add_lazy(row, fx[a + 1], df32(v.z, v.w));
            }
            if (W & 1) row = df_mul_add_lazy(row, fx[W - 1], base[c * PP + W - 1]);
            row = df_two_sum(row.hi, row.lo);
            const float2 wy = wv[c * pw];
            acc = df_mul_add(acc, df32(wy.x, wy.y), row);
        }
        d.u[d.trg_idx[e]] = acc.to_double();
    }
    __syncthreads();
}

/* window width as a template parameter */
#define YK_W_SWITCH(W_, CALL)                                                                    \
    switch (W_) {                                                                                \
    case 2: CALL(2); break;                                                                      \
    case 3: CALL(3); break;                                                                      \
    case 4: CALL(4); break;                                                                      \
    case 5: CALL(5); break;                                                                      \
    case 6: CALL(6); break;                                                                      \
    case 7: CALL(7); break;                                                                      \
    case 8: CALL(8); break;                                                                      \
    case 9: CALL(9); break;                                                                      \
    case 10: CALL(10); break;                                                                    \
    case 11: CALL(11); break;                                                                    \
    case 12: CALL(12); break;                                                                    \
    case 13: CALL(13); break;                                                                    \
    case 14: CALL(14); break;                                                                    \
    case 15: CALL(15); break;                                                                    \
    default: CALL(16); break;                                                                    \
    }

/* run one work item of stage `stage` for instance d (all threads of the CTA) */
template <typename R>
__device__ __forceinline__ void run_stage(const Inst &d, int stage, int item, unsigned char *sm);

template <>
__device__ __forceinline__ void run_stage<double>(const Inst &d, int stage, int item,
                                                  unsigned char *sm)
{
    switch (stage) {
    case ST_SPREAD:
        if (d.fft_df && d.part) {
#define YK_C(W)                                                                                  \
    if (d.dip) st_spread_owner_df<W, true>(d, item, sm);                                         \
    else st_spread_owner_df<W, false>(d, item, sm)
            YK_W_SWITCH(d.g.w, YK_C)
#undef YK_C
        } else {
#define YK_C(W) st_spread64<W>(d, item, sm)
            YK_W_SWITCH(d.g.w, YK_C)
#undef YK_C
        }
        break;
    case ST_ROW_FWD:
        if (d.fft_df) st_row_fwd<df32>(d, item, sm);
        else st_row_fwd<double>(d, item, sm);
        break;
    case ST_COLUMNS:
        if (d.fft_df) st_columns<df32>(d, item, sm);
        else st_columns<double>(d, item, sm);
        break;
    case ST_ROW_INV:
        if (d.fft_df) st_row_inv<df32>(d, item, sm);
        else st_row_inv<double>(d, item, sm);
        break;
    default:
        if (d.fft_df) {
#define YK_C(W) st_interp_df<W>(d, item, sm)
            YK_W_SWITCH(d.g.w, YK_C)
#undef YK_C
        } else {
#define YK_C(W) st_interp64<W>(d, item, sm)
            YK_W_SWITCH(d.g.w, YK_C)
#undef YK_C
        }
        break;
    }
}

template <>
__device__ __forceinline__ void run_stage<float>(const Inst &d, int stage, int item,
                                                 unsigned char *sm)
{
    switch (stage) {
    case ST_SPREAD: {
#define YK_C(W)                                                                                  \
    if (d.dip) st_spread_owner32<W, true>(d, item, sm);                                          \
    else st_spread_owner32<W, false>(d, item, sm)
        YK_W_SWITCH(d.g.w, YK_C)
#undef YK_C
    } break;
    case ST_ROW_FWD: st_row_fwd<float>(d, item, sm); break;
    case ST_COLUMNS: st_columns<float>(d, item, sm); break;
    case ST_ROW_INV: st_row_inv<float>(d, item, sm); break;
    default: {
#define YK_C(W) st_interp32<W>(d, item, sm)
        YK_W_SWITCH(d.g.w, YK_C)
#undef YK_C
    } break;
    }
}

/* the same dispatch for one compile-time window width (the batch kernel is instantiated per
 * width, so its registers are those of that width's stage bodies, not of the widest) */
template <typename R, int W>
__device__ __forceinline__ void run_stage_w(const Inst &d, int stage, int item, unsigned char *sm)
{
    if constexpr (std::is_same<R, float>::value) {
        switch (stage) {
        case ST_SPREAD:
            if (d.dip) st_spread_owner32<W, true>(d, item, sm);
            else st_spread_owner32<W, false>(d, item, sm);
            break;
        case ST_ROW_FWD: st_row_fwd<float>(d, item, sm); break;
        case ST_COLUMNS: st_columns<float>(d, item, sm); break;
        case ST_ROW_INV: st_row_inv<float>(d, item, sm); break;
        default: st_interp32<W>(d, item, sm); break;
        }
    } else {
        switch (stage) {
        case ST_SPREAD:
            if (d.fft_df && d.part && d.dip) st_spread_owner_df<W, true>(d, item, sm);
            else if (d.fft_df && d.part) st_spread_owner_df<W, false>(d, item, sm);
            else st_spread64<W>(d, item, sm);
            break;
        case ST_ROW_FWD:
            if (d.fft_df) st_row_fwd<df32>(d, item, sm);
            else st_row_fwd<double>(d, item, sm);
            break;
        case ST_COLUMNS:
            if (d.fft_df) st_columns<df32>(d, item, sm);
            else st_columns<double>(d, item, sm);
            break;
        case ST_ROW_INV:
            if (d.fft_df) st_row_inv<df32>(d, item, sm);
            else st_row_inv<double>(d, item, sm);
            break;
        default:
            if (d.fft_df) st_interp_df<W>(d, item, sm);
            else st_interp64<W>(d, item, sm);
            break;
        }
    }
}

} /* namespace yk */

#endif /* YK_STAGES_CUH */
