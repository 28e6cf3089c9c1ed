/*
 * yk_kernels.cu — sm_103a kernels of the long-range evaluator (FP64 and FP32C paths).
 *
 *   bin        sources -> (source, tile) entries for every tile a source's w x w window touches;
 *              targets -> the tile of their grid cell (counting sort: count, scan, fill)
 *   spread     type-1 step (Section 5.2, eq. disrete_sigma_hat): one CTA per output tile
 *              accumulates the windows of its entries in shared memory and writes its tile of the
 *              grid once; no global atomics.  FP64: 64-bit fixed point (exact, so the result does
 *              not depend on the order of the entries).  FP32C: FP32 products with compensated
 *              (two-sum) hi + lo accumulation.
 *   row_fwd    real-to-complex FFT of every grid row, pruned to |m_x| <= M, stored transposed
 *   columns    per kept m_x: forward FFT along y, multiply by the symbol of eq. sh_fourier (with
 *              the window deconvolution folded in), zero |m_y| > M, inverse FFT along y
 *   row_inv    complex-to-real inverse FFT of every row
 *   interp     type-2 step: one CTA per target tile stages the tile plus halo of the grid in
 *              shared memory and each thread sums the w x w window of one target (FP32C: FP32 row
 *              sums combined in FP64)
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "yk_internal.h"

namespace yk {

namespace {

template <typename R> struct V2;
template <> struct V2<double> {
    using T = double2;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <> struct V2<float> {
    using T = float2;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};

/* a point is accepted when it lies in the plan's box (closed) */
__device__ __forceinline__ bool in_box(const Geom &g, double x, double y)
{
    return x >= g.box[0] && x <= g.box[1] && y >= g.box[2] && y <= g.box[3];
}

constexpr double kMagic = 6755399441055744.0; /* 1.5 * 2^52: fma(a, b, kMagic) rounds a*b to an integer */

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

/* entry layouts: FP64 keeps the grid coordinate t (double2); FP32C keeps the first tap l0 and
 * the offset s = l0 - t in FP32, both computed from t in FP64 at set-up, so the FP32 kernels
 * never see absolute coordinates (k h |x| eps_32 would otherwise dominate the error) */
template <int W> __device__ __forceinline__ double2 pack_f64(double2 t) { return t; }
template <int W> __device__ __forceinline__ double2 pack_f32c(double2 t)
{
    const int lx = first_tap<W>(t.x), ly = first_tap<W>(t.y);
    const float sx = (float)((double)lx - t.x), sy = (float)((double)ly - t.y);
    double2 r;
    int4 *q = reinterpret_cast<int4 *>(&r);
    *q = make_int4(lx, ly, __float_as_int(sx), __float_as_int(sy));
    return r;
}

/* ----------------------------------------------------------------------------------------- */
/* binning                                                                                    */

template <int W>
__global__ void k_bin_src_count(int64_t ns, const double *__restrict__ xs,
                                const double *__restrict__ ys, Geom g, double2 *__restrict__ src_t,
                                int *__restrict__ cnt, int *__restrict__ err)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    const double tx = (xs[j] - g.ox) * g.inv_h, ty = (ys[j] - g.oy) * g.inv_h;
    if (!in_box(g, xs[j], ys[j]) ||
        !(tx >= 0.0 && tx < (double)g.n && ty >= 0.0 && ty < (double)g.n)) {
        atomicOr(err, ERR_POINT_OUTSIDE);
        src_t[j] = make_double2(-1.0, -1.0);
        return;
    }
    src_t[j] = make_double2(tx, ty);
    const int lx = first_tap<W>(tx), ly = first_tap<W>(ty);
    const int ax0 = wrap(lx, g.n) / g.T, ax1 = wrap(lx + W - 1, g.n) / g.T;
    const int ay0 = wrap(ly, g.n) / g.T, ay1 = wrap(ly + W - 1, g.n) / g.T;
    atomicAdd(&cnt[ay0 * g.nt + ax0], 1);
    if (ax1 != ax0) atomicAdd(&cnt[ay0 * g.nt + ax1], 1);
    if (ay1 != ay0) {
        atomicAdd(&cnt[ay1 * g.nt + ax0], 1);
        if (ax1 != ax0) atomicAdd(&cnt[ay1 * g.nt + ax1], 1);
    }
}

template <int W, bool F32>
__global__ void k_bin_src_fill(int64_t ns, const double2 *__restrict__ src_t, Geom g,
                               const int *__restrict__ ptr, int *__restrict__ cur,
                               double2 *__restrict__ ent_t, int *__restrict__ ent_j)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    const double2 t = src_t[j];
    if (t.x < 0.0) return;
    const int lx = first_tap<W>(t.x), ly = first_tap<W>(t.y);
    const int ax[2] = {wrap(lx, g.n) / g.T, wrap(lx + W - 1, g.n) / g.T};
    const int ay[2] = {wrap(ly, g.n) / g.T, wrap(ly + W - 1, g.n) / g.T};
    const int nx = ax[1] != ax[0] ? 2 : 1, ny = ay[1] != ay[0] ? 2 : 1;
    const double2 rec = F32 ? pack_f32c<W>(t) : pack_f64<W>(t);
    for (int b = 0; b < ny; ++b)
        for (int a = 0; a < nx; ++a) {
            const int tile = ay[b] * g.nt + ax[a];
            const int slot = ptr[tile] + atomicAdd(&cur[tile], 1);
            ent_t[slot] = rec;
            ent_j[slot] = (int)j;
        }
}

__global__ void k_bin_trg_count(int64_t nt, const double *__restrict__ xt,
                                const double *__restrict__ yt, Geom g, double2 *__restrict__ tmp,
                                int *__restrict__ cnt, int *__restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const double tx = (xt[i] - g.ox) * g.inv_h, ty = (yt[i] - g.oy) * g.inv_h;
    if (!in_box(g, xt[i], yt[i]) ||
        !(tx >= 0.0 && tx < (double)g.n && ty >= 0.0 && ty < (double)g.n)) {
        atomicOr(err, ERR_POINT_OUTSIDE);
        tmp[i] = make_double2(-1.0, -1.0);
        return;
    }
    tmp[i] = make_double2(tx, ty);
    const int tile = ((int)ty / g.T) * g.nt + (int)tx / g.T;
    atomicAdd(&cnt[tile], 1);
}

template <int W, bool F32>
__global__ void k_bin_trg_fill(int64_t nt, const double2 *__restrict__ tmp, Geom g,
                               const int *__restrict__ ptr, int *__restrict__ cur,
                               double2 *__restrict__ trg_t, int *__restrict__ trg_idx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const double2 t = tmp[i];
    if (t.x < 0.0) return;
    const int tile = ((int)t.y / g.T) * g.nt + (int)t.x / g.T;
    const int slot = ptr[tile] + atomicAdd(&cur[tile], 1);
    trg_t[slot] = F32 ? pack_f32c<W>(t) : pack_f64<W>(t);
    trg_idx[slot] = (int)i;
}

/* exclusive scan of cnt[0..count) into ptr[0..count] by one CTA of 1024 threads, each owning a
 * contiguous chunk */
__global__ void __launch_bounds__(1024) k_scan(const int *__restrict__ cnt, int *__restrict__ ptr,
                                               int count)
{
    __shared__ int part[1024];
    const int nthr = blockDim.x;
    const int chunk = (count + nthr - 1) / nthr;
    const int b = threadIdx.x * chunk, e = min(count, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < nthr; off <<= 1) {
        int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
    for (int i = b; i < e; ++i) {
        ptr[i] = run;
        run += cnt[i];
    }
    if (threadIdx.x == nthr - 1) ptr[count] = part[nthr - 1];
}

/* heavy-first processing order of the tiles: tiles bucketed by floor(log2(entries)) and listed
 * from the fullest bucket down, so that the costly tiles start first and the short ones fill the
 * tail (one CTA; the order inside a bucket does not affect any result) */
__global__ void __launch_bounds__(1024) k_tile_order(const int *__restrict__ ptr, int ntiles,
                                                     int *__restrict__ order)
{
    __shared__ int hist[33], base[33];
    if (threadIdx.x < 33) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const int c = ptr[t + 1] - ptr[t];
        atomicAdd(&hist[c > 0 ? 32 - __clz(c) : 0], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 32; b >= 0; --b) {
            base[b] = run;
            run += hist[b];
            hist[b] = 0;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const int c = ptr[t + 1] - ptr[t];
        const int b = c > 0 ? 32 - __clz(c) : 0;
        order[base[b] + atomicAdd(&hist[b], 1)] = t;
    }
}

/* ----------------------------------------------------------------------------------------- */
/* spread (type 1)                                                                            */

template <int W>
__global__ void __launch_bounds__(256)
    k_spread(const int *__restrict__ tile_ptr, const int *__restrict__ order,
             const double2 *__restrict__ ent_t, const int *__restrict__ ent_j,
             const double *__restrict__ wq, const double *__restrict__ dens, Geom g,
             double *__restrict__ grid)
{
    extern __shared__ unsigned long long acc[]; /* T x T fixed-point accumulators */
    __shared__ double red[32];
    __shared__ int s_k;
    const int T = g.T, tile = order ? order[blockIdx.x] : blockIdx.x;
    const int tyi = tile / g.nt, txi = tile - tyi * g.nt;
    const int X0 = txi * T, Y0 = tyi * T;
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) acc[i] = 0ull;
    const int beg = tile_ptr[tile], end = tile_ptr[tile + 1];

    /* per-tile scale 2^k: every product |q| phi phi <= max|q| stays below 2^51 (so one fma
     * with 1.5 * 2^52 rounds it to an integer) and the sum of all of them below 2^62 */
    double mq = 0.0;
    for (int e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const int j = ent_j[e];
        mq = fmax(mq, fabs(wq[j] * dens[j]));
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
            const double2 t = ent_t[e];
            const int j = ent_j[e];
            const double qs = ldexp(wq[j] * dens[j], kexp);
            const int lx = first_tap<W>(t.x), ly = first_tap<W>(t.y);
            double fx[W], fy[W];
#pragma unroll
            for (int a = 0; a < W; ++a) {
                fx[a] = es_window<double>((double)(lx + a) - t.x, g.beta, g.c);
                fy[a] = es_window<double>((double)(ly + a) - t.y, g.beta, g.c);
            }
            int dx0 = (lx - X0) % g.n;
            if (dx0 < 0) dx0 += g.n;
            int dy0 = (ly - Y0) % g.n;
            if (dy0 < 0) dy0 += g.n;
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
}

/* FP32C spread: FP32 window values and products, compensated (two-sum) accumulation.  Each warp
 * owns a private hi + lo copy of the tile; it evaluates the windows of 32 entries (one per lane),
 * then walks them one entry at a time with one lane per tap, so the taps a warp updates together
 * are distinct cells and no atomics are needed.  The warps' copies are combined in a fixed order
 * with two-sum at the end. */
constexpr int kSpreadWarps = 8;

template <int W>
__global__ void __launch_bounds__(32 * kSpreadWarps)
    k_spread32(const int *__restrict__ tile_ptr, const int *__restrict__ order,
               const int4 *__restrict__ ent, const int *__restrict__ ent_j,
               const double *__restrict__ wq, const double *__restrict__ dens, Geom g,
               float *__restrict__ grid)
{
    extern __shared__ __align__(16) unsigned char sm32[];
    const int T = g.T, PT = T + 1; /* padded pitch (float2 units) */
    float2 *acc = reinterpret_cast<float2 *>(sm32);                 /* [warps][T][PT] */
    float *wbuf = reinterpret_cast<float *>(acc + kSpreadWarps * T * PT); /* [warps][32][2W] */
    int *obuf = reinterpret_cast<int *>(wbuf + kSpreadWarps * 32 * 2 * W); /* [warps][32][2] */
    const int tile = order ? order[blockIdx.x] : blockIdx.x;
    const int tyi = tile / g.nt, txi = tile - tyi * g.nt;
    const int X0 = txi * T, Y0 = tyi * T;
    for (int i = threadIdx.x; i < kSpreadWarps * T * PT; i += blockDim.x)
        acc[i] = make_float2(0.0f, 0.0f);
    __syncthreads();
    const int beg = tile_ptr[tile], end = tile_ptr[tile + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *mine = acc + warp * T * PT;
    float *wb = wbuf + warp * 32 * 2 * W;
    int *ob = obuf + warp * 64;
    const float beta = (float)g.beta, cw = (float)g.c;
    for (int b0 = beg + warp * 32; b0 < end; b0 += kSpreadWarps * 32) {
        const int e = b0 + lane;
        if (e < end) {
            const int4 r = ent[e];
            const int j = ent_j[e];
            const float q = (float)(wq[j] * dens[j]);
            const float sx = __int_as_float(r.z), sy = __int_as_float(r.w);
#pragma unroll
            for (int a = 0; a < W; ++a) {
                wb[lane * 2 * W + a] = q * es_window_stable<float>(sy + (float)a, beta, cw);
                wb[lane * 2 * W + W + a] = es_window_stable<float>(sx + (float)a, beta, cw);
            }
            int dx0 = (r.x - X0) % g.n;
            if (dx0 < 0) dx0 += g.n;
            int dy0 = (r.y - Y0) % g.n;
            if (dy0 < 0) dy0 += g.n;
            ob[2 * lane] = dx0;
            ob[2 * lane + 1] = dy0;
        }
        __syncwarp();
        const int cnt = min(32, end - b0);
        for (int k = 0; k < cnt; ++k) {
            const int dx0 = ob[2 * k], dy0 = ob[2 * k + 1];
            const float *wk = wb + k * 2 * W;
#pragma unroll
            for (int t0 = 0; t0 < W * W; t0 += 32) {
                const int t = t0 + lane;
                if (t < W * W) {
                    const int c = t / W, a = t - c * W;
                    int yy = dy0 + c;
                    if (yy >= g.n) yy -= g.n;
                    int xx = dx0 + a;
                    if (xx >= g.n) xx -= g.n;
                    if (yy < T && xx < T) {
                        const float v = wk[c] * wk[W + a];
                        float2 cell = mine[yy * PT + xx];
                        const float s = __fadd_rn(cell.x, v);
                        const float bp = __fsub_rn(s, cell.x);
                        const float err =
                            __fadd_rn(__fsub_rn(cell.x, __fsub_rn(s, bp)), __fsub_rn(v, bp));
                        cell.x = s;
                        cell.y = __fadd_rn(cell.y, err);
                        mine[yy * PT + xx] = cell;
                    }
                }
            }
            __syncwarp(); /* the next entry may touch the same cells through other lanes */
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
        const int rr = i / T, cc = i - rr * T;
        float hi = 0.0f, lo = 0.0f;
        for (int w = 0; w < kSpreadWarps; ++w) {
            const float2 p = acc[w * T * PT + rr * PT + cc];
            const float s = __fadd_rn(hi, p.x);
            const float bp = __fsub_rn(s, hi);
            lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p.x, bp)), p.y));
            hi = s;
        }
        grid[(size_t)(Y0 + rr) * g.n + X0 + cc] = hi + lo;
    }
}

/* ----------------------------------------------------------------------------------------- */
/* FFT passes                                                                                 */

template <typename R, typename TW>
__device__ __forceinline__ void fft_fwd(cpx<R> *x, const FftStages &st, const TW *tw, int nrows,
                                        int rowlen)
{
    for (int s = 0; s < st.n; ++s) {
        const int nb = st.L / st.r[s];
        for (int i = threadIdx.x; i < nrows * nb; i += blockDim.x) {
            const int r = i / nb, t = i - r * nb;
            dif_butterfly<R>(x + (size_t)r * rowlen, st, s, t, tw, 1);
        }
        __syncthreads();
    }
}

template <typename R, typename TW>
__device__ __forceinline__ void fft_inv(cpx<R> *x, const FftStages &st, const TW *tw, int nrows,
                                        int rowlen)
{
    for (int s = st.n - 1; s >= 0; --s) {
        const int nb = st.L / st.r[s];
        for (int i = threadIdx.x; i < nrows * nb; i += blockDim.x) {
            const int r = i / nb, t = i - r * nb;
            idif_butterfly<R>(x + (size_t)r * rowlen, st, s, t, tw, 1);
        }
        __syncthreads();
    }
}

template <typename R>
__global__ void __launch_bounds__(256)
    k_row_fwd(const R *__restrict__ grid, typename V2<R>::T *__restrict__ spec,
              const typename V2<R>::T *__restrict__ tw, const int *__restrict__ perm_h,
              FftStages st, int n, int M, int rows)
{
    using C2 = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R> *x = reinterpret_cast<cpx<R> *>(smraw);
    const int L = n >> 1;
    const int y0 = blockIdx.x * rows;
    const int nr = min(rows, n - y0);
    for (int i = threadIdx.x; i < nr * L; i += blockDim.x) {
        const int r = i / L, l = i - r * L;
        const C2 v = reinterpret_cast<const C2 *>(grid + (size_t)(y0 + r) * n)[l];
        x[i] = mk<R>(v.x, v.y);
    }
    __syncthreads();
    fft_fwd<R>(x, st, tw, nr, L);
    for (int i = threadIdx.x; i < nr * (M + 1); i += blockDim.x) {
        const int m = i / nr, r = i - m * nr;
        const cpx<R> Zm = x[r * L + perm_h[m]];
        const cpx<R> Zc = x[r * L + perm_h[m == 0 ? 0 : L - m]];
        const C2 wm = tw[m];
        const cpx<R> X = r2c_post<R>(Zm, Zc, mk<R>(wm.x, wm.y));
        spec[(size_t)m * n + y0 + r] = V2<R>::make(X.re, X.im);
    }
}

template <typename R>
__global__ void __launch_bounds__(512)
    k_columns(typename V2<R>::T *__restrict__ spec, const R *__restrict__ mult,
              const typename V2<R>::T *__restrict__ tw, const int *__restrict__ iperm_f,
              FftStages st, int n, int M)
{
    using C2 = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R> *x = reinterpret_cast<cpx<R> *>(smraw);
    const int kx = blockIdx.x;
    C2 *col = spec + (size_t)kx * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const C2 v = col[i];
        x[i] = mk<R>(v.x, v.y);
    }
    __syncthreads();
    fft_fwd<R>(x, st, tw, 1, n);
    const R *mrow = mult + (size_t)kx * (2 * M + 1);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int m = iperm_f[i];
        const int my = m <= (n >> 1) ? m : m - n;
        if (my >= -M && my <= M) x[i] = scale(x[i], mrow[my + M]);
        else x[i] = mk<R>((R)0, (R)0);
    }
    __syncthreads();
    fft_inv<R>(x, st, tw, 1, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = V2<R>::make(x[i].re, x[i].im);
}

template <typename R>
__global__ void __launch_bounds__(256)
    k_row_inv(const typename V2<R>::T *__restrict__ spec, R *__restrict__ grid,
              const typename V2<R>::T *__restrict__ tw, const int *__restrict__ perm_h,
              FftStages st, int n, int M, int rows)
{
    using C2 = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    cpx<R> *x = reinterpret_cast<cpx<R> *>(smraw);
    const int L = n >> 1;
    const int y0 = blockIdx.x * rows;
    const int nr = min(rows, n - y0);
    for (int i = threadIdx.x; i < nr * L; i += blockDim.x) {
        const int m = i / nr, r = i - m * nr;
        const int mc = L - m; /* in (0, L]; X[L] is zero because M < L */
        C2 a = V2<R>::make((R)0, (R)0), b = V2<R>::make((R)0, (R)0);
        if (m <= M) a = spec[(size_t)m * n + y0 + r];
        if (mc <= M) b = spec[(size_t)mc * n + y0 + r];
        const C2 wm = tw[m];
        x[r * L + perm_h[m]] = c2r_pre<R>(mk<R>(a.x, a.y), mk<R>(b.x, b.y), mk<R>(wm.x, wm.y));
    }
    __syncthreads();
    fft_inv<R>(x, st, tw, nr, L);
    for (int i = threadIdx.x; i < nr * L; i += blockDim.x) {
        const int r = i / L, l = i - r * L;
        reinterpret_cast<C2 *>(grid + (size_t)(y0 + r) * n)[l] = V2<R>::make(x[i].re, x[i].im);
    }
}

/* ----------------------------------------------------------------------------------------- */
/* interpolation (type 2)                                                                     */

template <typename R>
__device__ __forceinline__ void stage_halo(R *sg, const R *__restrict__ grid, const Geom &g,
                                           int X0, int Y0, int P)
{
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
        const int r = i / P, c = i - r * P;
        int gy = (Y0 + r) % g.n;
        if (gy < 0) gy += g.n;
        int gx = (X0 + c) % g.n;
        if (gx < 0) gx += g.n;
        sg[i] = grid[(size_t)gy * g.n + gx];
    }
}

template <int W>
__global__ void __launch_bounds__(256)
    k_interp(const int *__restrict__ trg_ptr, const double2 *__restrict__ trg_t,
             const int *__restrict__ trg_idx, Geom g, const double *__restrict__ grid,
             double *__restrict__ u)
{
    extern __shared__ double sg[];
    const int T = g.T, P = T + W, lo = W / 2;
    const int tile = blockIdx.x;
    const int tyi = tile / g.nt, txi = tile - tyi * g.nt;
    const int beg = trg_ptr[tile], end = trg_ptr[tile + 1];
    if (beg == end) return;
    const int X0 = txi * T - lo, Y0 = tyi * T - lo;
    stage_halo<double>(sg, grid, g, X0, Y0, P);
    __syncthreads();
    for (int e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const double2 t = trg_t[e];
        const int lx = first_tap<W>(t.x), ly = first_tap<W>(t.y);
        double fx[W], fy[W];
#pragma unroll
        for (int a = 0; a < W; ++a) {
            fx[a] = es_window<double>((double)(lx + a) - t.x, g.beta, g.c);
            fy[a] = es_window<double>((double)(ly + a) - t.y, g.beta, g.c);
        }
        const double *base = sg + (ly - Y0) * P + (lx - X0);
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < W; ++c) {
            double row = 0.0;
#pragma unroll
            for (int a = 0; a < W; ++a) row = fma(fx[a], base[c * P + a], row);
            acc = fma(fy[c], row, acc);
        }
        u[trg_idx[e]] = acc;
    }
}

template <int W>
__global__ void __launch_bounds__(256)
    k_interp32(const int *__restrict__ trg_ptr, const int4 *__restrict__ trg,
               const int *__restrict__ trg_idx, Geom g, const float *__restrict__ grid,
               double *__restrict__ u)
{
    extern __shared__ float sgf[];
    const int T = g.T, P = T + W, lo = W / 2;
    const int tile = blockIdx.x;
    const int tyi = tile / g.nt, txi = tile - tyi * g.nt;
    const int beg = trg_ptr[tile], end = trg_ptr[tile + 1];
    if (beg == end) return;
    const int X0 = txi * T - lo, Y0 = tyi * T - lo;
    stage_halo<float>(sgf, grid, g, X0, Y0, P);
    __syncthreads();
    const float beta = (float)g.beta, c = (float)g.c;
    for (int e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const int4 r = trg[e];
        const float sx = __int_as_float(r.z), sy = __int_as_float(r.w);
        float fx[W], fy[W];
#pragma unroll
        for (int a = 0; a < W; ++a) {
            fx[a] = es_window_stable<float>(sx + (float)a, beta, c);
            fy[a] = es_window_stable<float>(sy + (float)a, beta, c);
        }
        const float *base = sgf + (r.y - Y0) * P + (r.x - X0);
        double acc = 0.0;
#pragma unroll
        for (int cc = 0; cc < W; ++cc) {
            float row = 0.0f;
#pragma unroll
            for (int a = 0; a < W; ++a) row = fmaf(fx[a], base[cc * P + a], row);
            acc = fma((double)fy[cc], (double)row, acc);
        }
        u[trg_idx[e]] = acc;
    }
}

/* ----------------------------------------------------------------------------------------- */
/* multiplier: mult[kx][my + M] = exp(-delta (alpha^2 + k^2)) / (alpha^2 + k^2) / P^2          */
/*                                 * dfac[kx] * dfac[|my|],  k = (2 pi / P) (kx, my)            */
/* (eq. sh_fourier with Delta k = 2 pi / P, so (Delta k)^2 / (2 pi)^2 = 1 / P^2; dfac is the   */
/* squared inverse window transform that undoes spreading and interpolation).  Evaluated in    */
/* FP64 and rounded once to the table's type.                                                  */
template <typename R>
__global__ void k_build_mult(R *__restrict__ mult, const double *__restrict__ dfac, int M,
                             double alpha, double delta, double dk, double period)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t w = 2 * M + 1;
    if (i >= (int64_t)(M + 1) * w) return;
    const int kx = (int)(i / w), my = (int)(i - (int64_t)kx * w) - M;
    const double k2 = dk * dk * ((double)kx * kx + (double)my * my);
    const double s = alpha * alpha + k2;
    mult[i] = (R)(exp(-delta * s) / s / (period * period) * dfac[kx] * dfac[my < 0 ? -my : my]);
}

template <typename K> cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

inline int rows_per_cta(int n, size_t cbytes)
{
    const int bytes_per_row = (n / 2) * (int)cbytes;
    int r = (96 * 1024) / bytes_per_row;
    return r < 1 ? 1 : (r > 16 ? 16 : r);
}

} /* namespace */

/* ----------------------------------------------------------------------------------------- */
/* launchers                                                                                  */

#define YK_W_DISPATCH(W_, CALL)                                                                  \
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
    case 16: CALL(16); break;                                                                    \
    default: return cudaErrorInvalidValue;                                                       \
    }

cudaError_t launch_bin_sources(const Geom &g, int64_t ns, const double *xs, const double *ys,
                               double2 *src_t, int *tile_cnt, int *tile_ptr, int *tile_cur,
                               double2 *ent_t, int *ent_j, int *err, cudaStream_t st, bool f32)
{
    const int ntiles = g.nt * g.nt;
    cudaError_t e = cudaMemsetAsync(tile_cnt, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(tile_cur, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((ns + 255) / 256);
    if (ns > 0) {
#define YK_CALL(W) k_bin_src_count<W><<<blocks, 256, 0, st>>>(ns, xs, ys, g, src_t, tile_cnt, err)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    k_scan<<<1, 1024, 0, st>>>(tile_cnt, tile_ptr, ntiles);
    if (ns > 0) {
#define YK_CALL(W)                                                                              \
    if (f32)                                                                                    \
        k_bin_src_fill<W, true><<<blocks, 256, 0, st>>>(ns, src_t, g, tile_ptr, tile_cur, ent_t, \
                                                        ent_j);                                 \
    else                                                                                        \
        k_bin_src_fill<W, false><<<blocks, 256, 0, st>>>(ns, src_t, g, tile_ptr, tile_cur,      \
                                                         ent_t, ent_j)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    return cudaGetLastError();
}

cudaError_t launch_bin_targets(const Geom &g, int64_t nt, const double *xt, const double *yt,
                               double2 *trg_tmp, int *cnt, int *ptr, int *cur, double2 *trg_t,
                               int *trg_idx, int *err, cudaStream_t st, bool f32)
{
    const int ntiles = g.nt * g.nt;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(cur, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((nt + 255) / 256);
    if (nt > 0) k_bin_trg_count<<<blocks, 256, 0, st>>>(nt, xt, yt, g, trg_tmp, cnt, err);
    k_scan<<<1, 1024, 0, st>>>(cnt, ptr, ntiles);
    if (nt > 0) {
#define YK_CALL(W)                                                                              \
    if (f32)                                                                                    \
        k_bin_trg_fill<W, true><<<blocks, 256, 0, st>>>(nt, trg_tmp, g, ptr, cur, trg_t, trg_idx); \
    else                                                                                        \
        k_bin_trg_fill<W, false><<<blocks, 256, 0, st>>>(nt, trg_tmp, g, ptr, cur, trg_t, trg_idx)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const int *tile_ptr, int ntiles, int *order, cudaStream_t st)
{
    k_tile_order<<<1, 1024, 0, st>>>(tile_ptr, ntiles, order);
    return cudaGetLastError();
}

cudaError_t launch_spread(const Geom &g, const int *tile_ptr, const int *order,
                          const double2 *ent_t, const int *ent_j, const double *wq,
                          const double *dens, double *grid, cudaStream_t st)
{
    const size_t smem = sizeof(unsigned long long) * g.T * g.T;
    const int ntiles = g.nt * g.nt;
    cudaError_t e = cudaSuccess;
#define YK_CALL(W)                                                                          \
    e = set_smem(k_spread<W>, smem);                                                        \
    if (e != cudaSuccess) return e;                                                         \
    k_spread<W><<<ntiles, 256, smem, st>>>(tile_ptr, order, ent_t, ent_j, wq, dens, g, grid)
    YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    return cudaGetLastError();
}

cudaError_t launch_spread32(const Geom &g, const int *tile_ptr, const int *order,
                            const double2 *ent_t, const int *ent_j, const double *wq,
                            const double *dens, float *grid, cudaStream_t st)
{
    const size_t smem = sizeof(float2) * kSpreadWarps * g.T * (g.T + 1) +
                        sizeof(float) * kSpreadWarps * 32 * 2 * g.w +
                        sizeof(int) * kSpreadWarps * 64;
    const int ntiles = g.nt * g.nt;
    const int4 *ent = reinterpret_cast<const int4 *>(ent_t);
    cudaError_t e = cudaSuccess;
#define YK_CALL(W)                                                                          \
    e = set_smem(k_spread32<W>, smem);                                                      \
    if (e != cudaSuccess) return e;                                                         \
    k_spread32<W><<<ntiles, 32 * kSpreadWarps, smem, st>>>(tile_ptr, order, ent, ent_j, wq, dens, \
                                                           g, grid)
    YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_row_fwd_t(const R *grid, typename V2<R>::T *spec, const typename V2<R>::T *tw,
                             const int *perm_h, const FftStages &sth, int n, int M,
                             cudaStream_t st)
{
    const int rows = rows_per_cta(n, sizeof(cpx<R>));
    const size_t smem = sizeof(cpx<R>) * (size_t)rows * (n / 2);
    cudaError_t e = set_smem(k_row_fwd<R>, smem);
    if (e != cudaSuccess) return e;
    k_row_fwd<R><<<(n + rows - 1) / rows, 256, smem, st>>>(grid, spec, tw, perm_h, sth, n, M, rows);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_columns_t(typename V2<R>::T *spec, const R *mult, const typename V2<R>::T *tw,
                             const int *iperm_f, const FftStages &stf, int n, int M,
                             cudaStream_t st)
{
    const size_t smem = sizeof(cpx<R>) * (size_t)n;
    cudaError_t e = set_smem(k_columns<R>, smem);
    if (e != cudaSuccess) return e;
    k_columns<R><<<M + 1, 512, smem, st>>>(spec, mult, tw, iperm_f, stf, n, M);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_row_inv_t(const typename V2<R>::T *spec, R *grid, const typename V2<R>::T *tw,
                             const int *perm_h, const FftStages &sth, int n, int M,
                             cudaStream_t st)
{
    const int rows = rows_per_cta(n, sizeof(cpx<R>));
    const size_t smem = sizeof(cpx<R>) * (size_t)rows * (n / 2);
    cudaError_t e = set_smem(k_row_inv<R>, smem);
    if (e != cudaSuccess) return e;
    k_row_inv<R><<<(n + rows - 1) / rows, 256, smem, st>>>(spec, grid, tw, perm_h, sth, n, M, rows);
    return cudaGetLastError();
}

cudaError_t launch_row_fwd(const double *grid, double2 *spec, const double2 *tw, const int *perm_h,
                           const FftStages &sth, int n, int M, cudaStream_t st)
{
    return launch_row_fwd_t<double>(grid, spec, tw, perm_h, sth, n, M, st);
}
cudaError_t launch_columns(double2 *spec, const double *mult, const double2 *tw,
                           const int *iperm_f, const FftStages &stf, int n, int M,
                           cudaStream_t st)
{
    return launch_columns_t<double>(spec, mult, tw, iperm_f, stf, n, M, st);
}
cudaError_t launch_row_inv(const double2 *spec, double *grid, const double2 *tw,
                           const int *perm_h, const FftStages &sth, int n, int M,
                           cudaStream_t st)
{
    return launch_row_inv_t<double>(spec, grid, tw, perm_h, sth, n, M, st);
}
cudaError_t launch_row_fwd32(const float *grid, float2 *spec, const float2 *tw, const int *perm_h,
                             const FftStages &sth, int n, int M, cudaStream_t st)
{
    return launch_row_fwd_t<float>(grid, spec, tw, perm_h, sth, n, M, st);
}
cudaError_t launch_columns32(float2 *spec, const float *mult, const float2 *tw,
                             const int *iperm_f, const FftStages &stf, int n, int M,
                             cudaStream_t st)
{
    return launch_columns_t<float>(spec, mult, tw, iperm_f, stf, n, M, st);
}
cudaError_t launch_row_inv32(const float2 *spec, float *grid, const float2 *tw, const int *perm_h,
                             const FftStages &sth, int n, int M, cudaStream_t st)
{
    return launch_row_inv_t<float>(spec, grid, tw, perm_h, sth, n, M, st);
}

cudaError_t launch_interp(const Geom &g, const int *trg_ptr, const double2 *trg_t,
                          const int *trg_idx, const double *grid, double *u, cudaStream_t st)
{
    const size_t smem = sizeof(double) * (size_t)(g.T + g.w) * (g.T + g.w);
    const int ntiles = g.nt * g.nt;
    cudaError_t e = cudaSuccess;
#define YK_CALL(W)                                                                          \
    e = set_smem(k_interp<W>, smem);                                                        \
    if (e != cudaSuccess) return e;                                                         \
    k_interp<W><<<ntiles, 256, smem, st>>>(trg_ptr, trg_t, trg_idx, g, grid, u)
    YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    return cudaGetLastError();
}

cudaError_t launch_interp32(const Geom &g, const int *trg_ptr, const double2 *trg_t,
                            const int *trg_idx, const float *grid, double *u, cudaStream_t st)
{
    const size_t smem = sizeof(float) * (size_t)(g.T + g.w) * (g.T + g.w);
    const int ntiles = g.nt * g.nt;
    const int4 *trg = reinterpret_cast<const int4 *>(trg_t);
    cudaError_t e = cudaSuccess;
#define YK_CALL(W)                                                                          \
    e = set_smem(k_interp32<W>, smem);                                                      \
    if (e != cudaSuccess) return e;                                                         \
    k_interp32<W><<<ntiles, 256, smem, st>>>(trg_ptr, trg, trg_idx, g, grid, u)
    YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    return cudaGetLastError();
}

cudaError_t launch_build_mult(double *mult, const double *dfac, int M, double alpha, double delta,
                              double dk, double period, cudaStream_t st)
{
    const int64_t total = (int64_t)(M + 1) * (2 * M + 1);
    k_build_mult<double><<<(int)((total + 255) / 256), 256, 0, st>>>(mult, dfac, M, alpha, delta,
                                                                     dk, period);
    return cudaGetLastError();
}

cudaError_t launch_build_mult32(float *mult, const double *dfac, int M, double alpha,
                                double delta, double dk, double period, cudaStream_t st)
{
    const int64_t total = (int64_t)(M + 1) * (2 * M + 1);
    k_build_mult<float><<<(int)((total + 255) / 256), 256, 0, st>>>(mult, dfac, M, alpha, delta,
                                                                    dk, period);
    return cudaGetLastError();
}

} /* namespace yk */
