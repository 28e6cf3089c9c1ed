/*
 * yk_kernels.cu — sm_103a kernels of the long-range evaluator (FP64 and FP32C paths): the binning
 * kernels and one kernel per evaluation stage, each a thin wrapper (one CTA per work item) around
 * the stage bodies in yk_stages.cuh.
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
#include <string.h>

#include "yk_stages.cuh"

namespace yk {

namespace {

/* a point is accepted when it lies in the plan's box (closed) */
__device__ __forceinline__ bool in_box(const Geom &g, double x, double y)
{
    return x >= g.box[0] && x <= g.box[1] && y >= g.box[2] && y <= g.box[3];
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
/* per-stage kernels: one CTA per work item                                                   */

template <int W> __global__ void __launch_bounds__(256) k_spread(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_spread64<W>(d, blockIdx.x, sm);
}
template <int W> __global__ void __launch_bounds__(32 * kSpreadWarps) k_spread32(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_spread32<W>(d, blockIdx.x, sm);
}
template <int W> __global__ void __launch_bounds__(32 * kSpreadWarps) k_spread_df(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_spread_df<W>(d, blockIdx.x, sm);
}
template <int W> __global__ void __launch_bounds__(256) k_interp_df(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_interp_df<W>(d, blockIdx.x, sm);
}
template <typename R> __global__ void __launch_bounds__(512) k_row_fwd(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_row_fwd<R>(d, blockIdx.x, sm);
}
template <typename R> __global__ void __launch_bounds__(1024) k_columns(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_columns<R>(d, blockIdx.x, sm);
}
template <typename R> __global__ void __launch_bounds__(512) k_row_inv(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_row_inv<R>(d, blockIdx.x, sm);
}
template <int W> __global__ void __launch_bounds__(256) k_interp(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_interp64<W>(d, blockIdx.x, sm);
}
template <int W> __global__ void __launch_bounds__(256) k_interp32(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_interp32<W>(d, blockIdx.x, sm);
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

/* an Inst holding only what one launcher needs */
Inst blank_inst(int n, int M)
{
    Inst d;
    memset(&d, 0, sizeof d);
    d.n = n;
    d.M = M;
    return d;
}

} /* namespace */

/* ----------------------------------------------------------------------------------------- */
/* stage geometry                                                                              */

int rows_per_item(int n, bool f32)
{
    const int bytes_per_row = (n / 2) * (f32 ? 8 : 16);
    int r = (96 * 1024) / bytes_per_row;
    return r < 1 ? 1 : (r > 16 ? 16 : r);
}

int stage_items(const Inst &d, int stage)
{
    switch (stage) {
    case ST_SPREAD:
    case ST_INTERP: return d.g.nt * d.g.nt;
    case ST_ROW_FWD:
    case ST_ROW_INV: return (d.n + d.rows - 1) / d.rows;
    default: return d.M + 1;
    }
}

int stage_smem(const Inst &d, int stage)
{
    const int T = d.g.T, W = d.g.w;
    const int win_bytes = d.win ? (int)sizeof(double) * (d.wdeg + 1) * W : 0;
    const int c = d.f32 ? 8 : 16; /* bytes of a complex value */
    switch (stage) {
    case ST_SPREAD:
        if (d.fft_df)
            return (int)(sizeof(df32) * kSpreadWarps * T * (T + 1) +
                         sizeof(df32) * kSpreadWarps * 32 * 2 * W + sizeof(int) * kSpreadWarps * 64 +
                         sizeof(df32) * (d.wdeg + 1) * W);
        return d.f32 ? (int)(sizeof(float2) * kSpreadWarps * T * (T + 1) +
                             sizeof(float) * kSpreadWarps * 32 * 2 * W + sizeof(int) * kSpreadWarps * 64)
                     : (int)(sizeof(unsigned long long) * T * T + win_bytes);
    case ST_ROW_FWD:
    case ST_ROW_INV: return c * d.rows * (d.n / 2);
    case ST_COLUMNS: return c * d.n;
    default:
        if (d.fft_df) return 8 * (T + W) * (T + W) + (int)sizeof(df32) * (d.wdeg + 1) * W;
        return d.f32 ? 4 * (T + W) * (T + W) : 8 * (T + W) * (T + W) + win_bytes;
    }
}

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
    Inst d = blank_inst(g.n, 0);
    d.g = g;
    d.tile_ptr = tile_ptr;
    d.order = order;
    d.ent_t = ent_t;
    d.ent_j = ent_j;
    d.wq = wq;
    d.dens = dens;
    d.grid = grid;
    const size_t smem = stage_smem(d, ST_SPREAD);
    cudaError_t e = cudaSuccess;
#define YK_CALL(W)                                                                              \
    e = set_smem(k_spread<W>, smem);                                                            \
    if (e != cudaSuccess) return e;                                                             \
    k_spread<W><<<g.nt * g.nt, 256, smem, st>>>(d)
    YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    return cudaGetLastError();
}

cudaError_t launch_spread32(const Geom &g, const int *tile_ptr, const int *order,
                            const double2 *ent_t, const int *ent_j, const double *wq,
                            const double *dens, float *grid, cudaStream_t st)
{
    Inst d = blank_inst(g.n, 0);
    d.g = g;
    d.f32 = 1;
    d.tile_ptr = tile_ptr;
    d.order = order;
    d.ent_t = ent_t;
    d.ent_j = ent_j;
    d.wq = wq;
    d.dens = dens;
    d.grid = grid;
    const size_t smem = stage_smem(d, ST_SPREAD);
    cudaError_t e = cudaSuccess;
#define YK_CALL(W)                                                                              \
    e = set_smem(k_spread32<W>, smem);                                                          \
    if (e != cudaSuccess) return e;                                                             \
    k_spread32<W><<<g.nt * g.nt, 32 * kSpreadWarps, smem, st>>>(d)
    YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_t(int stage, const void *grid_in, void *grid_out, void *spec,
                         const void *mult, const void *tw, const int *perm_h, const int *iperm_f,
                         const FftStages &sth, const FftStages &stf, int n, int M,
                         cudaStream_t st)
{
    Inst d = blank_inst(n, M);
    d.f32 = sizeof(R) == 4;
    d.rows = rows_per_item(n, d.f32);
    d.grid = stage == ST_ROW_FWD ? const_cast<void *>(grid_in) : grid_out;
    d.spec = spec;
    d.mult = mult;
    d.tw = tw;
    d.perm_h = perm_h;
    d.iperm_f = iperm_f;
    d.sth = sth;
    d.stf = stf;
    const size_t smem = stage_smem(d, stage);
    const int items = stage_items(d, stage);
    cudaError_t e = cudaSuccess;
    if (stage == ST_ROW_FWD) {
        if ((e = set_smem(k_row_fwd<R>, smem)) != cudaSuccess) return e;
        k_row_fwd<R><<<items, 512, smem, st>>>(d);
    } else if (stage == ST_COLUMNS) {
        if ((e = set_smem(k_columns<R>, smem)) != cudaSuccess) return e;
        k_columns<R><<<items, 1024, smem, st>>>(d);
    } else {
        if ((e = set_smem(k_row_inv<R>, smem)) != cudaSuccess) return e;
        k_row_inv<R><<<items, 512, smem, st>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_row_fwd(const double *grid, double2 *spec, const double2 *tw, const int *perm_h,
                           const FftStages &sth, int n, int M, cudaStream_t st)
{
    return launch_fft_t<double>(ST_ROW_FWD, grid, nullptr, spec, nullptr, tw, perm_h, nullptr,
                                sth, sth, n, M, st);
}
cudaError_t launch_columns(double2 *spec, const double *mult, const double2 *tw,
                           const int *iperm_f, const FftStages &stf, int n, int M,
                           cudaStream_t st)
{
    return launch_fft_t<double>(ST_COLUMNS, nullptr, nullptr, spec, mult, tw, nullptr, iperm_f,
                                stf, stf, n, M, st);
}
cudaError_t launch_row_inv(const double2 *spec, double *grid, const double2 *tw,
                           const int *perm_h, const FftStages &sth, int n, int M,
                           cudaStream_t st)
{
    return launch_fft_t<double>(ST_ROW_INV, nullptr, grid, const_cast<double2 *>(spec), nullptr,
                                tw, perm_h, nullptr, sth, sth, n, M, st);
}
cudaError_t launch_row_fwd32(const float *grid, float2 *spec, const float2 *tw, const int *perm_h,
                             const FftStages &sth, int n, int M, cudaStream_t st)
{
    return launch_fft_t<float>(ST_ROW_FWD, grid, nullptr, spec, nullptr, tw, perm_h, nullptr, sth,
                               sth, n, M, st);
}
cudaError_t launch_columns32(float2 *spec, const float *mult, const float2 *tw,
                             const int *iperm_f, const FftStages &stf, int n, int M,
                             cudaStream_t st)
{
    return launch_fft_t<float>(ST_COLUMNS, nullptr, nullptr, spec, mult, tw, nullptr, iperm_f,
                               stf, stf, n, M, st);
}
cudaError_t launch_row_inv32(const float2 *spec, float *grid, const float2 *tw, const int *perm_h,
                             const FftStages &sth, int n, int M, cudaStream_t st)
{
    return launch_fft_t<float>(ST_ROW_INV, nullptr, grid, const_cast<float2 *>(spec), nullptr,
                               tw, perm_h, nullptr, sth, sth, n, M, st);
}

template <bool F32>
cudaError_t launch_interp_t(const Geom &g, const int *trg_ptr, const double2 *trg_t,
                            const int *trg_idx, const void *grid, double *u, cudaStream_t st)
{
    Inst d = blank_inst(g.n, 0);
    d.g = g;
    d.f32 = F32;
    d.trg_ptr = trg_ptr;
    d.trg_t = trg_t;
    d.trg_idx = trg_idx;
    d.grid = const_cast<void *>(grid);
    d.u = u;
    const size_t smem = stage_smem(d, ST_INTERP);
    cudaError_t e = cudaSuccess;
    if (F32) {
#define YK_CALL(W)                                                                              \
    e = set_smem(k_interp32<W>, smem);                                                          \
    if (e != cudaSuccess) return e;                                                             \
    k_interp32<W><<<g.nt * g.nt, 256, smem, st>>>(d)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    } else {
#define YK_CALL(W)                                                                              \
    e = set_smem(k_interp<W>, smem);                                                            \
    if (e != cudaSuccess) return e;                                                             \
    k_interp<W><<<g.nt * g.nt, 256, smem, st>>>(d)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    return cudaGetLastError();
}

cudaError_t launch_interp(const Geom &g, const int *trg_ptr, const double2 *trg_t,
                          const int *trg_idx, const double *grid, double *u, cudaStream_t st)
{
    return launch_interp_t<false>(g, trg_ptr, trg_t, trg_idx, grid, u, st);
}

cudaError_t launch_interp32(const Geom &g, const int *trg_ptr, const double2 *trg_t,
                            const int *trg_idx, const float *grid, double *u, cudaStream_t st)
{
    return launch_interp_t<true>(g, trg_ptr, trg_t, trg_idx, grid, u, st);
}

cudaError_t launch_stage(const Inst &d, int stage, cudaStream_t st)
{
    const size_t smem = stage_smem(d, stage);
    const int items = stage_items(d, stage);
    if (items <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define YK_LAUNCH(K, THREADS)                                                                   \
    do {                                                                                        \
        if ((e = set_smem(K, smem)) != cudaSuccess) return e;                                   \
        K<<<items, THREADS, smem, st>>>(d);                                                     \
    } while (0)
    switch (stage) {
    case ST_SPREAD:
        if (d.f32) {
#define YK_CALL(W) YK_LAUNCH(k_spread32<W>, 32 * kSpreadWarps)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else if (d.fft_df) {
#define YK_CALL(W) YK_LAUNCH(k_spread_df<W>, 32 * kSpreadWarps)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else {
#define YK_CALL(W) YK_LAUNCH(k_spread<W>, 256)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        }
        break;
    case ST_ROW_FWD:
        if (d.f32) YK_LAUNCH(k_row_fwd<float>, 512);
        else if (d.fft_df) YK_LAUNCH(k_row_fwd<df32>, 512);
        else YK_LAUNCH(k_row_fwd<double>, 512);
        break;
    case ST_COLUMNS:
        if (d.f32) YK_LAUNCH(k_columns<float>, 1024);
        else if (d.fft_df) YK_LAUNCH(k_columns<df32>, 1024);
        else YK_LAUNCH(k_columns<double>, 1024);
        break;
    case ST_ROW_INV:
        if (d.f32) YK_LAUNCH(k_row_inv<float>, 512);
        else if (d.fft_df) YK_LAUNCH(k_row_inv<df32>, 512);
        else YK_LAUNCH(k_row_inv<double>, 512);
        break;
    default:
        if (d.f32) {
#define YK_CALL(W) YK_LAUNCH(k_interp32<W>, 256)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else if (d.fft_df) {
#define YK_CALL(W) YK_LAUNCH(k_interp_df<W>, 256)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else {
#define YK_CALL(W) YK_LAUNCH(k_interp<W>, 256)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        }
        break;
    }
#undef YK_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_build_mult_df(void *mult, const double *dfac, int M, double alpha,
                                 double delta, double dk, double period, cudaStream_t st)
{
    const int64_t total = (int64_t)(M + 1) * (2 * M + 1);
    k_build_mult<df32><<<(int)((total + 255) / 256), 256, 0, st>>>(static_cast<df32 *>(mult),
                                                                   dfac, M, alpha, delta, dk,
                                                                   period);
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
