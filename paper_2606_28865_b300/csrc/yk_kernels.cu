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

#include <algorithm>
#include <climits>

#include "yk_stages.cuh"

namespace yk {

namespace {

/* a point is accepted when it lies in the plan's box (closed) */
__device__ __forceinline__ bool in_box(const Geom &g, double x, double y)
{
    return x >= g.box[0] && x <= g.box[1] && y >= g.box[2] && y <= g.box[3];
}

/* legacy entry layout of the all-FP64 path: the grid coordinate t (double2) */
template <int W> __device__ __forceinline__ double2 pack_f64(double2 t) { return t; }
/* ----------------------------------------------------------------------------------------- */
/* binning                                                                                    */

/* Warp-aggregated atomics: consecutive points mostly fall into the same tile, so the lanes of a
 * warp that share a key make one atomic add (by their lowest lane) instead of one each.  Lanes
 * with valid == false take part in the match with a key of their own and do nothing. */
__device__ __forceinline__ void agg_count(int *cnt, int key, bool valid)
{
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(0xffffffffu, valid ? key : -1 - lane);
    if (valid && lane == __ffs(grp) - 1) atomicAdd(&cnt[key], __popc(grp));
}

/* reserve one slot per lane in cur[key]; returns the lane's offset within its key's range */
__device__ __forceinline__ int agg_reserve(int *cur, int key, bool valid)
{
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(0xffffffffu, valid ? key : -1 - lane);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(&cur[key], __popc(grp));
    base = __shfl_sync(grp, base, leader);
    return base + __popc(grp & ((1u << lane) - 1u));
}

/* the (up to four) tiles a source's w x w window touches; -1 where there is none */
template <int W> __device__ __forceinline__ void src_tiles(double2 t, const Geom &g, int tiles[4])
{
    const int lx = first_tap<W>(t.x), ly = first_tap<W>(t.y);
    const int ax0 = wrap(lx, g.n) / g.T, ax1 = wrap(lx + W - 1, g.n) / g.T;
    const int ay0 = wrap(ly, g.n) / g.T, ay1 = wrap(ly + W - 1, g.n) / g.T;
    tiles[0] = ay0 * g.nt + ax0;
    tiles[1] = ax1 != ax0 ? ay0 * g.nt + ax1 : -1;
    tiles[2] = ay1 != ay0 ? ay1 * g.nt + ax0 : -1;
    tiles[3] = (ay1 != ay0 && ax1 != ax0) ? ay1 * g.nt + ax1 : -1;
}

/* grid coordinates of a point and whether it lies in the plan's box (and so in the grid) */
__device__ __forceinline__ bool grid_coords(const Geom &g, double x, double y, double2 &t)
{
    t = make_double2((x - g.ox) * g.inv_h, (y - g.oy) * g.inv_h);
    return in_box(g, x, y) && t.x >= 0.0 && t.x < (double)g.n && t.y >= 0.0 && t.y < (double)g.n;
}

/* the block size of the binning kernels is a multiple of 32 and every lane reaches the warp
 * collectives (no early return) */
template <int W>
__global__ void k_bin_src_count(int64_t ns, const double *__restrict__ xs,
                                const double *__restrict__ ys, Geom g, double2 *__restrict__ src_t,
                                int *__restrict__ cnt, int *__restrict__ err)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = false;
    int tiles[4] = {-1, -1, -1, -1};
    if (j < ns) {
        double2 t;
        ok = grid_coords(g, xs[j], ys[j], t);
        if (!ok) {
            atomicOr(err, ERR_POINT_OUTSIDE);
            t = make_double2(-1.0, -1.0);
        } else {
            src_tiles<W>(t, g, tiles);
        }
        src_t[j] = t;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) agg_count(cnt, tiles[r], tiles[r] >= 0);
}

template <int W>
__global__ void k_bin_src_fill(int64_t ns, const double2 *__restrict__ src_t, Geom g,
                               const int *__restrict__ ptr, int *__restrict__ cur,
                               double2 *__restrict__ ent_t, int *__restrict__ ent_j, int joff)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int tiles[4] = {-1, -1, -1, -1};
    double2 t = make_double2(-1.0, -1.0);
    if (j < ns) t = src_t[j];
    if (t.x >= 0.0) src_tiles<W>(t, g, tiles);
    const double2 rec = pack_f64<W>(t);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const bool v = tiles[r] >= 0;
        const int off = agg_reserve(cur, tiles[r], v);
        if (v) {
            const int slot = ptr[tiles[r]] + off;
            ent_t[slot] = rec;
            ent_j[slot] = (int)j + joff;
        }
    }
}

__global__ void k_bin_trg_count(int64_t nt, const double *__restrict__ xt,
                                const double *__restrict__ yt, Geom g, double2 *__restrict__ tmp,
                                int *__restrict__ cnt, int *__restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int tile = -1;
    if (i < nt) {
        double2 t;
        if (!grid_coords(g, xt[i], yt[i], t)) {
            atomicOr(err, ERR_POINT_OUTSIDE);
            t = make_double2(-1.0, -1.0);
        } else {
            tile = ((int)t.y / g.Ti) * g.nti + (int)t.x / g.Ti;
        }
        tmp[i] = t;
    }
    agg_count(cnt, tile, tile >= 0);
}

template <int W>
__global__ void k_bin_trg_fill(int64_t nt, const double2 *__restrict__ tmp, Geom g,
                               const int *__restrict__ ptr, int *__restrict__ cur,
                               double2 *__restrict__ trg_t, int *__restrict__ trg_idx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double2 t = make_double2(-1.0, -1.0);
    if (i < nt) t = tmp[i];
    const bool v = t.x >= 0.0;
    const int tile = v ? ((int)t.y / g.Ti) * g.nti + (int)t.x / g.Ti : -1;
    const int off = agg_reserve(cur, tile, v);
    if (v) {
        const int slot = ptr[tile] + off;
        trg_t[slot] = pack_f64<W>(t);
        trg_idx[slot] = (int)i;
    }
}

/* ----------------------------------------------------------------------------------------- */
/* point preparation in fixed point (double-float and FP32C paths)                            */

/* T = t 2^44 rounded to the nearest integer, ties to even (one FMA, the only FP64 work per
 * coordinate; the rounding is done on the bits, since a double-to-int64 conversion costs several
 * FMAs of the FP64 pipe) */
__device__ __forceinline__ long long fixed_coord(double x, double A, double B)
{
    return round_even_ll(fma(x, A, B));
}

/* first tap l0 = ceil(t - w/2) and u = l0 - t + w/2 in [0, 1) from T = t 2^44, with u as an exact
 * FP32 pair: its 44 fraction bits split into 24 + 20 (both conversions exact), then renormalised */
template <int W> __device__ __forceinline__ void tap_frac(long long T, int &l0, float &uh, float &ul)
{
    const long long v = T - ((long long)W << (kFixBits - 1));            /* (t - w/2) 2^44 */
    const long long l = (v + ((1ll << kFixBits) - 1)) >> kFixBits;         /* ceil */
    const long long uf = (l << kFixBits) - v;                              /* u 2^44 */
    l0 = (int)l;
    const float hi = __int2float_rn((int)(uf >> 20)) * 5.9604644775390625e-8f;         /* 2^-24 */
    const float lo = __int2float_rn((int)(uf & 0xfffff)) * 5.684341886080801487e-14f;  /* 2^-44 */
    const df32 u = df_fast_two_sum(hi, lo); /* hi >= lo unless hi == 0 */
    uh = u.hi;
    ul = u.lo;
}

/* s = l0 - t = u - w/2 rounded to FP32 (the FP32C kernels' window offset) */
template <int W> __device__ __forceinline__ float frac_offset(float uh, float ul)
{
    const df32 s = df32(uh, 0.0f) + df32(-0.5f * W, 0.0f);
    return YK_FADD(s.hi, YK_FADD(s.lo, ul));
}

/* the tiles (up to four) a window with first taps (lx, ly) touches; -1 where there is none */
__device__ __forceinline__ void tap_tiles(int lx, int ly, int W, const Geom &g, int tiles[4])
{
    const int ax0 = wrap(lx, g.n) / g.T, ax1 = wrap(lx + W - 1, g.n) / g.T;
    const int ay0 = wrap(ly, g.n) / g.T, ay1 = wrap(ly + W - 1, g.n) / g.T;
    tiles[0] = ay0 * g.nt + ax0;
    tiles[1] = ax1 != ax0 ? ay0 * g.nt + ax1 : -1;
    tiles[2] = ay1 != ay0 ? ay1 * g.nt + ax0 : -1;
    tiles[3] = (ay1 != ay0 && ax1 != ax0) ? ay1 * g.nt + ax1 : -1;
}

/* a finite double (exponent field not all ones), tested on its bits */
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

/* prepare one point: false when it lies outside the box or the grid (the box test in the fixed
 * point of the coordinates, so no FP64 comparison is needed) */
template <int W>
__device__ __forceinline__ bool prep_point(const Geom &g, double x, double y, int2 &tap,
                                           float4 &fr, long long &Tx, long long &Ty)
{
    Tx = fixed_coord(x, g.A, g.Bx);
    Ty = fixed_coord(y, g.A, g.By);
    if (!(finite_bits(x) && finite_bits(y) && Tx >= g.tbox[0] && Tx <= g.tbox[1] &&
          Ty >= g.tbox[2] && Ty <= g.tbox[3] && Tx >= 0 && Tx < g.n44 && Ty >= 0 && Ty < g.n44))
        return false;
    tap_frac<W>(Tx, tap.x, fr.x, fr.y);
    tap_frac<W>(Ty, tap.y, fr.z, fr.w);
    return true;
}

template <int W, bool OWNER>
__global__ void k_prep_src_count(int64_t ns, const double *__restrict__ xs,
                                 const double *__restrict__ ys, Geom g, int2 *__restrict__ tap,
                                 float4 *__restrict__ frac, int *__restrict__ cnt,
                                 int *__restrict__ err)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int tiles[4] = {-1, -1, -1, -1};
    if (j < ns) {
        int2 tp;
        float4 fr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        long long Tx, Ty;
        if (!prep_point<W>(g, xs[j], ys[j], tp, fr, Tx, Ty)) {
            atomicOr(err, ERR_POINT_OUTSIDE);
            tp = make_int2(INT_MIN, 0);
        } else if (OWNER) {
            tiles[0] = (wrap(tp.y, g.n) / g.T) * g.nt + wrap(tp.x, g.n) / g.T;
        } else {
            tap_tiles(tp.x, tp.y, W, g, tiles);
        }
        tap[j] = tp;
        frac[j] = fr;
    }
#pragma unroll
    for (int r = 0; r < (OWNER ? 1 : 4); ++r) agg_count(cnt, tiles[r], tiles[r] >= 0);
}

template <int W, bool OWNER>
__global__ void k_prep_src_fill(int64_t ns, const int2 *__restrict__ tap,
                                const float4 *__restrict__ frac, Geom g,
                                const int *__restrict__ ptr, int *__restrict__ cur,
                                double2 *__restrict__ ent_t, int *__restrict__ ent_j, int joff)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int tiles[4] = {-1, -1, -1, -1};
    int2 tp = make_int2(INT_MIN, 0);
    if (j < ns) tp = tap[j];
    int4 rec = make_int4(0, 0, 0, 0);
    if (tp.x != INT_MIN) {
        const float4 fr = frac[j];
        const float sx = frac_offset<W>(fr.x, fr.y), sy = frac_offset<W>(fr.z, fr.w);
        if (OWNER) {
            const int wx = wrap(tp.x, g.n), wy = wrap(tp.y, g.n);
            tiles[0] = (wy / g.T) * g.nt + wx / g.T;
            rec = make_int4((wy % g.T) * owner_pitch(g.T, W) + wx % g.T, (int)j + joff,
                            __float_as_int(sx), __float_as_int(sy));
        } else {
            tap_tiles(tp.x, tp.y, W, g, tiles);
            rec = make_int4(tp.x, tp.y, __float_as_int(sx), __float_as_int(sy));
        }
    }
#pragma unroll
    for (int r = 0; r < (OWNER ? 1 : 4); ++r) {
        const bool v = tiles[r] >= 0;
        const int off = agg_reserve(cur, tiles[r], v);
        if (v) {
            const int slot = ptr[tiles[r]] + off;
            *reinterpret_cast<int4 *>(ent_t + slot) = rec;
            ent_j[slot] = (int)j + joff;
        }
    }
}

/* targets: tap4 = (l0x, l0y, tile of the cell floor(t), 0), tile -1 outside the box */
template <int W>
__global__ void k_prep_trg_count(int64_t nt, const double *__restrict__ xt,
                                 const double *__restrict__ yt, Geom g, int4 *__restrict__ tap4,
                                 float4 *__restrict__ frac, int *__restrict__ cnt,
                                 int *__restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int tile = -1;
    if (i < nt) {
        int2 tp = make_int2(0, 0);
        float4 fr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        long long Tx, Ty;
        if (!prep_point<W>(g, xt[i], yt[i], tp, fr, Tx, Ty)) {
            atomicOr(err, ERR_POINT_OUTSIDE);
        } else {
            tile = ((int)(Ty >> kFixBits) / g.Ti) * g.nti + (int)(Tx >> kFixBits) / g.Ti;
        }
        tap4[i] = make_int4(tp.x, tp.y, tile, 0);
        frac[i] = fr;
    }
    agg_count(cnt, tile, tile >= 0);
}

/* targets grouped by the tile of their cell: records (lx, ly, sx, sy) and, when trg_frac is
 * given, the window arguments in the same order.  Each thread takes kFillPer targets (a block's
 * targets strided by the block size) and issues their slot reservations back to back, so the
 * atomics' latencies overlap (uniformly spread targets rarely share a tile within a warp). */
constexpr int kFillPer = 4;

template <int W>
__global__ void k_prep_trg_fill(int64_t nt, const int4 *__restrict__ tap4,
                                const float4 *__restrict__ frac, const int *__restrict__ ptr,
                                int *__restrict__ cur, double2 *__restrict__ trg_t,
                                float4 *__restrict__ trg_frac, int *__restrict__ trg_idx)
{
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kFillPer + threadIdx.x;
    int4 tp[kFillPer];
    float4 fr[kFillPer];
#pragma unroll
    for (int k = 0; k < kFillPer; ++k) {
        const int64_t i = i0 + (int64_t)k * blockDim.x;
        tp[k] = i < nt ? tap4[i] : make_int4(0, 0, -1, 0);
        if (tp[k].z >= 0) fr[k] = frac[i];
    }
    /* agg_reserve split in two passes: all groups' atomics first, then the broadcasts */
    const int lane = threadIdx.x & 31;
    unsigned grp[kFillPer];
    int base[kFillPer], off[kFillPer];
#pragma unroll
    for (int k = 0; k < kFillPer; ++k) {
        const bool v = tp[k].z >= 0;
        grp[k] = __match_any_sync(0xffffffffu, v ? tp[k].z : -1 - lane);
        base[k] = 0;
        if (v && lane == __ffs(grp[k]) - 1) base[k] = atomicAdd(&cur[tp[k].z], __popc(grp[k]));
    }
#pragma unroll
    for (int k = 0; k < kFillPer; ++k)
        off[k] = __shfl_sync(grp[k], base[k], __ffs(grp[k]) - 1) +
                 __popc(grp[k] & ((1u << lane) - 1u));
#pragma unroll
    for (int k = 0; k < kFillPer; ++k) {
        if (tp[k].z < 0) continue;
        const int64_t i = i0 + (int64_t)k * blockDim.x;
        const int slot = ptr[tp[k].z] + off[k];
        *reinterpret_cast<int4 *>(trg_t + slot) =
            make_int4(tp[k].x, tp[k].y, __float_as_int(frac_offset<W>(fr[k].x, fr[k].y)),
                      __float_as_int(frac_offset<W>(fr[k].z, fr[k].w)));
        if (trg_frac) trg_frac[slot] = fr[k];
        trg_idx[slot] = (int)i;
    }
}

/* Target binning by chunk histograms (no global atomics): CTA c prepares the targets of its chunk
 * and counts them per tile in shared memory, its row of counts goes to hist[c][.]; a column pass
 * turns each tile's counts into exclusive offsets over the chunks (and the tile totals); after the
 * scan of the totals, CTA c scatters its targets from per-tile cursors ptr[t] + hist[c][t] held in
 * shared memory.  Uniformly spread targets make per-target global atomics contend on few
 * addresses; shared-memory counters do not.  Used while the tiles' counters fit in shared memory
 * (kHistTiles). */
constexpr int kHistTiles = 16384;
constexpr int kHistThreads = 1024;

template <int W>
__global__ void __launch_bounds__(kHistThreads)
    k_trg_hist(int64_t nt, int64_t chunk, const double *__restrict__ xt,
               const double *__restrict__ yt, Geom g, int4 *__restrict__ tap4,
               float4 *__restrict__ frac, int *__restrict__ hist, int *__restrict__ err)
{
    extern __shared__ int sh_cnt[];
    const int ntiles = g.nti * g.nti;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) sh_cnt[t] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(nt, i0 + chunk);
    bool bad = false;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        int2 tp = make_int2(0, 0);
        float4 fr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        long long Tx, Ty;
        int tile = -1;
        if (prep_point<W>(g, xt[i], yt[i], tp, fr, Tx, Ty)) {
            tile = ((int)(Ty >> kFixBits) / g.Ti) * g.nti + (int)(Tx >> kFixBits) / g.Ti;
            atomicAdd(&sh_cnt[tile], 1);
        } else {
            bad = true;
        }
        tap4[i] = make_int4(tp.x, tp.y, tile, 0);
        frac[i] = fr;
    }
    if (bad) atomicOr(err, ERR_POINT_OUTSIDE);
    __syncthreads();
    int *row = hist + (int64_t)blockIdx.x * ntiles;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) row[t] = sh_cnt[t];
}

/* per tile t: hist[c][t] <- sum of hist[c'][t] over c' < c (in place), cnt[t] <- the total.  A
 * CTA takes 32 consecutive tiles: their counts of every chunk are read row by row (coalesced)
 * into shared memory, one thread per tile scans its column there, and the offsets are written
 * back the same way.  Needs nchunks * 33 ints of shared memory. */
__global__ void __launch_bounds__(256)
    k_hist_columns(int *__restrict__ hist, int nchunks, int ntiles, int *__restrict__ cnt)
{
    extern __shared__ int sh_col[]; /* [nchunks][33] */
    const int t0 = blockIdx.x * 32;
    /* eight loads in flight per thread before their stores */
    for (int idx0 = threadIdx.x; idx0 < nchunks * 32; idx0 += 8 * blockDim.x) {
        int v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = idx0 + u * blockDim.x, c = idx >> 5, j = idx & 31;
            v[u] = (idx < nchunks * 32 && t0 + j < ntiles) ? hist[(int64_t)c * ntiles + t0 + j] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = idx0 + u * blockDim.x;
            if (idx < nchunks * 32) sh_col[(idx >> 5) * 33 + (idx & 31)] = v[u];
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int run = 0;
        for (int c = 0; c < nchunks; ++c) {
            const int v = sh_col[c * 33 + threadIdx.x];
            sh_col[c * 33 + threadIdx.x] = run;
            run += v;
        }
        if (t0 + threadIdx.x < ntiles) cnt[t0 + threadIdx.x] = run;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nchunks * 32; idx += blockDim.x) {
        const int c = idx >> 5, j = idx & 31;
        if (t0 + j < ntiles) hist[(int64_t)c * ntiles + t0 + j] = sh_col[c * 33 + j];
    }
}

template <int W>
__global__ void __launch_bounds__(kHistThreads)
    k_trg_scatter(int64_t nt, int64_t chunk, const int4 *__restrict__ tap4,
                  const float4 *__restrict__ frac, const int *__restrict__ hist, int ntiles,
                  const int *__restrict__ ptr, double2 *__restrict__ trg_t,
                  float4 *__restrict__ trg_frac, int *__restrict__ trg_idx)
{
    extern __shared__ int sh_cur[];
    const int *row = hist + (int64_t)blockIdx.x * ntiles;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) sh_cur[t] = ptr[t] + row[t];
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(nt, i0 + chunk);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int4 tp = tap4[i];
        if (tp.z < 0) continue;
        const float4 fr = frac[i];
        const int slot = atomicAdd(&sh_cur[tp.z], 1);
        *reinterpret_cast<int4 *>(trg_t + slot) =
            make_int4(tp.x, tp.y, __float_as_int(frac_offset<W>(fr.x, fr.y)),
                      __float_as_int(frac_offset<W>(fr.z, fr.w)));
        if (trg_frac) trg_frac[slot] = fr;
        trg_idx[slot] = (int)i;
    }
}

/* exclusive scan of cnt[0..count) into ptr[0..count] in three passes over blocks of kScanBlock
 * elements: block sums into bsum, a scan of the block sums (one CTA), then each block adds its
 * offset.  bsum holds ceil(count / kScanBlock) ints. */
constexpr int kScanBlock = 4096;

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    const int excl = x - v + (wid > 0 ? warp_tot[wid - 1] : 0);
    __syncthreads();
    return excl;
}

/* pass 1 (blockDim 1024, 4 elements per thread): local exclusive prefix into ptr, block total */
__global__ void __launch_bounds__(1024) k_scan_local(const int *__restrict__ cnt,
                                                     int *__restrict__ ptr, int count,
                                                     int *__restrict__ bsum)
{
    __shared__ int wt[32];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 4;
    int v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < count ? cnt[base + k] : 0;
        s += v[k];
    }
    int total = 0;
    int run = block_exclusive_scan(s, wt, total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < count) ptr[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

/* pass 2 (one CTA): exclusive scan of the block sums in place; ptr[count] = grand total */
__global__ void __launch_bounds__(1024) k_scan_sums(int *__restrict__ bsum, int nb,
                                                    int *__restrict__ ptr, int count)
{
    __shared__ int wt[32];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int i = b0 + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        int total = 0;
        const int ex = block_exclusive_scan(v, wt, total);
        if (i < nb) bsum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) ptr[count] = carry;
}

/* pass 3: add each block's offset */
__global__ void __launch_bounds__(1024) k_scan_add(int *__restrict__ ptr, int count,
                                                   const int *__restrict__ bsum)
{
    const int add = bsum[blockIdx.x];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < count) ptr[base + k] += add;
}

/* the whole scan in one CTA for counts up to kScanSingle: blocks of kScanBlock elements in turn,
 * each scanned as in pass 1 and offset by the running total (one launch instead of three; beyond
 * two blocks the serial blocks cost more than the two launches saved) */
constexpr int kScanSingle = 2 * kScanBlock;

__global__ void __launch_bounds__(1024) k_scan_single(const int *__restrict__ cnt,
                                                      int *__restrict__ ptr, int count)
{
    __shared__ int wt[32];
    int carry = 0;
    for (int b0 = 0; b0 < count; b0 += kScanBlock) {
        const int base = b0 + threadIdx.x * 4;
        int v[4], s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = base + k < count ? cnt[base + k] : 0;
            s += v[k];
        }
        int total = 0;
        int run = carry + block_exclusive_scan(s, wt, total);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k < count) ptr[base + k] = run;
            run += v[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) ptr[count] = carry;
}

/* heavy-first processing order of the tiles: tiles bucketed by floor(log2(entries)) and listed
 * from the fullest bucket down, so that the costly tiles start first and the short ones fill the
 * tail (the order inside a bucket does not affect any result).  scratch: 80 ints, zeroed. */
__device__ __forceinline__ int tile_bucket(const int *ptr, int t)
{
    const int c = ptr[t + 1] - ptr[t];
    return c > 0 ? 32 - __clz(c) : 0;
}

__global__ void k_order_hist(const int *__restrict__ ptr, int ntiles, int *__restrict__ scratch)
{
    __shared__ int h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x)
        atomicAdd(&h[tile_bucket(ptr, t)], 1);
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&scratch[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_order_base(int *__restrict__ scratch)
{
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 32; b >= 0; --b) {
            scratch[40 + b] = run; /* first position of bucket b */
            run += scratch[b];
        }
    }
}

__global__ void k_order_fill(const int *__restrict__ ptr, int ntiles, int *__restrict__ scratch,
                             int *__restrict__ order)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool v = t < ntiles;
    const int b = v ? tile_bucket(ptr, t) : 0;
    const int off = agg_reserve(scratch + 40, b, v); /* scratch[40+b] doubles as the cursor */
    if (v) order[off] = t;
}

/* the same order in one CTA for up to kOrderSingle tiles (one launch instead of a memset and the
 * three kernels above): bucket counts and then cursors in shared memory, warp-aggregated adds.
 * Up to 8,192 tiles this saves 2-3 us; at 15,000-22,500 tiles the one CTA took 2-7 us longer
 * than the three grid-wide kernels on B300. */
constexpr int kOrderSingle = 8192;

__global__ void __launch_bounds__(1024)
    k_order_single(const int *__restrict__ ptr, int ntiles, int *__restrict__ order)
{
    __shared__ int h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0;
    __syncthreads();
    /* the trip count is the same for every thread: the warp-wide match sees all 32 lanes */
    for (int t0 = 0; t0 < ntiles; t0 += blockDim.x) {
        const int t = t0 + (int)threadIdx.x;
        const bool v = t < ntiles;
        agg_count(h, v ? tile_bucket(ptr, t) : 0, v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 32; b >= 0; --b) { /* the fullest bucket first */
            const int c = h[b];
            h[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int t0 = 0; t0 < ntiles; t0 += blockDim.x) {
        const int t = t0 + (int)threadIdx.x;
        const bool v = t < ntiles;
        const int off = agg_reserve(h, v ? tile_bucket(ptr, t) : 0, v);
        if (v) order[off] = t;
    }
}

/* Shared-memory layout of the window tables in the window kernel.  Per piece, the coefficients
 * of order <= 2 as double-float pairs and those of order >= 3 as FP32 values: over a piece (1/64
 * of a cell) the window's k-th coefficient is at most 4e-3, 2.3e-5, 7.3e-8, 2.6e-10 of its peak
 * for k = 1..4 at w = 12, so the orders >= 3 carry ~1e-7 of the value and an FP32 rounding of
 * them costs ~1e-14, far below the tables' own ~1e-13.  A row holds the W taps padded with zeros
 * to 4 ceil(W / 4) (the kernel's four lanes per point read ceil(W / 4) taps each); the piece
 * strides are odd in words, so the pieces that the lanes of a warp read spread over the banks. */
__host__ __device__ constexpr int win_row(int W) { return 4 * ((W + 3) / 4); }
/* coefficients of orders 0 .. min(D, 2) (double-float) and 3 .. D (FP32) */
__host__ __device__ constexpr int win_ndf(int D) { return (D < 2 ? D : 2) + 1; }
__host__ __device__ constexpr int win_nf(int D) { return D < 3 ? 0 : D - 2; }
__host__ __device__ constexpr int win_stride_df(int W, int D) { return win_ndf(D) * win_row(W) + 1; }
__host__ __device__ constexpr int win_stride_f(int W, int D) { return win_nf(D) * win_row(W) + 1; }

/* TPL window values (taps a0 .. a0 + TPL - 1) of one coordinate by Horner on the piece's
 * polynomials (compile-time degree D; the lane's taps interleaved: TPL independent chains): the
 * orders >= 3 in FP32 with the argument's high word, then c_2 + q x, c_1 + p x and c_0 + p x as
 * fused double-float multiply-adds (exact product terms added to c_k by two-sum) whose pairs are
 * left unnormalised between the steps (each keeps the exact error of its high words) and
 * normalised once at the end.  Taps past the window (a >= W) read the zero pad of the row. */
template <int TPL, int D, int WE>
__device__ __forceinline__ void windows_taps(const df32 *c, const float *cf, int a0, df32 x,
                                             df32 (&p)[TPL])
{
    if (D >= 3) {
        float q[TPL];
#pragma unroll
        for (int j = 0; j < TPL; ++j) q[j] = cf[(D - 3) * WE + a0 + j];
#pragma unroll
        for (int k = D - 1; k >= 3; --k)
#pragma unroll
            for (int j = 0; j < TPL; ++j) q[j] = fmaf(q[j], x.hi, cf[(k - 3) * WE + a0 + j]);
#pragma unroll
        for (int j = 0; j < TPL; ++j) p[j] = df_mul_add_lazy(c[2 * WE + a0 + j], q[j], x);
#pragma unroll
        for (int k = 1; k >= 0; --k)
#pragma unroll
            for (int j = 0; j < TPL; ++j) p[j] = df_mul_add_lazy(c[k * WE + a0 + j], p[j], x);
    } else {
#pragma unroll
        for (int j = 0; j < TPL; ++j) p[j] = c[D * WE + a0 + j];
#pragma unroll
        for (int k = D - 1; k >= 0; --k)
#pragma unroll
            for (int j = 0; j < TPL; ++j) p[j] = df_mul_add_lazy(c[k * WE + a0 + j], p[j], x);
    }
#pragma unroll
    for (int j = 0; j < TPL; ++j) p[j] = df_fast_two_sum(p[j].hi, p[j].lo);
}

/* double-float window values per point (see launch_frac_windows_df): four lanes per point, each
 * evaluating TPL = ceil(W / 4) consecutive taps of both coordinates on the kWinPieces-piece
 * per-tap polynomials staged in shared memory (piece h of u = l0 - t + w/2 in [0, 1) is
 * [h/P, (h+1)/P), argument x = 2P u - 2h - 1).  The four lanes of a point read one piece's
 * coefficients at consecutive taps, so a half-warp reads only four pieces; the argument comes
 * from the point's exact FP32 pair u (no FP64 arithmetic). */
template <int W>
__global__ void __launch_bounds__(256)
    k_frac_windows_df(int64_t n, const float4 *__restrict__ frac, const int *__restrict__ count,
                      const float2 *__restrict__ coef, int deriv, int64_t pitch,
                      float2 *__restrict__ out, const int *__restrict__ idx, int64_t idx_lim)
{
    constexpr int NP = kWinPieces, D = kPieceDeg[W], WE = win_row(W);
    constexpr int TPL = (W + 3) / 4;
    constexpr int S0 = win_stride_df(W, D), S1 = win_stride_df(W, D - 1);
    constexpr int F0 = win_stride_f(W, D), F1 = win_stride_f(W, D - 1);
    extern __shared__ __align__(16) unsigned char sm[];
    df32 *cw = reinterpret_cast<df32 *>(sm);
    const int md = NP * S0 + (deriv ? NP * S1 : 0);
    float *cf = reinterpret_cast<float *>(cw + md);
    const int mf = NP * F0 + (deriv ? NP * F1 : 0);
    /* the tables (window, then derivative) in the padded layout; the pad cells are zero */
    for (int i = threadIdx.x; i < md; i += blockDim.x) cw[i] = df32(0.0f, 0.0f);
    for (int i = threadIdx.x; i < mf; i += blockDim.x) cf[i] = 0.0f;
    __syncthreads();
    const int n0 = NP * (D + 1) * W, n1 = deriv ? NP * D * W : 0;
    for (int i = threadIdx.x; i < n0 + n1; i += blockDim.x) {
        const bool dv = i >= n0;
        const int j = dv ? i - n0 : i, rows = dv ? D : D + 1;
        const int a = j % W, hk = j / W, h = hk / rows, k = hk - h * rows;
        if (k <= 2)
            cw[(dv ? NP * S0 : 0) + h * (dv ? S1 : S0) + k * WE + a] = df32(coef[i].x, coef[i].y);
        else
            cf[(dv ? NP * F0 : 0) + h * (dv ? F1 : F0) + (k - 3) * WE + a] = coef[i].x;
    }
    __syncthreads();
    const int64_t nv = count ? min(n, (int64_t)*count) : n;
    const int stride = deriv ? 4 * W : 2 * W;
    const int q = threadIdx.x & 3, a0 = q * TPL; /* this lane's first tap */
    /* the argument x = 2P u - (2h + 1) of u = (uh, ul): 2P uh and the integer are exact in FP32,
     * so one two-sum gives their difference exactly; 2P ul is added to its low word */
    auto piece_arg = [&](float uh, float ul, int &h) {
        h = max(0, min(NP - 1, __float2int_rz(uh * (float)NP)));
        const df32 s = df32(YK_FMUL(2.0f * NP, uh), 0.0f) + df32(-(float)(2 * h + 1), 0.0f);
        return df_fast_two_sum(s.hi, YK_FADD(s.lo, YK_FMUL(2.0f * NP, ul)));
    };
    /* grid-stride over groups of points (blockDim / 4 per CTA), tables staged once per CTA */
    for (int64_t base = (int64_t)blockIdx.x * (blockDim.x >> 2); base < nv;
         base += (int64_t)gridDim.x * (blockDim.x >> 2)) {
        const int64_t i = base + (threadIdx.x >> 2);
        bool ok = i < nv;
        float4 fr = make_float4(0.5f, 0.0f, 0.5f, 0.0f);
        if (ok && idx) { /* point i is frac[idx[i]]; indices >= idx_lim get no values */
            const int k = idx[i];
            ok = k < idx_lim;
            if (ok) fr = frac[k];
        } else if (ok) {
            fr = frac[i];
        }
        if (!ok) continue; /* no warp-wide operation follows */
        /* part pq (W values) of point i: value-major planes (value k at k * pitch + i) or the
         * point-major record (values i * stride + pq W + a) */
        auto emit = [&](int pq, const df32 (&v)[TPL]) {
#pragma unroll
            for (int j = 0; j < TPL; ++j) {
                const int a = a0 + j;
                if (a < W) {
                    const float2 val = make_float2(v[j].hi, v[j].lo);
                    if (pitch) out[(int64_t)(pq * W + a) * pitch + i] = val;
                    else out[(size_t)i * stride + pq * W + a] = val;
                }
            }
        };
        int hx, hy;
        const df32 ax = piece_arg(fr.x, fr.y, hx), ay = piece_arg(fr.z, fr.w, hy);
        df32 p[TPL];
        windows_taps<TPL, D, WE>(cw + hy * S0, cf + hy * F0, a0, ay, p);
        emit(0, p);
        windows_taps<TPL, D, WE>(cw + hx * S0, cf + hx * F0, a0, ax, p);
        emit(1, p);
        if (deriv) {
            const df32 *cwd = cw + NP * S0;
            const float *cfd = cf + NP * F0;
            windows_taps<TPL, D - 1, WE>(cwd + hy * S1, cfd + hy * F1, a0, ay, p);
            emit(2, p);
            windows_taps<TPL, D - 1, WE>(cwd + hx * S1, cfd + hx * F1, a0, ax, p);
            emit(3, p);
        }
    }
}

/* ----------------------------------------------------------------------------------------- */
/* per-stage kernels: one CTA per work item                                                   */

template <int W> __global__ void __launch_bounds__(256) k_spread(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_spread64<W>(d, blockIdx.x, sm);
}
template <int W> __global__ void __launch_bounds__(32 * kOwnerCopies, 3) k_spread_owner32(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_spread_owner32<W, false>(d, blockIdx.x, sm);
}
template <int W>
__global__ void __launch_bounds__(32 * kOwnerCopies, 2) k_spread_owner32_dip(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_spread_owner32<W, true>(d, blockIdx.x, sm);
}
template <int W> __global__ void __launch_bounds__(32 * kOwnerCopies, 3) k_spread_owner_df(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_spread_owner_df<W, false>(d, blockIdx.x, sm);
}
/* with dipole sources: twice the window values per source (2 CTAs per SM by shared memory) */
template <int W>
__global__ void __launch_bounds__(32 * kOwnerCopies, 2) k_spread_owner_df_dip(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_spread_owner_df<W, true>(d, blockIdx.x, sm);
}
template <int W> __global__ void __launch_bounds__(256) k_interp_df(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_interp_df<W>(d, blockIdx.x, sm);
}
template <typename R>
__global__ void __launch_bounds__(kRowThreads, 1024 / kRowThreads) k_row_fwd(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_row_fwd<R>(d, blockIdx.x, sm);
}
template <typename R>
__global__ void __launch_bounds__(kColumnThreads, 1024 / kColumnThreads) k_columns(Inst d)
{
    extern __shared__ __align__(16) unsigned char sm[];
    st_columns<R>(d, blockIdx.x, sm);
}
template <typename R>
__global__ void __launch_bounds__(kRowThreads, 1024 / kRowThreads) k_row_inv(Inst d)
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
/* radial multiplier at |k| from an equispaced table tab[i] = G(i H) by 10-point Lagrange
 * interpolation on the nearest nodes (truncated kernel) */
__device__ double table_interp(const double *__restrict__ tab, int ntab, double H, double k)
{
    constexpr int NP = 10;
    int i0 = (int)floor(k / H) - NP / 2 + 1;
    i0 = max(0, min(i0, ntab - NP));
    const double x = k / H - (double)i0;
    double pre[NP + 1], suf[NP + 1];
    pre[0] = 1.0;
    for (int j = 0; j < NP; ++j) pre[j + 1] = pre[j] * (x - (double)j);
    suf[NP] = 1.0;
    for (int j = NP - 1; j >= 0; --j) suf[j] = suf[j + 1] * (x - (double)j);
    /* weights 1 / prod_{m != j} (j - m) = (-1)^(NP-1-j) / (j! (NP-1-j)!) */
    double fact[NP];
    fact[0] = 1.0;
    for (int j = 1; j < NP; ++j) fact[j] = fact[j - 1] * (double)j;
    double sum = 0.0;
    for (int j = 0; j < NP; ++j) {
        const double den = fact[j] * fact[NP - 1 - j] * (((NP - 1 - j) & 1) ? -1.0 : 1.0);
        sum += tab[i0 + j] * pre[j] * suf[j + 1] / den;
    }
    return sum;
}

/* multiplier table (M+1) x (2M+1): Ghat(k)/P^2 times the window deconvolution of both axes, in
 * FP64 and rounded once to the table's type.  Ghat is exp(-delta(alpha^2+k^2))/(alpha^2+k^2)
 * (Section 5.1, eq. sh), or, for the truncated kernel, interpolated from tab. */
template <typename R>
__global__ void k_build_mult(R *__restrict__ mult, const double *__restrict__ dfac, int M,
                             double alpha, double delta, double dk, double period,
                             const double *__restrict__ tab, int ntab, double H)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t w = 2 * M + 1;
    if (i >= (int64_t)(M + 1) * w) return;
    const int kx = (int)(i / w), my = (int)(i - (int64_t)kx * w) - M;
    const double k2 = dk * dk * ((double)kx * kx + (double)my * my);
    const double s = alpha * alpha + k2;
    const double gh = tab ? table_interp(tab, ntab, H, sqrt(k2)) : exp(-delta * s) / s;
    mult[i] = (R)(gh / (period * period) * dfac[kx] * dfac[my < 0 ? -my : my]);
}

/* Fourier transform of the truncated history kernel G_T = G_H chi (chi = 1 for r <= R0, a smooth
 * step to 0 on [R0, R1]) at k_i = i H, one warp per table entry:
 *   Ghat_T(k) = [exp(-delta(alpha^2+k^2)) + R0 k J1(k R0) K0(alpha R0) - R0 alpha J0(k R0)
 *                K1(alpha R0)] / (alpha^2 + k^2)  +  sum_q f_q J0(k r_q),
 * the first term the exact transform of G_H on the disc r <= R0 (where G_H = K0(alpha r)/(2 pi)
 * minus a local part supported well inside it), the sum a quadrature of the transition
 * int_R0^R1 K0(alpha r) chi(r) J0(k r) r dr with weights folded into f_q. */
__global__ void k_trunc_table(double *__restrict__ tab, int ntab, double H, double alpha,
                              double delta, double R0, double k0a, double k1a,
                              const double2 *__restrict__ nodes, int nq)
{
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= ntab) return; /* whole warps exit together */
    const double k = (double)warp * H;
    double sum = 0.0;
    for (int q = lane; q < nq; q += 32) {
        const double2 nd = nodes[q];
        sum += nd.y * j0(k * nd.x);
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
        const double s = alpha * alpha + k * k;
        const double disc = (exp(-delta * s) + R0 * k * j1(k * R0) * k0a -
                             R0 * alpha * j0(k * R0) * k1a) / s;
        tab[warp] = disc + sum;
    }
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

int rows_per_item(int n, bool f32, bool fill_sms)
{
    const int bytes_per_row = (n / 2) * (f32 ? 8 : 16);
    int r = kRowItemBytes / bytes_per_row;
    r = r < 1 ? 1 : (r > 16 ? 16 : r);
    if (!fill_sms) return r;
    /* FP32 rows (at most 14,400 complex values, 115 KB): at most two per item, so that more CTAs
     * hide the latency of the fold's loads (row passes -7..14% against three to six rows per item
     * on B300 at n = 1,600 and 2,880) */
    if (f32 && r > 2) r = 2;
    /* a launch of its own: no more rows than leave 1024 / kRowThreads work items (the CTAs that
     * share an SM at <= 64 registers) per SM of a 148-SM part (FP32 rows of small grids would
     * otherwise fit 15 or 16 to a CTA and leave SMs idle: 107 CTAs at n = 1600); the batch
     * kernel, which runs many instances' items at once, keeps the larger items (fewer items,
     * less per-item overhead) */
    const int per_sm = 1024 / kRowThreads;
    const int fill = (n + per_sm * 148 - 1) / (per_sm * 148);
    return r < fill ? r : (fill < 1 ? 1 : fill);
}

int stage_items(const Inst &d, int stage)
{
    switch (stage) {
    case ST_SPREAD: return d.g.nt * d.g.nt;
    case ST_INTERP: return d.g.nti * d.g.nti;
    case ST_ROW_FWD:
    case ST_ROW_INV: return (d.n + d.rows - 1) / d.rows;
    default: return d.M + 1;
    }
}

int stage_smem(const Inst &d, int stage)
{
    const int T = d.g.T, W = d.g.w;
    /* window coefficients (and, with dipoles, the derivative's) staged by the FP64 kernels */
    const int ncoef = (d.wdeg + 1) * W + (d.dip ? d.wdeg * W : 0);
    const int win_bytes = d.win ? (int)sizeof(double) * ncoef : 0;
    const int SW = d.dip ? 4 * W : 2 * W; /* window values kept per spread entry */
    const int c = d.f32 ? 8 : 16;          /* bytes of a complex value */
    switch (stage) {
    case ST_SPREAD:
        if (d.f32) /* FP32C owner-tile spread: padded copies of (hi, lo) pairs per warp */
            return (int)(sizeof(float2) * d.spread_warps * owner_copy_cells(T, W) +
                         sizeof(float) * d.spread_warps * d.spread_batch * (SW + 1) +
                         sizeof(int) * d.spread_warps * d.spread_batch +
                         (d.dip ? sizeof(float) * ncoef : 0));
        if (d.fft_df) /* double-float owner-tile spread */
            return (int)(sizeof(df32) * d.spread_warps *
                             (owner_copy_cells(T, W) +
                              d.spread_batch * (owner_batch_stride(W, d.dip != 0) + 1)) +
                         sizeof(int) * d.spread_warps * d.spread_batch);
        return (int)(sizeof(unsigned long long) * T * T + win_bytes);
    case ST_ROW_FWD:
    case ST_ROW_INV: return c * d.rows * (d.n / 2);
    case ST_COLUMNS: return c * d.n;
    default: {
        const int nw = (d.wdeg + 1) * W; /* interpolation stages the window only */
        const int Ti = d.g.Ti;
        if (d.fft_df) return 2 * 8 * (Ti + W) * halo_pair_pitch(Ti + W); /* the paired halo */
        return d.f32 ? 4 * 4 * (Ti + W) * halo_quad_pitch(Ti + W) /* the four-copy halo */
                     : 8 * (Ti + W) * (Ti + W) + (d.win ? (int)sizeof(double) * nw : 0);
    }
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

/* exclusive scan of cnt into ptr; cur (>= ceil(count / kScanBlock) ints) is scratch and is left
 * zeroed for the fill pass.  Up to kScanSingle counts: one CTA. */
cudaError_t launch_scan(const int *cnt, int *ptr, int count, int *cur, cudaStream_t st)
{
    if (count <= 0) return cudaMemsetAsync(ptr, 0, sizeof(int), st);
    const int nb = (count + kScanBlock - 1) / kScanBlock;
    if (count <= kScanSingle) {
        k_scan_single<<<1, 1024, 0, st>>>(cnt, ptr, count);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemsetAsync(cur, 0, sizeof(int) * nb, st);
        return e;
    }
    k_scan_local<<<nb, 1024, 0, st>>>(cnt, ptr, count, cur);
    k_scan_sums<<<1, 1024, 0, st>>>(cur, nb, ptr, count);
    k_scan_add<<<nb, 1024, 0, st>>>(ptr, count, cur);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(cur, 0, sizeof(int) * nb, st);
    return e;
}

cudaError_t launch_bin_sources(const Geom &g, int64_t ns, const double *xs, const double *ys,
                               int64_t nd, const double *xd, const double *yd, double2 *src_t,
                               int *tile_cnt, int *tile_ptr, int *tile_cur, double2 *ent_t,
                               int *ent_j, int *err, cudaStream_t st)
{
    const int ntiles = g.nt * g.nt;
    cudaError_t e = cudaMemsetAsync(tile_cnt, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(tile_cur, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    /* the two point sets: charges, then dipoles (index offset ns) */
    const int64_t cnt[2] = {ns, nd};
    const double *px[2] = {xs, xd}, *py[2] = {ys, yd};
    double2 *pt[2] = {src_t, src_t + ns};
    for (int k = 0; k < 2; ++k) {
        if (cnt[k] <= 0) continue;
        const int blocks = (int)((cnt[k] + 255) / 256);
#define YK_CALL(W)                                                                              \
    k_bin_src_count<W><<<blocks, 256, 0, st>>>(cnt[k], px[k], py[k], g, pt[k], tile_cnt, err)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    if ((e = launch_scan(tile_cnt, tile_ptr, ntiles, tile_cur, st)) != cudaSuccess) return e;
    for (int k = 0; k < 2; ++k) {
        if (cnt[k] <= 0) continue;
        const int blocks = (int)((cnt[k] + 255) / 256);
        const int joff = k ? (int)ns : 0;
#define YK_CALL(W)                                                                              \
    k_bin_src_fill<W><<<blocks, 256, 0, st>>>(cnt[k], pt[k], g, tile_ptr, tile_cur, ent_t, ent_j, \
                                              joff)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    return cudaGetLastError();
}

__global__ void k_pack_wnu(int64_t nd, const double *__restrict__ wd, const double *__restrict__ nx,
                           const double *__restrict__ ny, double2 *__restrict__ wnu)
{
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d < nd) wnu[d] = make_double2(wd[d] * nx[d], wd[d] * ny[d]);
}

cudaError_t launch_frac_windows_df(const Geom &g, int64_t n, const float4 *frac, const int *count,
                                   const float2 *coef, int deg, bool deriv, float2 *out,
                                   cudaStream_t st, int64_t pitch, const int *idx, int64_t idx_lim)
{
    if (n <= 0) return cudaSuccess;
    if (g.w < 2 || g.w > 16 || deg != kPieceDeg[g.w]) return cudaErrorInvalidValue;
    /* coefficient tables in the padded layout */
    const size_t smem =
        sizeof(df32) * kWinPieces *
            (win_stride_df(g.w, deg) + (deriv ? win_stride_df(g.w, deg - 1) : 0)) +
        sizeof(float) * kWinPieces * (win_stride_f(g.w, deg) + (deriv ? win_stride_f(g.w, deg - 1) : 0));
    /* grid-stride: at most 8 CTAs of 64 points per SM of a 148-SM part, looping over the rest */
    const int blocks = (int)std::min<int64_t>((n + 63) / 64, 148 * 8);
    cudaError_t e = cudaSuccess;
#define YK_CALL(W)                                                                              \
    if ((e = set_smem(k_frac_windows_df<W>, smem)) != cudaSuccess) return e;                   \
    k_frac_windows_df<W><<<blocks, 256, smem, st>>>(n, frac, count, coef, deriv ? 1 : 0, pitch,  \
                                                    out, idx, idx_lim)
    YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    return cudaGetLastError();
}

cudaError_t launch_prep_sources(const Geom &g, int64_t ns, const double *xs, const double *ys,
                                int64_t nd, const double *xd, const double *yd, int2 *tap,
                                float4 *frac, int *tile_cnt, int *tile_ptr, int *tile_cur,
                                double2 *ent_t, int *ent_j, int *err, cudaStream_t st, bool owner)
{
    const int ntiles = g.nt * g.nt;
    cudaError_t e = cudaMemsetAsync(tile_cnt, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(tile_cur, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    /* the two point sets: charges, then dipoles (index offset ns) */
    const int64_t cnt[2] = {ns, nd};
    const double *px[2] = {xs, xd}, *py[2] = {ys, yd};
    for (int k = 0; k < 2; ++k) {
        if (cnt[k] <= 0) continue;
        const int blocks = (int)((cnt[k] + 255) / 256);
        const int64_t o = k ? ns : 0;
#define YK_CALL(W)                                                                              \
    if (owner)                                                                                  \
        k_prep_src_count<W, true><<<blocks, 256, 0, st>>>(cnt[k], px[k], py[k], g, tap + o,     \
                                                          frac + o, tile_cnt, err);             \
    else                                                                                        \
        k_prep_src_count<W, false><<<blocks, 256, 0, st>>>(cnt[k], px[k], py[k], g, tap + o,    \
                                                           frac + o, tile_cnt, err)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    if ((e = launch_scan(tile_cnt, tile_ptr, ntiles, tile_cur, st)) != cudaSuccess) return e;
    for (int k = 0; k < 2; ++k) {
        if (cnt[k] <= 0) continue;
        const int blocks = (int)((cnt[k] + 255) / 256);
        const int64_t o = k ? ns : 0;
#define YK_CALL(W)                                                                              \
    if (owner)                                                                                  \
        k_prep_src_fill<W, true><<<blocks, 256, 0, st>>>(cnt[k], tap + o, frac + o, g, tile_ptr, \
                                                         tile_cur, ent_t, ent_j, (int)o);       \
    else                                                                                        \
        k_prep_src_fill<W, false><<<blocks, 256, 0, st>>>(cnt[k], tap + o, frac + o, g,         \
                                                          tile_ptr, tile_cur, ent_t, ent_j,     \
                                                          (int)o)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    return cudaGetLastError();
}

/* chunks of the histogram binning for nt targets over ntiles tiles: about 4096 targets each, at
 * most enough that the histogram matrix stays below 8M counters; 0 when the tiles' counters do
 * not fit in shared memory (the global-atomic binning is used then) */
int64_t hist_chunks(int64_t nt, int ntiles)
{
    if (ntiles > kHistTiles || nt <= 0) return 0;
    /* at least 4096 targets a chunk and one chunk (a CTA of kHistThreads) per SM of a 148-SM
     * part at most: a chunk zeroes, fills and writes a whole row of tile counters, so its
     * targets should outnumber its counters */
    return std::max<int64_t>(1, std::min<int64_t>((nt + 4095) / 4096, 148));
}

cudaError_t launch_prep_targets(const Geom &g, int64_t nt, const double *xt, const double *yt,
                                int4 *tap_tmp, float4 *frac_tmp, int *cnt, int *ptr, int *cur,
                                double2 *trg_t, float4 *trg_frac, int *trg_idx, int *err,
                                cudaStream_t st, int *hist)
{
    const int ntiles = g.nti * g.nti;
    const int64_t nch = hist ? hist_chunks(nt, ntiles) : 0;
    cudaError_t e = cudaSuccess;
    if (nch > 0) {
        const int64_t chunk = (nt + nch - 1) / nch;
        const size_t smem = sizeof(int) * (size_t)ntiles;
#define YK_CALL(W)                                                                              \
    if ((e = set_smem(k_trg_hist<W>, smem)) != cudaSuccess) return e;                          \
    if ((e = set_smem(k_trg_scatter<W>, smem)) != cudaSuccess) return e;                       \
    k_trg_hist<W><<<(int)nch, kHistThreads, smem, st>>>(nt, chunk, xt, yt, g, tap_tmp, frac_tmp,  \
                                                        hist, err)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
        const size_t csm = sizeof(int) * 33 * (size_t)nch;
        if ((e = set_smem(k_hist_columns, csm)) != cudaSuccess) return e;
        k_hist_columns<<<(ntiles + 31) / 32, 256, csm, st>>>(hist, (int)nch, ntiles, cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_scan(cnt, ptr, ntiles, cur, st)) != cudaSuccess) return e;
#define YK_CALL(W)                                                                              \
    k_trg_scatter<W><<<(int)nch, kHistThreads, smem, st>>>(nt, chunk, tap_tmp, frac_tmp, hist,     \
                                                           ntiles, ptr, trg_t, trg_frac, trg_idx)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
        return cudaGetLastError();
    }
    e = cudaMemsetAsync(cnt, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(cur, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((nt + 255) / 256);
    if (nt > 0) {
#define YK_CALL(W)                                                                              \
    k_prep_trg_count<W><<<blocks, 256, 0, st>>>(nt, xt, yt, g, tap_tmp, frac_tmp, cnt, err)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    if ((e = launch_scan(cnt, ptr, ntiles, cur, st)) != cudaSuccess) return e;
    if (nt > 0) {
        const int fblocks = (int)((nt + 256 * kFillPer - 1) / (256 * kFillPer));
#define YK_CALL(W)                                                                              \
    k_prep_trg_fill<W><<<fblocks, 256, 0, st>>>(nt, tap_tmp, frac_tmp, ptr, cur, trg_t, trg_frac, \
                                                trg_idx)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_wnu(int64_t nd, const double *wd, const double *nx, const double *ny,
                            double2 *wnu, cudaStream_t st)
{
    if (nd <= 0) return cudaSuccess;
    k_pack_wnu<<<(int)((nd + 255) / 256), 256, 0, st>>>(nd, wd, nx, ny, wnu);
    return cudaGetLastError();
}

cudaError_t launch_bin_targets(const Geom &g, int64_t nt, const double *xt, const double *yt,
                               double2 *trg_tmp, int *cnt, int *ptr, int *cur, double2 *trg_t,
                               int *trg_idx, int *err, cudaStream_t st)
{
    const int ntiles = g.nti * g.nti;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(cur, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((nt + 255) / 256);
    if (nt > 0) k_bin_trg_count<<<blocks, 256, 0, st>>>(nt, xt, yt, g, trg_tmp, cnt, err);
    if ((e = launch_scan(cnt, ptr, ntiles, cur, st)) != cudaSuccess) return e;
    if (nt > 0) {
#define YK_CALL(W)                                                                              \
    k_bin_trg_fill<W><<<blocks, 256, 0, st>>>(nt, trg_tmp, g, ptr, cur, trg_t, trg_idx)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    }
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const int *tile_ptr, int ntiles, int *order, int *scratch,
                              cudaStream_t st)
{
    if (ntiles <= 0) return cudaSuccess;
    if (ntiles <= kOrderSingle) {
        k_order_single<<<1, 1024, 0, st>>>(tile_ptr, ntiles, order);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int) * 80, st);
    if (e != cudaSuccess) return e;
    const int blocks = (ntiles + 255) / 256;
    k_order_hist<<<blocks < 148 ? blocks : 148, 256, 0, st>>>(tile_ptr, ntiles, scratch);
    k_order_base<<<1, 32, 0, st>>>(scratch);
    k_order_fill<<<blocks, 256, 0, st>>>(tile_ptr, ntiles, scratch, order);
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

template <typename R>
cudaError_t launch_fft_t(int stage, const void *grid_in, void *grid_out, void *spec,
                         const void *mult, const void *tw, const int *perm_h, const int *iperm_f,
                         const FftStages &sth, const FftStages &stf, int n, int M,
                         cudaStream_t st)
{
    Inst d = blank_inst(n, M);
    d.f32 = sizeof(R) == 4;
    d.rows = rows_per_item(n, d.f32, true);
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
        k_row_fwd<R><<<items, kRowThreads, smem, st>>>(d);
    } else if (stage == ST_COLUMNS) {
        if ((e = set_smem(k_columns<R>, smem)) != cudaSuccess) return e;
        k_columns<R><<<items, kColumnThreads, smem, st>>>(d);
    } else {
        if ((e = set_smem(k_row_inv<R>, smem)) != cudaSuccess) return e;
        k_row_inv<R><<<items, kRowThreads, smem, st>>>(d);
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
    k_interp32<W><<<g.nti * g.nti, 256, smem, st>>>(d)
        YK_W_DISPATCH(g.w, YK_CALL)
#undef YK_CALL
    } else {
#define YK_CALL(W)                                                                              \
    e = set_smem(k_interp<W>, smem);                                                            \
    if (e != cudaSuccess) return e;                                                             \
    k_interp<W><<<g.nti * g.nti, 256, smem, st>>>(d)
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
        if (d.f32 && d.dip) {
#define YK_CALL(W) YK_LAUNCH(k_spread_owner32_dip<W>, 32 * d.spread_warps)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else if (d.f32) {
#define YK_CALL(W) YK_LAUNCH(k_spread_owner32<W>, 32 * d.spread_warps)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else if (d.fft_df && d.dip) {
#define YK_CALL(W) YK_LAUNCH(k_spread_owner_df_dip<W>, 32 * d.spread_warps)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else if (d.fft_df) {
#define YK_CALL(W) YK_LAUNCH(k_spread_owner_df<W>, 32 * d.spread_warps)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else {
#define YK_CALL(W) YK_LAUNCH(k_spread<W>, 256)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        }
        break;
    case ST_ROW_FWD:
        if (d.f32) YK_LAUNCH(k_row_fwd<float>, kRowThreads);
        else if (d.fft_df) YK_LAUNCH(k_row_fwd<df32>, kRowThreads);
        else YK_LAUNCH(k_row_fwd<double>, kRowThreads);
        break;
    case ST_COLUMNS:
        if (d.f32) YK_LAUNCH(k_columns<float>, kColumnThreads);
        else if (d.fft_df) YK_LAUNCH(k_columns<df32>, kColumnThreads);
        else YK_LAUNCH(k_columns<double>, kColumnThreads);
        break;
    case ST_ROW_INV:
        if (d.f32) YK_LAUNCH(k_row_inv<float>, kRowThreads);
        else if (d.fft_df) YK_LAUNCH(k_row_inv<df32>, kRowThreads);
        else YK_LAUNCH(k_row_inv<double>, kRowThreads);
        break;
    default:
        if (d.f32) {
#define YK_CALL(W) YK_LAUNCH(k_interp32<W>, d.interp_threads)
            YK_W_DISPATCH(d.g.w, YK_CALL)
#undef YK_CALL
        } else if (d.fft_df) {
#define YK_CALL(W) YK_LAUNCH(k_interp_df<W>, d.interp_threads)
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
                                 double delta, double dk, double period, cudaStream_t st,
                                 const double *tab, int ntab, double H)
{
    const int64_t total = (int64_t)(M + 1) * (2 * M + 1);
    k_build_mult<df32><<<(int)((total + 255) / 256), 256, 0, st>>>(
        static_cast<df32 *>(mult), dfac, M, alpha, delta, dk, period, tab, ntab, H);
    return cudaGetLastError();
}

cudaError_t launch_build_mult(double *mult, const double *dfac, int M, double alpha, double delta,
                              double dk, double period, cudaStream_t st, const double *tab,
                              int ntab, double H)
{
    const int64_t total = (int64_t)(M + 1) * (2 * M + 1);
    k_build_mult<double><<<(int)((total + 255) / 256), 256, 0, st>>>(mult, dfac, M, alpha, delta,
                                                                     dk, period, tab, ntab, H);
    return cudaGetLastError();
}

cudaError_t launch_build_mult32(float *mult, const double *dfac, int M, double alpha,
                                double delta, double dk, double period, cudaStream_t st,
                                const double *tab, int ntab, double H)
{
    const int64_t total = (int64_t)(M + 1) * (2 * M + 1);
    k_build_mult<float><<<(int)((total + 255) / 256), 256, 0, st>>>(mult, dfac, M, alpha, delta,
                                                                    dk, period, tab, ntab, H);
    return cudaGetLastError();
}

cudaError_t launch_trunc_table(double *tab, int ntab, double H, double alpha, double delta,
                               double R0, double k0a, double k1a, const double2 *nodes, int nq,
                               cudaStream_t st)
{
    if (ntab <= 0) return cudaSuccess;
    const int64_t threads = (int64_t)ntab * 32;
    k_trunc_table<<<(int)((threads + 255) / 256), 256, 0, st>>>(tab, ntab, H, alpha, delta, R0,
                                                                 k0a, k1a, nodes, nq);
    return cudaGetLastError();
}

} /* namespace yk */
