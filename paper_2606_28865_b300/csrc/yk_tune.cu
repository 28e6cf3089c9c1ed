/*
 * yk_tune.cu — launch-shape autotuner and its cache.
 *
 * The tile edge T (grid cells per side of a spread/interpolation tile; a divisor of the grid size
 * n with w <= T <= 64, or <= 32 for the owner-tile spreads, and n >= 2T) decides how many grid
 * cells a tile's padded copy adds, how much shared memory a CTA holds and how evenly work spreads
 * over the SMs; the spread's warps per CTA (its padded copies) and sources per batch trade
 * shared memory and registers against latency hiding; the interpolation's threads per CTA set its
 * occupancy, and the targets' tile edge (apart from T on the owner-tile paths) how often the
 * interpolation reads a halo.  yk_autotune times every admissible T with the default shape on the
 * caller's own points (CUDA events around the evaluation's kernels, through the public ABI), then,
 * at the fastest T, every spread shape, every targets' tile edge and every interpolation block
 * size (each stage timed alone), and
 * records the winners in a process-wide cache keyed by precision, window width, grid size band and
 * sources per grid cell band.  Plans created with opts.use_tuned take the admissible divisor of
 * their n nearest to the cached tile and the cached shape.  The paper has no counterpart (its
 * NUFFT library chooses its own bins).
 */
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "yk_internal.h"

namespace {

using Key = std::tuple<int, int, int, int>; /* precision, w, log2 n band, log2 density band */

struct Shape {
    int tile, spread_warps, spread_batch, interp_threads, interp_tile;
};

std::mutex g_tune_mutex;
std::map<Key, Shape> g_tuned;

int band(double v) { return v > 0 ? (int)std::floor(2.0 * std::log2(v) + 0.5) : -999; }

Key key_of(int precision, int w, int64_t n, int64_t n_src)
{
    const double dens = n > 0 ? (double)n_src / ((double)n * (double)n) : 0.0;
    return Key(precision, w, band((double)n), band(dens));
}

/* set_points once, one warm-up evaluation, then the mean per-stage device time of three */
yk_status time_plan(double alpha, const yk_opts &oc, int64_t n_src, const double *xs,
                    const double *ys, const double *w, const double *density, int64_t n_trg,
                    const double *xt, const double *yt, double *u, double *ms)
{
    yk_plan_t p = nullptr;
    yk_status s = yk_plan(alpha, &oc, &p);
    if (s != YK_OK) return s;
    s = yk_set_points(p, n_src, xs, ys, w, n_trg, xt, yt);
    if (s == YK_OK) s = yk_eval_longrange(p, density, u);
    if (s == YK_OK) s = yk_stage_times(p, ms);
    for (int r = 0; r < 3 && s == YK_OK; ++r) s = yk_eval_longrange(p, density, u);
    if (s == YK_OK) s = yk_stage_times(p, ms);
    yk_destroy(p);
    return s;
}

double eval_ms(const double *ms)
{
    double t = 0.0;
    for (int st = YK_STAGE_SPREAD; st <= YK_STAGE_INTERP; ++st) t += ms[st] > 0 ? ms[st] : 0.0;
    return t;
}

} /* namespace */

/* launch shape recorded for a plan's key — used by yk_plan when opts.use_tuned is set */
bool yk_tuned_shape(int precision, int w, int64_t n, int64_t n_src_hint, int *tile,
                    int *spread_warps, int *spread_batch, int *interp_threads, int *interp_tile)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key_of(precision, w, n, n_src_hint));
    if (it == g_tuned.end()) return false;
    *tile = it->second.tile;
    *spread_warps = it->second.spread_warps;
    *spread_batch = it->second.spread_batch;
    *interp_threads = it->second.interp_threads;
    *interp_tile = it->second.interp_tile;
    return true;
}

extern "C" {

YK_API yk_status yk_autotune(double alpha, const yk_opts *o, int64_t n_src, const double *xs,
                             const double *ys, const double *w, const double *density,
                             int64_t n_trg, const double *xt, const double *yt,
                             yk_tune_result *res)
{
    if (!res) return YK_ERR_ARG;
    std::memset(res, 0, sizeof *res);
    yk_opts def;
    yk_opts_default(&def);
    if (!o) o = &def;
    yk_info info;
    yk_status s = yk_plan_params(alpha, o, n_src, n_trg, &info);
    if (s != YK_OK) return s;
    if (info.n_grid == 0 || n_src == 0 || n_trg == 0) return YK_OK; /* nothing to tune */
    const int64_t n = info.n_grid;
    const bool owner = o->precision == YK_FP32C || !o->fft_fp64;
    const int tmax = owner ? 32 : 64;
    std::vector<int> cand;
    for (int t = tmax; t >= info.w && (int)cand.size() < YK_TUNE_MAX; --t)
        if (n % t == 0 && n >= 2 * t) cand.push_back(t);
    /* an output buffer for the timed evaluations */
    double *u = nullptr;
    if (cudaMalloc(&u, sizeof(double) * (size_t)n_trg) != cudaSuccess) {
        cudaGetLastError();
        return YK_ERR_OOM;
    }
    yk_opts base = *o;
    base.profile = 1;
    base.use_tuned = 0;
    double ms[YK_NUM_STAGES];
    /* 1. the tile edge, with the caller's (or the default) launch shape */
    double best = 1e300;
    for (size_t k = 0; k < cand.size(); ++k) {
        yk_opts oc = base;
        oc.tile = cand[k];
        s = time_plan(alpha, oc, n_src, xs, ys, w, density, n_trg, xt, yt, u, ms);
        if (s != YK_OK) {
            cudaFree(u);
            return s;
        }
        res->tile[k] = cand[k];
        res->ms[k] = eval_ms(ms);
        if (res->ms[k] < best) {
            best = res->ms[k];
            res->best_tile = cand[k];
            res->spread_ms = ms[YK_STAGE_SPREAD];
            res->interp_ms = ms[YK_STAGE_INTERP];
        }
    }
    res->n_tried = (int)cand.size();
    res->n_grid = n;
    base.tile = res->best_tile;
    {
        yk_info di;
        if ((s = yk_plan_params(alpha, &base, n_src, n_trg, &di)) != YK_OK) {
            cudaFree(u);
            return s;
        }
        res->best_spread_warps = di.spread_warps;
        res->best_spread_batch = di.spread_batch;
        res->best_interp_threads = di.interp_threads;
        res->best_interp_tile = di.interp_tile;
    }
    if (owner && res->best_tile > 0) {
        /* 2. the spread's warps per CTA and sources per batch at that tile (spread time alone) */
        const int batches32[3] = {8, 16, 32}, batches_df[3] = {4, 8, 16};
        const int *batches = o->precision == YK_FP32C ? batches32 : batches_df;
        for (int sw = 2; sw <= 4; ++sw)
            for (int b = 1; b < 3; ++b) {
                yk_opts oc = base;
                oc.spread_warps = sw;
                oc.spread_batch = batches[b];
                s = time_plan(alpha, oc, n_src, xs, ys, w, density, n_trg, xt, yt, u, ms);
                if (s != YK_OK) {
                    cudaFree(u);
                    return s;
                }
                if (ms[YK_STAGE_SPREAD] > 0 && ms[YK_STAGE_SPREAD] < res->spread_ms) {
                    res->spread_ms = ms[YK_STAGE_SPREAD];
                    res->best_spread_warps = sw;
                    res->best_spread_batch = batches[b];
                }
            }
        /* 3. the targets' tile edge, then the interpolation's threads per CTA (interpolation
         * time alone) */
        base.spread_warps = res->best_spread_warps;
        base.spread_batch = res->best_spread_batch;
        for (int ti = 32; ti >= info.w; --ti) {
            if (!(n % ti == 0 && n >= 2 * ti) || ti == res->best_interp_tile) continue;
            yk_opts oc = base;
            oc.interp_tile = ti;
            s = time_plan(alpha, oc, n_src, xs, ys, w, density, n_trg, xt, yt, u, ms);
            if (s != YK_OK) {
                cudaFree(u);
                return s;
            }
            if (ms[YK_STAGE_INTERP] > 0 && ms[YK_STAGE_INTERP] < res->interp_ms) {
                res->interp_ms = ms[YK_STAGE_INTERP];
                res->best_interp_tile = ti;
            }
        }
        base.interp_tile = res->best_interp_tile;
        for (int th : {128, 256}) {
            yk_opts oc = base;
            oc.interp_threads = th;
            s = time_plan(alpha, oc, n_src, xs, ys, w, density, n_trg, xt, yt, u, ms);
            if (s != YK_OK) {
                cudaFree(u);
                return s;
            }
            if (ms[YK_STAGE_INTERP] > 0 && ms[YK_STAGE_INTERP] < res->interp_ms) {
                res->interp_ms = ms[YK_STAGE_INTERP];
                res->best_interp_threads = th;
            }
        }
        /* the whole evaluation at the chosen shape */
        base.interp_threads = res->best_interp_threads;
        s = time_plan(alpha, base, n_src, xs, ys, w, density, n_trg, xt, yt, u, ms);
        if (s != YK_OK) {
            cudaFree(u);
            return s;
        }
        best = eval_ms(ms);
    }
    res->best_ms = best;
    cudaFree(u);
    if (res->best_tile > 0) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[key_of(o->precision, info.w, n, n_src)] =
            Shape{res->best_tile, res->best_spread_warps, res->best_spread_batch,
                  res->best_interp_threads, res->best_interp_tile};
    }
    return YK_OK;
}

YK_API yk_status yk_tune_cache_save(const char *path)
{
    if (!path) return YK_ERR_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f) return YK_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    std::fprintf(f, "# precision w n_band density_band tile spread_warps spread_batch "
                    "interp_threads interp_tile\n");
    for (const auto &kv : g_tuned)
        std::fprintf(f, "%d %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first),
                     std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
                     kv.second.tile, kv.second.spread_warps, kv.second.spread_batch,
                     kv.second.interp_threads, kv.second.interp_tile);
    std::fclose(f);
    return YK_OK;
}

YK_API yk_status yk_tune_cache_load(const char *path)
{
    if (!path) return YK_ERR_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) return YK_ERR_ARG;
    char line[256];
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    while (std::fgets(line, sizeof line, f)) {
        int a, b, c, d, t, sw = 0, sb = 0, it = 0, ti = 0;
        if (line[0] == '#') continue;
        /* five columns (tile only), eight (and the launch shape) or nine (and the targets' tile);
         * 0 = default */
        const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d", &a, &b, &c, &d, &t, &sw,
                                    &sb, &it, &ti);
        if (got >= 5 && t > 0) g_tuned[Key(a, b, c, d)] = Shape{t, sw, sb, it, ti};
    }
    std::fclose(f);
    return YK_OK;
}

YK_API void yk_tune_cache_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned.clear();
}

} /* extern "C" */
