/*
 * yk_tune.cu — tile-size autotuner and its cache.
 *
 * The tile edge T (grid cells per side of a spread/interpolation tile; a divisor of the grid size
 * n with w <= T <= 64, or <= 32 for FP32C, and n >= 2T) decides how many windows straddle tiles,
 * how much shared memory a CTA holds and how evenly work spreads over the SMs.  yk_autotune times
 * every admissible T on the caller's own points (CUDA events around the evaluation's kernels,
 * through the public ABI) and records the fastest in a process-wide cache keyed by precision,
 * window width, grid size band and sources per grid cell band.  Plans created with
 * opts.use_tuned take the admissible divisor of their n nearest to the cached tile.  The paper has
 * no counterpart (its NUFFT library chooses its own bins).
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

std::mutex g_tune_mutex;
std::map<Key, int> g_tuned;

int band(double v) { return v > 0 ? (int)std::floor(2.0 * std::log2(v) + 0.5) : -999; }

Key key_of(int precision, int w, int64_t n, int64_t n_src)
{
    const double dens = n > 0 ? (double)n_src / ((double)n * (double)n) : 0.0;
    return Key(precision, w, band((double)n), band(dens));
}

} /* namespace */

/* preferred tile for a plan (0: nothing cached) — used by yk_plan when opts.use_tuned is set */
int yk_tuned_tile(int precision, int w, int64_t n, int64_t n_src_hint)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key_of(precision, w, n, n_src_hint));
    return it == g_tuned.end() ? 0 : it->second;
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
    const int tmax = (o->precision == YK_FP32C || !o->fft_fp64) ? 32 : 64;
    std::vector<int> cand;
    for (int t = tmax; t >= info.w && (int)cand.size() < YK_TUNE_MAX; --t)
        if (n % t == 0 && n >= 2 * t) cand.push_back(t);
    /* an output buffer for the timed evaluations */
    double *u = nullptr;
    if (cudaMalloc(&u, sizeof(double) * (size_t)n_trg) != cudaSuccess) {
        cudaGetLastError();
        return YK_ERR_OOM;
    }
    double best = 1e300;
    for (size_t k = 0; k < cand.size(); ++k) {
        yk_opts oc = *o;
        oc.tile = cand[k];
        oc.profile = 1;
        oc.use_tuned = 0;
        yk_plan_t p = nullptr;
        s = yk_plan(alpha, &oc, &p);
        if (s != YK_OK) {
            cudaFree(u);
            return s;
        }
        double ms[YK_NUM_STAGES];
        s = yk_set_points(p, n_src, xs, ys, w, n_trg, xt, yt);
        /* one warm-up evaluation, then the mean of three timed ones */
        if (s == YK_OK) s = yk_eval_longrange(p, density, u);
        if (s == YK_OK) s = yk_stage_times(p, ms);
        for (int r = 0; r < 3 && s == YK_OK; ++r) s = yk_eval_longrange(p, density, u);
        if (s == YK_OK) s = yk_stage_times(p, ms);
        yk_destroy(p);
        if (s != YK_OK) {
            cudaFree(u);
            return s;
        }
        double t_eval = 0.0;
        for (int st = YK_STAGE_SPREAD; st <= YK_STAGE_INTERP; ++st) t_eval += ms[st] > 0 ? ms[st] : 0.0;
        res->tile[k] = cand[k];
        res->ms[k] = t_eval;
        if (t_eval < best) {
            best = t_eval;
            res->best_tile = cand[k];
            res->best_ms = t_eval;
        }
    }
    cudaFree(u);
    res->n_tried = (int)cand.size();
    res->n_grid = n;
    if (res->best_tile > 0) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[key_of(o->precision, info.w, n, n_src)] = res->best_tile;
    }
    return YK_OK;
}

YK_API yk_status yk_tune_cache_save(const char *path)
{
    if (!path) return YK_ERR_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f) return YK_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    std::fprintf(f, "# precision w n_band density_band tile\n");
    for (const auto &kv : g_tuned)
        std::fprintf(f, "%d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                     std::get<2>(kv.first), std::get<3>(kv.first), kv.second);
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
        int a, b, c, d, t;
        if (line[0] == '#') continue;
        if (std::sscanf(line, "%d %d %d %d %d", &a, &b, &c, &d, &t) == 5 && t > 0)
            g_tuned[Key(a, b, c, d)] = t;
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
