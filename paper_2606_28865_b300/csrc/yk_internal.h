/*
 * yk_internal.h — plan structure and kernel launchers shared by the host API (yk_api.cu) and the
 * kernels (yk_kernels.cu).  Not part of the public ABI.
 */
#ifndef YK_INTERNAL_H
#define YK_INTERNAL_H

#include <cuda_runtime.h>
#include <stdint.h>

#include "yk_core.h"
#include "../../include/yk.h"

namespace yk {

/* pieces per tap of the double-float window polynomials, and their degree for window width w
 * (index w, 2..16): the lowest degree whose error at the interior taps is within 3% of
 * eps = 10^(1-w) (w <= 14; w = 15, 16 take the degree at which the fit reaches FP64 rounding),
 * found by interpolating at Chebyshev points in long double (at w = 12: 4.3e-14 at degree 4 with
 * 64 pieces, against 1.4e-13 at degree 6 with 8; the two edge taps carry the window's
 * square-root edge, ~1.1e-13 at w = 12 either way) */
constexpr int kWinPieces = 64;
constexpr int kPieceDeg[17] = {1, 1, 1, 1, 2, 2, 2, 3, 3, 3, 4, 4, 4, 5, 5, 5, 5};

/* grid geometry handed to kernels by value */
struct Geom {
    double ox, oy;  /* lower-left corner of the periodic box */
    double inv_h;   /* n / P */
    double beta;    /* window shape */
    double c;       /* 4 / w^2 */
    int n;          /* grid points per axis */
    int T;          /* tile edge (cells); divides n, T >= w, n >= 2T */
    int nt;         /* tiles per axis = n / T */
    int Ti;         /* tile edge of the target binning and the interpolation (divides n, Ti >= w,
                       n >= 2 Ti): T, or the plan's separate choice on the owner-tile paths */
    int nti;        /* target tiles per axis = n / Ti */
    int w;          /* window width */
    double box[4];  /* xmin, xmax, ymin, ymax: points outside are rejected */
    /* fixed-point grid coordinates of the double-float and FP32C paths: T = rint(x A + B) is
     * t 2^44 (t = (x - origin) / h in cells), A = 2^44 / h, B = -origin 2^44 / h per axis; a
     * coordinate in [0, n) has T in [0, n44), n44 = n 2^44 */
    double A, Bx, By;
    long long n44;
    long long tbox[4]; /* the box edges in the same fixed point (rounding is monotonic, so a
                          point in the box has tbox[0] <= T_x <= tbox[1], tbox[2] <= T_y <= tbox[3]) */
};

/* fraction bits of the fixed-point grid coordinate */
constexpr int kFixBits = 44;
/* threads per CTA of the per-plan FFT passes (the batch kernel runs every stage with 256); the
 * launch bounds keep them at <= 64 registers, so 1024 / threads CTAs share an SM.  Small CTAs
 * let one CTA's butterflies run while another waits at its stage barrier: 256 threads instead of
 * 1024 (columns) and 512 (rows) took the column pass -19..24% and the row passes -5..13% on B300.
 * A row work item holds at most kRowItemBytes of rows (two 2,560-point double-float rows). */
constexpr int kRowThreads = 256, kColumnThreads = 256;
constexpr int kRowItemBytes = 48 * 1024;

/* device error bits (sticky in the plan / batch) */
enum { ERR_POINT_OUTSIDE = 1, ERR_WAIT_TIMEOUT = 2 };

/* stages of one evaluation, in order (the batch kernel's per-instance counters follow them) */
enum { ST_SPREAD = 0, ST_ROW_FWD = 1, ST_COLUMNS = 2, ST_ROW_INV = 3, ST_INTERP = 4, ST_COUNT = 5 };

/* Everything a stage needs about one evaluation: the plan's grid and tables, the resident point
 * layout and this evaluation's density and output.  Handed by value to the per-stage kernels and
 * stored in device memory (one per instance) for the batch kernel. */
struct Inst {
    Geom g;
    FftStages sth, stf;       /* n/2-point (rows) and n-point (columns) transforms */
    int n, M, rows, f32;      /* rows: grid rows per row-FFT work item */
    int fft_df;               /* FP64 path: FFT arithmetic in double-float (tables in that form) */
    const int *tile_ptr;      /* source entries of tile t: [tile_ptr[t], tile_ptr[t+1]) */
    const int *order;         /* heavy-first tile order, or NULL */
    const double2 *ent_t;     /* entries (FP64: grid coordinate; FP32C: first tap + offset) */
    const int *ent_j;         /* source index of each entry */
    const double *wq;         /* quadrature weights (original order) */
    const int *trg_ptr;       /* targets of tile t: [trg_ptr[t], trg_ptr[t+1]) */
    const double2 *trg_t;     /* targets grouped by tile */
    const int *trg_idx;       /* original index of each grouped target */
    const double *dens;       /* density of this evaluation (n_src, device) */
    double *u;                /* output (n_trg, device) */
    void *grid;               /* R[n*n] */
    void *spec;               /* R2[(M+1)*n] */
    const void *mult;         /* R[(M+1)*(2M+1)] */
    const void *tw;           /* R2[n] */
    const int *perm_h, *iperm_f;
    const double *win;        /* FP64 windows as polynomials: win[k * w + a] is the coefficient of
                                 x^k for tap a, x = 2u - 1, u = l0 - t + w/2 in [0, 1); NULL: the
                                 window formula is evaluated directly */
    int wdeg;                 /* polynomial degree */
    const float2 *win_df;     /* the same coefficients as FP32 pairs (hi, lo), double-float path */
    /* double layer: entries with source index j >= n_chg are dipoles d = j - n_chg of vector
     * strength mu[d] * wnu[d] (weight times unit normal), spread with the window's gradient.
     * With dip set, win / win_df / win32 hold after the window's (wdeg+1) x w coefficients the
     * wdeg x w coefficients of its derivative phi'(z) (z in cells) in the same variable x. */
    int dip;                  /* nonzero: this evaluation has dipole sources */
    int n_chg;                /* number of charge sources (dipoles follow in the index space) */
    const double *mu;         /* double-layer density (n_dip, device) */
    const double2 *wnu;       /* wd * (nx, ny) per dipole (device) */
    const float *win32;       /* FP32C with dipoles: window and derivative polynomials in FP32 */
    double dmax;              /* bound on |phi'| over the window (cells^-1), for the FP64 scale */
    /* double-float path: window values computed once per point at yk_set_points (they depend on
     * positions only): per charge [phi(Y - t_y) taps | phi(X - t_x) taps] (2w double-floats, in
     * the order of the owner-tile entries, so a batch of a tile's sources is one contiguous block),
     * per dipole [phi_y | phi_x | phi'_y | phi'_x] (4w, source order), per target in tile order
     * (2w planes of n_trg values) */
    const float2 *win_src, *win_dip, *win_trg;
    int64_t win_trg_pitch;    /* the target windows are value-major: value k of target e at
                                 k * win_trg_pitch + e (coalesced reads in the interpolation) */
    void *part;               /* owner-tile spread (double-float and FP32C paths): padded tile
                                 partials, tile t's (T + w - 1)^2 cells at t (T + w - 1)^2 (FP32
                                 pairs), folded into the grid by the row FFT's load; NULL: the
                                 spread writes the grid itself (fixed-point FP64 path) */
    int spread_warps;         /* owner-tile spread: warps (padded copies) per CTA */
    int spread_batch;         /* owner-tile spread: sources a warp takes at a time */
    int interp_threads;       /* threads per interpolation CTA (per-stage launches) */
    int pad_shape_[3];        /* keeps sizeof(Inst) a multiple of 16 */
    int items[ST_COUNT];      /* work items of each stage */
    int smem[ST_COUNT];       /* dynamic shared memory of each stage (bytes) */
};

/* launch one stage of one evaluation (one CTA per work item) */
cudaError_t launch_stage(const Inst &d, int stage, cudaStream_t st);

/* shared-memory and work-item sizes of each stage (host side of the kernels' layouts) */
int stage_smem(const Inst &d, int stage);
int stage_items(const Inst &d, int stage);
int rows_per_item(int n, bool f32, bool fill_sms);

/* kernel launchers (yk_kernels.cu); all enqueue on `st` and return the launch status. */
/* The all-FP64 path's binning (FP64 grid coordinates): sources ns charges (xs, ys) then nd dipoles
 * (xd, yd), one entry per tile a source's window touches (<= 4), entries holding the grid
 * coordinate (double2) and the source index (a dipole's carries ns + d); src_t holds the ns + nd
 * grid coordinates */
cudaError_t launch_bin_sources(const Geom &g, int64_t ns, const double *xs, const double *ys,
                               int64_t nd, const double *xd, const double *yd, double2 *src_t,
                               int *tile_cnt, int *tile_ptr, int *tile_cur, double2 *ent_t,
                               int *ent_j, int *err, cudaStream_t st);
/* Point preparation of the double-float and FP32C paths (no FP64 arithmetic past the
 * fixed-point coordinate): per point its first taps tap = (l0x, l0y) (INT_MIN: outside the box)
 * and the window arguments u = l0 - t + w/2 in [0, 1) of both axes as exact FP32 pairs,
 * frac = (ux.hi, ux.lo, uy.hi, uy.lo), in the original order (targets: tap_tmp also holds the
 * tile of the target's cell, -1 outside).  Sources: ns charges then nd
 * dipoles (index offset ns); one entry per source in its owner tile (owner) or one per tile its
 * window touches; entry records int4 (owner: padded-copy offset, source index, sx, sy; else lx,
 * ly, sx, sy) with s = l0 - t in FP32.  Targets: records int4 (lx, ly, sx, sy) grouped by the
 * tile of their cell, and (trg_frac non-NULL) their frac in the same order. */
cudaError_t launch_prep_sources(const Geom &g, int64_t ns, const double *xs, const double *ys,
                                int64_t nd, const double *xd, const double *yd, int2 *tap,
                                float4 *frac, int *tile_cnt, int *tile_ptr, int *tile_cur,
                                double2 *ent_t, int *ent_j, int *err, cudaStream_t st, bool owner);
/* hist (may be NULL): hist_chunks(nt, tiles) x tiles ints of scratch for the histogram binning
 * (no global atomics); without it, or when the tiles' counters do not fit in shared memory, the
 * targets are binned with warp-aggregated global atomics */
cudaError_t launch_prep_targets(const Geom &g, int64_t nt, const double *xt, const double *yt,
                                int4 *tap_tmp, float4 *frac_tmp, int *cnt, int *ptr, int *cur,
                                double2 *trg_t, float4 *trg_frac, int *trg_idx, int *err,
                                cudaStream_t st, int *hist = nullptr);
int64_t hist_chunks(int64_t nt, int ntiles);
/* double-float window values of points given by their window arguments frac (as above):
 * out[i * 2w ...] as described for Inst::win_src; with deriv, 4w values per point including the
 * derivative's; a point whose frac is never written gets none (tap.x == INT_MIN is not read
 * here: invalid points are those past *count or, through idx, with idx[i] >= idx_lim).
 * pitch > 0: value-major planes (value k of point i at k * pitch + i). */
cudaError_t launch_frac_windows_df(const Geom &g, int64_t n, const float4 *frac, const int *count,
                                   const float2 *coef, int deg, bool deriv, float2 *out,
                                   cudaStream_t st, int64_t pitch = 0, const int *idx = nullptr,
                                   int64_t idx_lim = 0);
/* exclusive scan of cnt[0..count) into ptr[0..count]; cur (>= ceil(count / 4096) ints) is scratch
 * and is left zeroed */
cudaError_t launch_scan(const int *cnt, int *ptr, int count, int *cur, cudaStream_t st);
/* wnu[d] = wd[d] * (nx[d], ny[d]) */
cudaError_t launch_pack_wnu(int64_t nd, const double *wd, const double *nx, const double *ny,
                            double2 *wnu, cudaStream_t st);
cudaError_t launch_bin_targets(const Geom &g, int64_t nt, const double *xt, const double *yt,
                               double2 *trg_tmp, int *cnt, int *ptr, int *cur, double2 *trg_t,
                               int *trg_idx, int *err, cudaStream_t st);
/* heavy-first tile order (order[i] = tile the i-th spread CTA takes); order may be NULL in the
 * spread launchers, meaning tile i for CTA i */
cudaError_t launch_tile_order(const int *tile_ptr, int ntiles, int *order, int *scratch,
                              cudaStream_t st);
cudaError_t launch_spread(const Geom &g, const int *tile_ptr, const int *order,
                          const double2 *ent_t, const int *ent_j, const double *wq,
                          const double *dens, double *grid, cudaStream_t st);
cudaError_t launch_row_fwd(const double *grid, double2 *spec, const double2 *tw, const int *perm_h,
                           const FftStages &sth, int n, int M, cudaStream_t st);
cudaError_t launch_columns(double2 *spec, const double *mult, const double2 *tw,
                           const int *iperm_f, const FftStages &stf, int n, int M,
                           cudaStream_t st);
cudaError_t launch_row_inv(const double2 *spec, double *grid, const double2 *tw,
                           const int *perm_h, const FftStages &sth, int n, int M,
                           cudaStream_t st);
cudaError_t launch_row_fwd32(const float *grid, float2 *spec, const float2 *tw, const int *perm_h,
                             const FftStages &sth, int n, int M, cudaStream_t st);
cudaError_t launch_columns32(float2 *spec, const float *mult, const float2 *tw,
                             const int *iperm_f, const FftStages &stf, int n, int M,
                             cudaStream_t st);
cudaError_t launch_row_inv32(const float2 *spec, float *grid, const float2 *tw, const int *perm_h,
                             const FftStages &sth, int n, int M, cudaStream_t st);
cudaError_t launch_interp(const Geom &g, const int *trg_ptr, const double2 *trg_t,
                          const int *trg_idx, const double *grid, double *u, cudaStream_t st);
cudaError_t launch_interp32(const Geom &g, const int *trg_ptr, const double2 *trg_t,
                            const int *trg_idx, const float *grid, double *u, cudaStream_t st);
/* multiplier tables; tab (ntab entries at spacing H) non-NULL: the truncated kernel's radial
 * transform, interpolated, replaces exp(-delta(alpha^2+k^2))/(alpha^2+k^2) */
cudaError_t launch_build_mult(double *mult, const double *dfac, int M, double alpha, double delta,
                              double dk, double period, cudaStream_t st,
                              const double *tab = nullptr, int ntab = 0, double H = 0.0);
cudaError_t launch_build_mult32(float *mult, const double *dfac, int M, double alpha,
                                double delta, double dk, double period, cudaStream_t st,
                                const double *tab = nullptr, int ntab = 0, double H = 0.0);
/* multiplier as double-float pairs (FP64 path with double-float FFT arithmetic) */
cudaError_t launch_build_mult_df(void *mult, const double *dfac, int M, double alpha,
                                 double delta, double dk, double period, cudaStream_t st,
                                 const double *tab = nullptr, int ntab = 0, double H = 0.0);
/* radial transform of the truncated kernel at k_i = i H (see k_trunc_table); nodes[q] =
 * (r_q, f_q) with f_q = K0(alpha r_q) chi(r_q) r_q times the quadrature weight */
cudaError_t launch_trunc_table(double *tab, int ntab, double H, double alpha, double delta,
                               double R0, double k0a, double k1a, const double2 *nodes, int nq,
                               cudaStream_t st);

/* largest grid the column pass supports (one column of n complex values in shared memory) */
constexpr int kMaxGridF64 = 14400;
constexpr int kMaxGridF32 = 28800;

} /* namespace yk */

/* a device buffer with its size (bytes) */
struct DevBuf {
    void *ptr;
    size_t bytes;
};

/* the plan */
struct yk_plan_s {
    /* parameters */
    double alpha, delta, tol, eps, kmax, period, h, beta;
    double ox, oy;
    double box[4];
    int64_t M, n;
    int w, T, nt, Ti, nti, precision;
    int spread_warps, spread_batch, interp_threads; /* launch shape (yk_opts) */
    int fft_df; /* FP64 path: FFT arithmetic in double-float (default) or in FP64 */
    bool zero; /* k_max == 0: history below tolerance, u = 0 */
    cudaStream_t stream;
    void *(*alloc)(size_t, void *, void *);
    void (*dealloc)(void *, void *, void *);
    void *alloc_ctx;
    int64_t bytes;

    yk::FftStages st_half, st_full;

    /* plan-time device buffers */
    /* real type R = double (FP64) or float (FP32C) */
    DevBuf grid;     /* R[n*n]: spread output, then inverse-FFT output */
    DevBuf spec;     /* R2[(M+1)*n]: half spectrum, transposed: spec[kx*n + y] */
    DevBuf mult;     /* R[(M+1)*(2M+1)]: multiplier incl. window deconvolution */
    DevBuf tw;       /* R2[n]: exp(-2 pi i j / n) */
    DevBuf perm_h;   /* int[n/2]: DIF position of frequency m (half-length transform) */
    DevBuf iperm_f;  /* int[n]: frequency held at DIF position i (full-length transform) */
    DevBuf win;      /* double[(wdeg+1) * w]: window polynomials of the FP64 path */
    DevBuf win_df;   /* float2[(wdeg+1) * w]: the same as FP32 pairs (double-float path) */
    DevBuf win32;    /* float: FP32C window + derivative polynomials (plans with dlp) */
    DevBuf win_pc;   /* float2: kWinPieces-piece window (+ derivative) polynomials of the double-float
                        window kernel, degree pdeg */
    int pdeg;
    int wdeg;
    int dlp;         /* plan takes dipole sources */
    int truncated;   /* the kernel is truncated at the box diagonal (small-alpha path) */
    double r0, r1;   /* truncation: chi = 1 on r <= r0, a smooth step to 0 on [r0, r1] */
    double dmax;     /* bound on |phi'| (cells^-1) */
    DevBuf tile_cnt, tile_ptr, tile_cur; /* int[nt^2], int[nt^2+1], int[nt^2] (sources) */
    DevBuf tile_order; /* int[nt^2]: heavy-first processing order of the source tiles */
    DevBuf part;     /* owner-tile spread: nt^2 padded tiles of (T + w - 1)^2 FP32 pairs */
    DevBuf trg_cnt, trg_ptr, trg_cur;    /* same for targets */
    DevBuf err;      /* int: device error bits */

    /* resident point layout (grown on demand) */
    bool points_set;
    int64_t layout_version; /* incremented by every yk_set_points */
    int64_t n_src, n_trg, n_dip;
    DevBuf w_src;    /* double[n_src]: quadrature weights, original order */
    DevBuf wnu;      /* double2[n_dip]: dipole weight times unit normal */
    DevBuf win_src, win_dip, win_trg; /* double-float path: per-point window values */
    DevBuf src_t;    /* double2[n_src]: grid coordinates of the sources, original order */
    DevBuf ent_t;    /* 16 B x (<= 4 n_src): (source, tile) entries grouped by tile; FP64: grid
                        coordinate (double2); FP32C: first tap and FP32 offset (int2 + float2) */
    DevBuf ent_j;    /* int[<= 4 n_src]: source index of each entry */
    DevBuf trg_t;    /* 16 B x n_trg: targets grouped by tile (same two layouts as ent_t) */
    DevBuf trg_idx;  /* int[n_trg]: original index of each grouped target */
    DevBuf trg_tmp;  /* double2[n_trg]: grid coordinates in original order (fixed-point
                        preparation: the targets' window arguments, float4) */
    /* fixed-point preparation (double-float and FP32C paths): src_t holds the sources' window
     * arguments (float4) and src_tap their first taps (int2); trg_tap the targets' first taps and
     * cell tiles (int4, original order) */
    DevBuf src_tap, trg_tap;
    DevBuf trg_hist; /* int[chunks * tiles]: the targets' histogram binning */
    /* staging copies of host arrays */
    DevBuf stage_x, stage_y, stage_w, stage_u;
    DevBuf stage_d[6]; /* dipole inputs xd, yd, wd, nx, ny and the density mu */
    int status;      /* sticky yk_status */

    /* optional stage timing: a ring of kEventRing runs per stage; events[r][2 s] and
     * events[r][2 s + 1] bracket run r of stage s */
    static constexpr int kEventRing = 64;
    bool profile;
    cudaEvent_t events[kEventRing][2 * YK_NUM_STAGES];
    int64_t stage_runs[YK_NUM_STAGES]; /* runs recorded since the last yk_stage_times */
};


/* describe one evaluation of plan p (density and output filled in later); false when the plan
 * needs no kernels (k_max = 0, no sources or no targets: u = 0) */
bool yk_fill_inst(const yk_plan_s *p, yk::Inst *d);

/* launch shape recorded by the autotuner for this key: false when none (the outputs are then
 * left as they are) */
bool yk_tuned_shape(int precision, int w, int64_t n, int64_t n_src_hint, int *tile,
                    int *spread_warps, int *spread_batch, int *interp_threads, int *interp_tile);

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1] */
void yk_gauss_legendre(int n, double *x, double *w);

/* set the calling thread's message returned by yk_last_error */
void yk_set_last_error(const char *msg);

#endif /* YK_INTERNAL_H */
