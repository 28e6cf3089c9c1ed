/*
 * yk.h — C ABI of the B300 long-range ("history") evaluator for the 2D modified Helmholtz
 * (Yukawa) equation  (-Lap + alpha^2) u = f  (Section 1, eq. mod_helm).
 *
 * What the library computes.  For sources y_j with strengths q_j = w_j * density_j (boundary
 * quadrature weights times a layer density, Section 3.2 eq. bdry_quad, then volume quadrature
 * weights times source values, Section 3.1 eq. vol_quad) and targets x_i:
 *
 *     u_i = sum_j q_j G_H(x_i - y_j),
 *     G_H(x) = int_delta^inf exp(-|x|^2/(4t) - alpha^2 t) / (4 pi t) dt     (Section 2.1, eq. sl_sh)
 *
 * i.e. the history parts S_H[sigma] + V_H[f] of the single layer and volume potentials.  The
 * evaluation is the paper's Fourier method (Section 5): a type-1 spread of q onto a uniform
 * periodic grid, a forward FFT, multiplication by e^{-delta(alpha^2+|k|^2)}/(alpha^2+|k|^2)
 * (eq. sh) on the truncated mode set (eqs. kmax, delta_k, sh_fourier), an inverse FFT and a type-2
 * interpolation at the targets.  Every step runs in the library's own CUDA kernels (sm_103a).
 *
 * Conventions for every call.
 *  - Arrays are FP64 at the ABI.  Each array pointer may be host or device memory (detected with
 *    cudaPointerGetAttributes); device pointers must be usable on the plan's stream.
 *  - The caller owns every array it passes; the library owns the plan and its device buffers.
 *  - Calls are ordered on the plan's stream.  A call whose arrays are all device memory or
 *    page-locked (pinned) host memory returns once its work and copies are enqueued: the caller
 *    must not change such inputs or read such outputs before yk_sync (or another call that waits
 *    for the stream).  A call with a pageable host input returns after the input has been copied,
 *    and one with a pageable host output after the stream has finished.
 *  - No call aborts or throws across the ABI; every failure is a yk_status.  The message of the
 *    last failure on the calling thread is yk_last_error().
 *  - Errors detected by kernels (a point outside the box) are sticky in the plan and are
 *    returned by the next call that synchronises (yk_sync, or a call with pageable host
 *    arrays).
 */
#ifndef YK_H
#define YK_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define YK_API __attribute__((visibility("default")))
#else
#define YK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct yk_plan_s *yk_plan_t; /* opaque, owned by the library */

typedef enum {
    YK_OK = 0,
    YK_ERR_ARG = 1,      /* invalid argument (alpha <= 0, tol outside (0,1), point outside box, ...) */
    YK_ERR_OOM = 2,      /* a device allocation failed */
    YK_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    YK_ERR_TIMEOUT = 4,  /* a bounded device-side wait ran out */
    YK_ERR_STATE = 5,    /* call out of order (eval before set_points, ...) */
    YK_ERR_INTERNAL = 6, /* an internal consistency check failed */
    YK_ERR_UNSUPPORTED = 7 /* a size beyond what the library handles (see yk_plan) */
} yk_status;

typedef enum {
    YK_FP64 = 0, /* FP64 end to end */
    YK_FP32C = 1 /* FP32 spread/FFT/interp with compensated accumulation, FP64 final sums */
} yk_precision;

typedef struct {
    int precision;     /* yk_precision */
    double tol;        /* requested relative accuracy, e.g. 1e-10 (FP64) or 1e-6 (FP32C) */
    double delta;      /* > 0: time-split parameter delta of Section 2.1, used as is;
                          0: delta from the mesh rule of Section 6.4 with h_vol and eps_hist */
    double h_vol;      /* volume mesh size dx for the delta rule (used when delta == 0) */
    double eps_hist;   /* history tolerance of the delta rule; 0 means 1e-6 (Section 6) */
    double box[4];     /* xmin, xmax, ymin, ymax: every source and target lies inside */
    double kmax;       /* > 0: Fourier cutoff k_max used as is (else from tol, eq. kmax) */
    int kmax_rule;     /* 0: the tail of the Fourier integral beyond k_max is at most eps G_H(0)
                          (eq. kmax read relative to the size of G_H; eps = tol / 4);
                          1: eq. kmax as printed, exp(-delta (alpha^2 + k_max^2)) <= eps, with its
                          k_max = 0 case (u = 0) when delta alpha^2 >= ln(1/eps) */
    double period;     /* > 0: period P of the grid used as is (else box span + decay length) */
    int tile;          /* > 0: tile edge in grid cells (else chosen by the plan) */
    int profile;       /* nonzero: record CUDA events around every stage (see yk_stage_times) */
    void *stream;      /* cudaStream_t for all work of the plan; NULL = legacy default stream */
    /* optional device allocator (e.g. a caching allocator); NULL = cudaMalloc / cudaFree */
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *alloc_ctx;
    int use_tuned;      /* nonzero (and tile == 0): take the tile edge yk_autotune recorded for
                           this precision, window, grid size and n_src_hint */
    int64_t n_src_hint; /* expected number of sources (selects the autotuner's density band) */
    int fft_fp64;       /* FP64 path only: nonzero runs the FFT passes in FP64 arithmetic; the
                           default (0) runs them in double-float (FP32 pairs, ~48-bit mantissa,
                           error ~1e-14), which B300 executes much faster than FP64 */
    int dlp;            /* nonzero: the plan also takes double-layer (dipole) sources through
                           yk_set_points_dl / yk_eval_longrange_dl; k_max then also meets the
                           double-layer cutoff (Section 5.1, eq. kmax_dlp, read as kmax_rule says:
                           0: the tail of int exp(-delta(alpha^2+k^2)) k^2/(alpha^2+k^2) dk beyond
                           k_max is at most eps times the whole integral; 1: as printed) */
    int truncate;       /* small-alpha path (the paper points to Vico et al. for alpha -> 0, Section
                           5.2): every source-target distance is at most the box diagonal D, so G_H
                           may be replaced by G_H chi with chi = 1 on r <= D and a smooth step to 0
                           on [D, D + 12 s], s = 20 / k_max; the period then only needs to exceed
                           the span by D + 12 s instead of by the decay length of G_H, and the
                           multiplier is that kernel's radial transform (computed on the device
                           at plan time).  0: automatic (when it gives the shorter period and
                           opts.period is 0), 1: never, 2: always */
    /* launch shape of the FP32C and double-float spreads and interpolations (0: the default, or
     * the autotuner's choice with use_tuned); other values are YK_ERR_ARG */
    int spread_warps;   /* warps per spread CTA, each with its own copy of the tile: 1..4
                           (default 4) */
    int spread_batch;   /* sources a spread warp takes at a time: 4, 8 or 16 on the double-float
                           path (default 16), 8, 16 or 32 on FP32C (default 32) */
    int interp_threads; /* threads per interpolation CTA: 64, 128 or 256 (default 256) */
    int interp_tile;    /* FP32C and double-float paths: > 0 sets the edge of the targets' tiles
                           (the target binning and the interpolation, which read one halo per
                           tile): a divisor of n_grid, >= w, <= 32, else YK_ERR_ARG; 0: the
                           autotuner's (use_tuned), else the largest admissible divisor up to 32.
                           The all-FP64 path (fft_fp64) uses the tile edge for both and takes 0 */
} yk_opts;

/* Parameters the plan chose (all derived from alpha, tol, delta and the box). */
typedef struct {
    double alpha, delta, tol, eps; /* eps: internal accuracy target (tol / 4) */
    double kmax;                   /* Fourier cutoff (Section 5.1, eq. kmax; relative reading) */
    double period;                 /* P; Delta k = 2 pi / P (eq. delta_k) */
    double origin[2];              /* lower-left corner of the periodic box */
    double h;                      /* grid spacing P / n_grid */
    int64_t n_modes;               /* M: modes |m_x|, |m_y| <= M are kept */
    int64_t n_grid;                /* fine grid points per axis */
    int w;                         /* window width in grid points */
    double beta;                   /* exponential-of-semicircle window shape */
    int tile;                      /* tile edge (grid cells) */
    int precision;                 /* yk_precision */
    int64_t device_bytes;          /* device memory held by the plan now */
    int truncated;                 /* 1: the truncated kernel is used (opts.truncate) */
    double r_support;              /* truncated kernel: radius beyond which it is zero */
    int spread_warps, spread_batch, interp_threads; /* launch shape (see yk_opts) */
    int interp_tile;               /* edge of the targets' tiles (the tile edge on fft_fp64) */
} yk_info;

/* Fill *o with defaults: FP64, tol 1e-10, delta rule with eps_hist 1e-6, box [-1.5,1.5]^2. */
YK_API void yk_opts_default(yk_opts *o);

/*
 * yk_plan: choose the evaluation parameters for one alpha and one box and allocate the plan's
 * device buffers (grid, half spectrum, multiplier table of Section 5.2 eq. sh_fourier with the
 * window deconvolution folded in, FFT tables).  alpha > 0 (Section 1); tol in (0, 1).
 * With kmax_rule = 1 and delta alpha^2 >= ln(1/eps) the history part is below tolerance
 * (Section 5.1, the k_max = 0 case): no grid is allocated and every evaluation writes u = 0.
 * Returns YK_ERR_ARG for invalid options, YK_ERR_UNSUPPORTED when the grid would exceed
 * n_grid = 14400 (a grid column must fit one CTA's shared memory), YK_ERR_OOM, YK_ERR_CUDA.
 */
YK_API yk_status yk_plan(double alpha, const yk_opts *o, yk_plan_t *out);

/*
 * yk_set_points: give the sources (n_src nodes xs, ys with quadrature weights w: boundary nodes
 * then volume nodes, Sections 3.1-3.2) and the targets (n_trg points xt, yt).  Bins and sorts
 * both into grid tiles on the device; the layout stays resident until the next yk_set_points, so
 * repeated evaluations with new densities (a Rothe time step) reuse it.  n_src, n_trg >= 0; a
 * point outside the plan's box is reported (sticky) as YK_ERR_ARG.
 */
YK_API yk_status yk_set_points(yk_plan_t p, int64_t n_src, const double *xs, const double *ys,
                        const double *w, int64_t n_trg, const double *xt, const double *yt);

/*
 * yk_eval_longrange: u[i] = sum_j w_j density_j G_H(x_i - y_j) for the points of the last
 * yk_set_points (density: n_src values, sigma at boundary nodes then f at volume nodes; u: n_trg
 * values, written).  Returns YK_ERR_STATE before any yk_set_points.
 */
YK_API yk_status yk_eval_longrange(yk_plan_t p, const double *density, double *u);

/*
 * Double layer (Section 2, eq. dlp; history part D_H of Section 2.1; Fourier form in Section 5.1).
 * Dipole sources at boundary nodes y_d with quadrature weights wd_d and outward unit normals
 * (nx_d, ny_d) add
 *
 *     D_H[mu](x_i) = sum_d mu_d wd_d nu_d . grad_y G_H(x_i - y_d)
 *
 * to u.  In Fourier space this is the factor -i k . nu of the paper's D_H formula (the derivative
 * of exp(ik.(x - y)) with respect to the source point; the printed +i k has the sign of the
 * derivative in x).  The library folds that factor into the spread: a dipole is spread with the
 * gradient of the window, so charges and dipoles share one grid, one FFT pair and one
 * interpolation.
 *
 * yk_set_points_dl: as yk_set_points, plus n_dip dipole nodes (xd, yd, wd, nx, ny; host or device,
 * FP64; the caller's normals are used as given).  The plan must have been created with opts.dlp
 * when n_dip > 0 (else YK_ERR_ARG).  yk_set_points is yk_set_points_dl with n_dip = 0.
 *
 * yk_eval_longrange_dl: u = S_H[sigma] + V_H[f] (density, n_src values) + D_H[mu] (mu: n_dip
 * values at the dipole nodes); u (n_trg) is written.  yk_eval_longrange on a plan whose points
 * include dipoles returns YK_ERR_ARG (mu is required).  Batches (yk_batch_*) and the
 * allocation-free entry point take charges only: a plan with dipoles there is YK_ERR_UNSUPPORTED.
 */
YK_API yk_status yk_set_points_dl(yk_plan_t p, int64_t n_src, const double *xs, const double *ys,
                                  const double *w, int64_t n_dip, const double *xd,
                                  const double *yd, const double *wd, const double *nx,
                                  const double *ny, int64_t n_trg, const double *xt,
                                  const double *yt);
YK_API yk_status yk_eval_longrange_dl(yk_plan_t p, const double *density, const double *mu,
                                      double *u);

/*
 * yk_slp_local: the single-layer local asymptotic part S_{L,A}[sigma](x_i) = int_0^{delta_star}
 * int_boundary H(t, x_i - x') sigma(x') ds dt (Section 2.1, eq. sla) by the expansion of Section
 * 4.1 (Lemma, eq. slp_local1) through its delta_star^2 term, at the closest boundary point
 * found by Newton on the panel polynomial (Section 3.2).  With the history part at the same
 * delta (yk_eval_longrange with opts.delta = delta_star) it gives the single layer potential
 * S = S_{L,A} + S_H up to O(delta_star^{5/2}) near the boundary (no dyadic levels).
 *  - alpha > 0, delta_star > 0.
 *  - xb, yb, sigma: n_panels * q values, panel by panel, at the q Gauss-Legendre nodes of each
 *    panel's parameter t in [-1, 1] in ascending order; panels in counter-clockwise order around
 *    the closed boundary (panel p + 1 follows panel p, the last is followed by the first);
 *    2 <= q <= 32.
 *  - xt, yt (n_trg) in, u (n_trg) written: u_i = S_{L,A} at target i, 0 beyond the locality radius
 *    sqrt(delta_star)(12 + 2 alpha sqrt(delta_star)) from the boundary (remark on locality).
 *  - Every array is device memory (else YK_ERR_ARG); the call allocates and frees its scratch
 *    (Legendre series, cell lists of the panels and the targets) stream-ordered, from the
 *    device's default memory pool, and returns after its work on `stream`
 *    (cudaStream_t, NULL = legacy default stream) has finished.  YK_ERR_OOM if the scratch
 *    cannot be allocated, YK_ERR_UNSUPPORTED beyond 2^30 nodes or 2^31 - 1 targets, YK_ERR_CUDA
 *    if a CUDA call fails.
 *  - Readings of the printed lemma: Z = 4 c2 exp(-c1^2/4 - c2^2)/sqrt(pi) (the printed Z lacks the
 *    factor c2); kappa0 is the boundary's curvature in the (tangent, outward normal) frame, i.e.
 *    negative on a convex piece; rho = sign((x - x0) . nu0).
 *  - The boundary's derivatives at x0 come from the panel's polynomial; on a panel shorter than
 *    0.006 of the boundary's extent (where differentiating the rounded nodes would amplify their
 *    rounding) those of order >= 2 come from a least-squares polynomial fit over the nodes of
 *    the neighbouring panels within about that length, in the frame of the panel's middle node.
 */
YK_API yk_status yk_slp_local(double alpha, double delta_star, int64_t n_panels, int q,
                              const double *xb, const double *yb, const double *sigma,
                              int64_t n_trg, const double *xt, const double *yt, double *u,
                              void *stream);

/*
 * yk_dlp_local: the double-layer local asymptotic part D_{L,A}[mu](x_i) = int_0^{delta_star}
 * int_boundary dH(t, x_i - x')/dnu' mu(x') ds dt (Section 2.1, eq. dla) by the expansion of
 * Section 4.1 (the double-layer lemma, eq. dlp_local1) through its delta_star^2 term, at the
 * closest boundary point found as for yk_slp_local.  The normal derivative is taken in the source
 * point, nu' the outward normal (the convention of yk_eval_longrange_dl's dipoles), so that with
 * the history part at the same delta it gives D = D_{L,A} + D_H up to O(delta_star^{5/2}).
 *  - Arguments, memory, scratch, stream and errors as yk_slp_local, with mu (n_panels * q, at
 *    the nodes) in place of sigma.
 *  - u_i = D_{L,A} at target i, 0 beyond the locality radius.  A target within
 *    1e-10 sqrt(delta_star) of the boundary is on it: u_i is the integral at that boundary point
 *    (the corollary, eq. dlp_local2); any other target within the radius carries the double
 *    layer's jump (u -> +-mu0/2 plus the corollary's value as the target approaches the boundary
 *    from outside / inside).
 *  - Readings of the printed lemma: its overall sign is that of a derivative in the target and is
 *    reversed here; the gamma'''' part of the delta_star^{3/2} bracket multiplies 3 Q0 + P2 (the
 *    expansion of eq. dla; the printed 3 Q0 - U3 holds for the kappa0^3 part, and both agree on the
 *    boundary); mu', mu'', mu'''' and gamma''', gamma'''' are derivatives in the tangent-line
 *    parameter at x0, taken from the panel's polynomial; Z, kappa0 and rho as for yk_slp_local.
 */
YK_API yk_status yk_dlp_local(double alpha, double delta_star, int64_t n_panels, int q,
                              const double *xb, const double *yb, const double *mu,
                              int64_t n_trg, const double *xt, const double *yt, double *u,
                              void *stream);

/*
 * yk_slp_dyadic: the dyadic corrections of the single-layer local part (Section 2.1, eqs. slp_dyad
 * and sld): u_i = sum_{j=1}^{J} S_{L,D}^{(j)}[sigma](x_i), S_{L,D}^{(j)} = int_boundary
 * K_j(|x_i - x'|) sigma(x') ds with the difference kernel K_j(r) = int_{delta/4^j}^{delta/4^(j-1)}
 * e^{-r^2/4t - alpha^2 t} / (4 pi t) dt (eq. diffker_s through eq. equiv_split).  With
 * yk_slp_local at delta_star = delta / 4^J and the history part at delta this gives the single
 * layer potential S = S_{L,A} + sum_j S_{L,D}^{(j)} + S_H.
 *  - alpha > 0, delta > 0, 1 <= J <= 10; panels, sigma, targets and u as for yk_slp_local.
 *  - Level j resamples every panel on m_j sub-panels of the same q-point rule (no longer than
 *    3 sqrt(delta_j), from the panel's polynomial: the paper's bisection by interpolation) and
 *    sums over the nodes within R_j = sqrt(delta_{j-1})(12 + 2 alpha sqrt(delta_{j-1})), K_j from
 *    a piecewise polynomial table accurate to ~1e-16 of its peak.
 *  - Device memory only; YK_ERR_OOM if a level's scratch cannot be allocated; other errors as
 *    yk_slp_local.
 */
YK_API yk_status yk_slp_dyadic(double alpha, double delta, int J, int64_t n_panels, int q,
                               const double *xb, const double *yb, const double *sigma,
                               int64_t n_trg, const double *xt, const double *yt, double *u,
                               void *stream);

/*
 * yk_dlp_dyadic: the dyadic corrections of the double-layer local part (Section 2.1, eqs. dld and
 * diffker_dlp): u_i = sum_{j=1}^{J} int_boundary nu(x') . (x_i - x') K^D_j(|x_i - x'|) mu(x') ds,
 * K^D_j(r) = int_{delta/4^j}^{delta/4^(j-1)} e^{-r^2/4t - alpha^2 t} / (8 pi t^2) dt (the
 * source-point normal derivative of the heat kernel integrated over the level; eq. diffker_dlp
 * with K_nu(x, y) = int_1^inf s^(nu-1) e^(-x s - y/s) ds), nu the outward normal of the
 * counter-clockwise boundary.  Arguments, resampling and errors as yk_slp_dyadic (mu in place of
 * sigma).
 */
YK_API yk_status yk_dlp_dyadic(double alpha, double delta, int J, int64_t n_panels, int q,
                               const double *xb, const double *yb, const double *mu,
                               int64_t n_trg, const double *xt, const double *yt, double *u,
                               void *stream);

/*
 * yk_vp_local: the volume local part V_L[f](x_i) = int_0^{delta_star} int_Omega H_t(x_i - x') f(x')
 * dx' dt (Section 2.1, eq. vl) by the expansion of the Lemma for V_L (Section 4.1, eq. vp_local1)
 * through its delta_star^2 term at targets within the locality radius of the boundary (closest
 * point as in yk_slp_local), and by its interior form (eq. vp_local3) elsewhere.  With the history
 * part V_H at delta = delta_star it gives the volume potential V = V_L + V_H.
 *  - alpha > 0, delta_star > 0; boundary panels xb, yb (n_panels * q) as for yk_slp_local.
 *  - xt, yt (n_trg): targets in the closure of the domain; fd (6 * n_trg, plane after plane): f,
 *    f_x, f_y, f_xx, f_xy, f_yy at the targets; u (n_trg) written.
 *  - Reading: kappa0 is the second derivative of the boundary graph in the lemma's frame
 *    (tangent, inward normal), positive where the domain is convex; f^(0,1), f^(0,2), f^(2,0) are
 *    f's derivatives along the inward normal and the tangent at the closest point.
 *  - Targets within the locality radius that lie outside the domain get NaN and the call returns
 *    YK_ERR_ARG after finishing the others; targets farther away are taken to be inside.
 *  - Device memory only, scratch and stream semantics as yk_slp_local; the same error codes.
 */
YK_API yk_status yk_vp_local(double alpha, double delta_star, int64_t n_panels, int q,
                             const double *xb, const double *yb, int64_t n_trg, const double *xt,
                             const double *yt, const double *fd, double *u, void *stream);

/*
 * yk_plan_params: the parameters yk_plan would choose for (alpha, o), and in info->device_bytes
 * the device memory such a plan would hold after yk_set_points with n_src sources and n_trg
 * targets.  Makes no CUDA call (usable for memory-based admission before any allocation).
 */
YK_API yk_status yk_plan_params(double alpha, const yk_opts *o, int64_t n_src, int64_t n_trg,
                         yk_info *info);

/*
 * Stages timed when the plan was created with opts.profile != 0, in this order:
 * YK_STAGE_BIN_SRC, YK_STAGE_BIN_TRG (yk_set_points), YK_STAGE_SPREAD, YK_STAGE_ROW_FWD,
 * YK_STAGE_COLUMNS, YK_STAGE_ROW_INV, YK_STAGE_INTERP (yk_eval_longrange).
 */
enum {
    YK_STAGE_BIN_SRC = 0,
    YK_STAGE_BIN_TRG = 1,
    YK_STAGE_SPREAD = 2,
    YK_STAGE_ROW_FWD = 3,
    YK_STAGE_COLUMNS = 4,
    YK_STAGE_ROW_INV = 5,
    YK_STAGE_INTERP = 6,
    YK_NUM_STAGES = 7
};

/*
 * yk_stage_times: mean device time (ms, from CUDA events recorded on the plan's stream around the
 * stage's kernels) of each stage over its runs since the previous yk_stage_times call (at most
 * the last 64 runs), then restarts the count; ms[YK_NUM_STAGES] is written, -1 for a stage that
 * has not run.  Waits for the plan's stream.  YK_ERR_STATE if the plan was created without
 * opts.profile.
 */
YK_API yk_status yk_stage_times(yk_plan_t p, double *ms);

/* Wait for the plan's stream; return the plan's sticky status. */
YK_API yk_status yk_sync(yk_plan_t p);

/* Parameters chosen by yk_plan. */
YK_API yk_status yk_plan_info(yk_plan_t p, yk_info *info);

/* Free the plan and every device buffer it holds (after its stream's work has finished). */
YK_API yk_status yk_destroy(yk_plan_t p);

/* Message of the last failure on the calling thread; never NULL ("" when none). */
YK_API const char *yk_last_error(void);

/*
 * Autotuner.  yk_autotune times, on the caller's points (all arrays device memory; density n_src
 * values), every admissible tile edge with the default launch shape, then at the fastest edge the
 * spread's warps per CTA and sources per batch, the targets' tile edge and the interpolation's
 * threads per CTA (each stage timed alone), and records the fastest of each in a process-wide cache used by plans created
 * with o->use_tuned (batch plans included).  The paper has no counterpart.
 */
#define YK_TUNE_MAX 16
typedef struct {
    int n_tried;              /* tile candidates timed */
    int tile[YK_TUNE_MAX];    /* candidate tile edges */
    double ms[YK_TUNE_MAX];   /* device ms of one evaluation (sum of its stages) per candidate */
    int best_tile;
    double best_ms;           /* one evaluation at the best tile and launch shape */
    int64_t n_grid;
    int best_spread_warps, best_spread_batch, best_interp_threads;
    double spread_ms, interp_ms; /* the spread and interpolation at the chosen launch shape */
    int best_interp_tile;        /* the targets' tile edge (FP32C and double-float paths) */
} yk_tune_result;

YK_API yk_status yk_autotune(double alpha, const yk_opts *o, int64_t n_src, const double *xs,
                             const double *ys, const double *w, const double *density,
                             int64_t n_trg, const double *xt, const double *yt,
                             yk_tune_result *res);
/* write / read / clear the tuned-tile cache (a small text file: key columns and the tile) */
YK_API yk_status yk_tune_cache_save(const char *path);
YK_API yk_status yk_tune_cache_load(const char *path);
YK_API void yk_tune_cache_clear(void);

/*
 * yk_fma_peak: measured FMA throughput of the current device in TFLOP/s (2 flops per FMA) from
 * independent chains on every SM, for `precision` = YK_FP64 (FP64 FMA), YK_FP32C (FP32 FMA),
 * YK_PEAK_DF (the double-float multiply-add acc + a*b with a renormalised result, the building
 * block of the FP64 path's FFT passes and interpolation) or YK_PEAK_DF_LAZY (its unnormalised
 * form, the spread's per-tap operation); a double-float multiply-add counts as 2 FP64-equivalent
 * flops.  Other values: YK_ERR_ARG.  A diagnostic used to report ALU-bound kernels against a
 * measured peak; the paper has no counterpart.
 */
enum { YK_PEAK_DF = 2, YK_PEAK_DF_LAZY = 3 };
YK_API yk_status yk_fma_peak(int precision, double *tflops);

/*
 * yk_eval_longrange_static: one evaluation (yk_plan + yk_set_points + yk_eval_longrange in a
 * single call) that allocates no device memory, for callers that cannot call cudaMalloc — for
 * example code embedded in a host application that owns every device allocation, or a process
 * that must not grow its device footprint after start-up.  The paper has no counterpart; this is
 * a deployment variant of the same kernels.
 *  - alpha, o: as for yk_plan (o->alloc/o->free must be NULL; o->stream is used; o->truncate is
 *    ignored: this entry point always uses the untruncated kernel and its period).
 *  - xs, ys, w, density (n_src) and xt, yt (n_trg) are inputs, u (n_trg) is written; every array
 *    must be device memory, or YK_ERR_ARG.
 *  - All scratch lives in one static device array of 32 MiB that every GPU loading the library
 *    holds until the process exits; a problem needing more returns YK_ERR_UNSUPPORTED (the grid,
 *    its spectrum and multiplier, and about 120 bytes per source and 36 per target must fit).
 *  - The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 *    with that device current); make that first call before any stream capture.
 *  - Every call reuses the same array and clears what must start at zero; calls whose work
 *    overlaps on the GPU (other streams or threads) race on it.  The call waits for o->stream.
 *  - msg (msg_len bytes, may be NULL) receives the failure message.
 */
YK_API yk_status yk_eval_longrange_static(double alpha, const yk_opts *o, int64_t n_src,
                                          const double *xs, const double *ys, const double *w,
                                          const double *density, int64_t n_trg, const double *xt,
                                          const double *yt, double *u, char *msg,
                                          size_t msg_len);

/*
 * Batches: many evaluations (uneven sizes, different alpha, FP64 and FP32C mixed) in one
 * persistent launch per precision.  The plans' stages become one work list (all spreads, then all
 * row FFTs, columns, inverse rows and interpolations); CTAs pull items with an atomic counter, and
 * an item waits for the previous stage of its own instance with a bounded poll, so a stall is
 * reported as YK_ERR_TIMEOUT instead of hanging.  The launch is captured once into a CUDA graph
 * and replayed by later yk_batch_run calls.  Not in the paper: a serving-side layer over the same
 * stages (Section 5.2).
 */
typedef struct yk_batch_s *yk_batch_t;

typedef struct {
    void *stream;       /* cudaStream_t of the batch; NULL = stream of plans[0], and if that is
                           the legacy default stream, a blocking stream owned by the batch */
    int use_graph;      /* nonzero (default): capture the launch once, replay it afterwards */
    int64_t spin_limit; /* polls (about 0.2 us apart) an item may wait for its predecessors before
                           the batch fails with YK_ERR_TIMEOUT; 0 = 5e6 (about a second) */
    int inject_stall;   /* test hook: one dependency is never met, so a wait must time out */
} yk_batch_opts;

YK_API void yk_batch_opts_default(yk_batch_opts *o);

/*
 * yk_batch_create: a batch over n plans whose points are set (yk_set_points).  The plans stay
 * owned by the caller and must outlive the batch; calling yk_set_points on one of them later makes
 * the next yk_batch_run rebuild the work list.  YK_ERR_STATE if a plan has no points.
 */
YK_API yk_status yk_batch_create(yk_plan_t *plans, int n, const yk_batch_opts *o,
                                 yk_batch_t *out);

/*
 * yk_batch_set_plans: point an existing batch at another set of plans (same rules as
 * yk_batch_create), reusing its device buffers; waits for the batch's previous run.
 */
YK_API yk_status yk_batch_set_plans(yk_batch_t b, yk_plan_t *plans, int n);

/*
 * yk_batch_run: enqueue one evaluation of every plan on the batch stream: u[i] (n_trg of plan i,
 * written) from density[i] (n_src of plan i).  All arrays must be device memory ready on the
 * batch stream; returns after enqueueing.  Instances may not share output arrays.
 */
YK_API yk_status yk_batch_run(yk_batch_t b, const double *const *density, double *const *u);

/* Wait for the batch stream; YK_ERR_TIMEOUT if a bounded wait ran out during the last run. */
YK_API yk_status yk_batch_sync(yk_batch_t b);

YK_API yk_status yk_batch_destroy(yk_batch_t b);

/* yk_batch_eval: create (without graph), run, sync and destroy in one call. */
YK_API yk_status yk_batch_eval(yk_plan_t *plans, const double *const *density, double *const *u,
                               int n);

#ifdef __cplusplus
}
#endif
#endif /* YK_H */
