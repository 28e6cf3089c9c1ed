/*
 * yk_static.cu — yk_eval_longrange_static: one whole long-range evaluation that allocates no
 * device memory, for callers that cannot call cudaMalloc (code running inside a host that owns
 * every device allocation, such as a plug-in given fixed buffers, or a process whose memory
 * budget is fixed up front).  The paper has no counterpart: it is a deployment variant of the
 * same kernels.
 *
 * All scratch (grid, half spectrum, multiplier, FFT tables, tile lists) lives in one file-scope
 * device array of kStaticScratchBytes.  Every GPU that loads the library holds that array until
 * the process exits.  Host code cannot use the array's name as a device address, so the first
 * call on each device looks the address up with cudaGetSymbolAddress (with that device current)
 * and keeps it for that device's current CUDA context; that first call should come before any
 * stream capture.  The kept address is tied to the context's unique id: after cudaDeviceReset,
 * or under another context on the same device, the module is loaded anew and the next call
 * repeats the look-up instead of using an address of the old context.  Every call shares the
 * array: the contents left by the previous call are overwritten, everything that must start at
 * zero is cleared by the call itself, and calls whose work overlaps on the GPU (different
 * streams, or different host threads) race on the array.  The call waits for its stream.
 */
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "yk_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20; /* 32 MiB */
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
/* per device: the scratch address and the unique id of the context it was looked up in */
void *g_scratch_addr[kMaxDevices];
unsigned long long g_scratch_ctx[kMaxDevices];

/* failure message into the caller's buffer (if any) */
struct Msg {
    char *buf;
    size_t len;
};
thread_local Msg g_msg = {nullptr, 0};

yk_status static_fail(yk_status s, const char *msg, const char *detail = "")
{
    if (g_msg.buf && g_msg.len) snprintf(g_msg.buf, g_msg.len, "%s%s", msg, detail);
    return s;
}

/* unique id of the calling thread's current CUDA context (driver entry points fetched through the
 * runtime, so the library needs no link against the driver library); the runtime has made its
 * primary context current by the time this runs (the pointer checks come first) */
typedef int (*ctx_current_fn)(void **);
typedef int (*ctx_id_fn)(void *, unsigned long long *);

yk_status current_context_id(unsigned long long *id)
{
    static ctx_current_fn get_current = nullptr;
    static ctx_id_fn get_id = nullptr;
    if (!get_current || !get_id) { /* under g_setup_mutex */
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                         cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess || !f1 || !f2 || q1 != cudaDriverEntryPointSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            return static_fail(YK_ERR_CUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId: ",
                               e != cudaSuccess ? cudaGetErrorString(e) : "not found");
        get_current = (ctx_current_fn)f1;
        get_id = (ctx_id_fn)f2;
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx)
        return static_fail(YK_ERR_CUDA, "no current CUDA context");
    if (get_id(ctx, id) != 0) return static_fail(YK_ERR_CUDA, "cuCtxGetId failed");
    return YK_OK;
}

/* device address of g_scratch for the current device: looked up once per device and context */
yk_status scratch_base(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(YK_ERR_CUDA, "cudaGetDevice: ", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(YK_ERR_UNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long ctx = 0;
    yk_status s = current_context_id(&ctx);
    if (s != YK_OK) return s;
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr)
            return static_fail(YK_ERR_CUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
        g_scratch_addr[dev] = ptr;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return YK_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* plan tables computed on the device (no host staging buffers)                                */

__global__ void k_static_twiddles(double2 *tw, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s, c;
    sincospi(2.0 * (double)j / (double)n, &s, &c);
    tw[j] = make_double2(c, -s);
}

/* position of frequency m after the DIF stages (digits little-endian in r_1, r_2, ...) */
__device__ int dif_pos(const yk::FftStages &st, int m)
{
    int p = 0;
    for (int s = 0; s < st.n; ++s) {
        const int d = m % st.r[s];
        m /= st.r[s];
        p += d * (st.B[s] / st.r[s]);
    }
    return p;
}

__global__ void k_static_perms(int *perm_h, int *iperm_f, yk::FftStages sth, yk::FftStages stf)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < sth.L) perm_h[m] = dif_pos(sth, m);
    if (m < stf.L) iperm_f[dif_pos(stf, m)] = m;
}

struct GLRule {
    double x[128], w[128];
};

/* dfac[m] = 1 / phi_hat(2 pi m / n)^2, phi_hat by Gauss-Legendre in theta with z = (w/2) sin */
__global__ void k_static_dfac(double *dfac, int M, int n, int w, double beta, GLRule gl)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > M) return;
    const double xi = 2.0 * 3.14159265358979323846 * (double)m / (double)n, half = 0.5 * w;
    double sum = 0.0;
    for (int i = 0; i < 128; ++i) {
        const double th = 0.25 * 3.14159265358979323846 * (gl.x[i] + 1.0);
        sum += 0.25 * 3.14159265358979323846 * gl.w[i] * exp(beta * (cos(th) - 1.0)) *
               cos(xi * half * sin(th)) * half * cos(th);
    }
    const double ph = 2.0 * sum;
    dfac[m] = 1.0 / (ph * ph);
}

/* 128-point Gauss-Legendre rule into fixed arrays (Newton on the Legendre recurrence) */
void gl128(GLRule &g)
{
    const int n = 128;
    for (int i = 0; i < n / 2; ++i) {
        double z = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), dp = 0.0;
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
        g.x[i] = -z;
        g.x[n - 1 - i] = z;
        g.w[i] = g.w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

bool stages_for(int L, int n_tab, yk::FftStages &st)
{
    std::memset(&st, 0, sizeof st);
    st.L = L;
    int m = L, s = 0;
    const int radices[4] = {4, 2, 3, 5};
    for (int r : radices)
        while (m % r == 0) {
            if (s >= YK_MAX_STAGES) return false;
            st.r[s++] = r;
            m /= r;
        }
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

/* device (or managed) memory of the current device: a pointer into another GPU's memory is
 * refused, since the kernels run on the current device */
bool is_device(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

/* bump allocator over the static array (offsets only; nothing is allocated) */
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};

} /* namespace */

extern "C" YK_API yk_status yk_eval_longrange_static(double alpha, const yk_opts *o,
                                                     int64_t n_src, const double *xs,
                                                     const double *ys, const double *w,
                                                     const double *density, int64_t n_trg,
                                                     const double *xt, const double *yt,
                                                     double *u, char *msg, size_t msg_len)
{
    g_msg.buf = msg;
    g_msg.len = msg_len;
    if (msg && msg_len) msg[0] = '\0';
    yk_opts def;
    yk_opts_default(&def);
    if (!o) o = &def;
    if (o->alloc || o->free) return static_fail(YK_ERR_ARG, "allocator callbacks are not used here");
    if (o->precision != YK_FP64) return static_fail(YK_ERR_UNSUPPORTED, "FP64 only");
    if (n_src < 0 || n_trg < 0) return static_fail(YK_ERR_ARG, "negative point count");
    if (n_src > (1ll << 28) || n_trg > (1ll << 30))
        return static_fail(YK_ERR_UNSUPPORTED, "too many points for 32-bit entry indices");
    if ((n_src > 0 && (!is_device(xs) || !is_device(ys) || !is_device(w) || !is_device(density))) ||
        (n_trg > 0 && (!is_device(xt) || !is_device(yt) || !is_device(u))))
        return static_fail(YK_ERR_ARG, "every array must be device memory of the current device (no "
                                       "staging copies)");
    /* this entry point builds the plain multiplier only: no truncated kernel */
    yk_opts oc = *o;
    oc.truncate = 1;
    o = &oc;
    yk_info info;
    yk_status s = yk_plan_params(alpha, o, n_src, n_trg, &info);
    if (s != YK_OK) return static_fail(s, "parameters: ", yk_last_error());
    cudaStream_t st = (cudaStream_t)o->stream;
    if (n_trg == 0) return YK_OK;
    if (info.n_grid == 0 || n_src == 0) {
        cudaError_t e = cudaMemsetAsync(u, 0, sizeof(double) * (size_t)n_trg, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? YK_OK : static_fail(YK_ERR_CUDA, "zero output: ", cudaGetErrorString(e));
    }

    const int64_t n = info.n_grid, M = info.n_modes;
    const int T = info.tile, nt = (int)(n / T);
    const size_t nt2 = (size_t)nt * nt, ns = (size_t)n_src, ntg = (size_t)n_trg;
    Carve c;
    const size_t o_err = c.take(sizeof(int));
    const size_t o_grid = c.take(sizeof(double) * n * n);
    const size_t o_spec = c.take(sizeof(double2) * (M + 1) * n);
    const size_t o_mult = c.take(sizeof(double) * (M + 1) * (2 * M + 1));
    const size_t o_tw = c.take(sizeof(double2) * n);
    const size_t o_ph = c.take(sizeof(int) * (n / 2));
    const size_t o_if = c.take(sizeof(int) * n);
    const size_t o_dfac = c.take(sizeof(double) * (M + 1));
    const size_t o_tcnt = c.take(sizeof(int) * nt2), o_tptr = c.take(sizeof(int) * (nt2 + 1));
    const size_t o_tcur = c.take(sizeof(int) * nt2);
    const size_t o_gcnt = c.take(sizeof(int) * nt2), o_gptr = c.take(sizeof(int) * (nt2 + 1));
    const size_t o_gcur = c.take(sizeof(int) * nt2);
    const size_t o_srct = c.take(sizeof(double2) * ns);
    const size_t o_entt = c.take(sizeof(double2) * 4 * ns), o_entj = c.take(sizeof(int) * 4 * ns);
    const size_t o_trgt = c.take(sizeof(double2) * ntg), o_trgi = c.take(sizeof(int) * ntg);
    const size_t o_tmp = c.take(sizeof(double2) * ntg);
    if (c.off > kStaticScratchBytes) {
        char b[160];
        snprintf(b, sizeof b, "%zu bytes needed, the static scratch holds %zu (grid %lld^2, %lld "
                              "sources, %lld targets)",
                 c.off, kStaticScratchBytes, (long long)n, (long long)n_src, (long long)n_trg);
        return static_fail(YK_ERR_UNSUPPORTED, "problem too large for the static scratch: ", b);
    }

    void *base = nullptr;
    if ((s = scratch_base(&base)) != YK_OK) return s;
    unsigned char *B = static_cast<unsigned char *>(base);
    auto at = [&](size_t off) { return (void *)(B + off); };

    yk::Geom g;
    g.ox = info.origin[0];
    g.oy = info.origin[1];
    g.inv_h = (double)n / info.period;
    g.beta = info.beta;
    g.c = 4.0 / ((double)info.w * info.w);
    g.n = (int)n;
    g.T = T;
    g.nt = nt;
    g.Ti = T;
    g.nti = nt;
    g.w = info.w;
    for (int k = 0; k < 4; ++k) g.box[k] = o->box[k];

    yk::FftStages sth, stf;
    if (!stages_for((int)(n / 2), (int)n, sth) || !stages_for((int)n, (int)n, stf))
        return static_fail(YK_ERR_INTERNAL, "FFT stage plan failed");
    static GLRule gl; /* filled once under the set-up lock; fixed storage, no allocation */
    static bool gl_ready = false;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!gl_ready) {
            gl128(gl);
            gl_ready = true;
        }
    }

    cudaError_t e = cudaMemsetAsync(at(o_err), 0, sizeof(int), st);
    const int nb = (int)((n + 255) / 256);
    if (e == cudaSuccess) {
        k_static_twiddles<<<nb, 256, 0, st>>>((double2 *)at(o_tw), (int)n);
        k_static_perms<<<nb, 256, 0, st>>>((int *)at(o_ph), (int *)at(o_if), sth, stf);
        k_static_dfac<<<(int)((M + 1 + 127) / 128), 128, 0, st>>>((double *)at(o_dfac), (int)M,
                                                                 (int)n, info.w, info.beta, gl);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = yk::launch_build_mult((double *)at(o_mult), (const double *)at(o_dfac), (int)M, alpha,
                                  info.delta, 2.0 * 3.14159265358979323846 / info.period,
                                  info.period, st);
    if (e == cudaSuccess)
        e = yk::launch_bin_sources(g, n_src, xs, ys, 0, nullptr, nullptr, (double2 *)at(o_srct),
                                   (int *)at(o_tcnt),
                                   (int *)at(o_tptr), (int *)at(o_tcur), (double2 *)at(o_entt),
                                   (int *)at(o_entj), (int *)at(o_err), st);
    if (e == cudaSuccess)
        e = yk::launch_bin_targets(g, n_trg, xt, yt, (double2 *)at(o_tmp), (int *)at(o_gcnt),
                                   (int *)at(o_gptr), (int *)at(o_gcur), (double2 *)at(o_trgt),
                                   (int *)at(o_trgi), (int *)at(o_err), st);
    if (e == cudaSuccess)
        e = yk::launch_spread(g, (const int *)at(o_tptr), nullptr, (const double2 *)at(o_entt),
                              (const int *)at(o_entj), w, density, (double *)at(o_grid), st);
    if (e == cudaSuccess)
        e = yk::launch_row_fwd((const double *)at(o_grid), (double2 *)at(o_spec),
                               (const double2 *)at(o_tw), (const int *)at(o_ph), sth, (int)n,
                               (int)M, st);
    if (e == cudaSuccess)
        e = yk::launch_columns((double2 *)at(o_spec), (const double *)at(o_mult),
                               (const double2 *)at(o_tw), (const int *)at(o_if), stf, (int)n,
                               (int)M, st);
    if (e == cudaSuccess)
        e = yk::launch_row_inv((const double2 *)at(o_spec), (double *)at(o_grid),
                               (const double2 *)at(o_tw), (const int *)at(o_ph), sth, (int)n,
                               (int)M, st);
    if (e == cudaSuccess)
        e = yk::launch_interp(g, (const int *)at(o_gptr), (const double2 *)at(o_trgt),
                              (const int *)at(o_trgi), (const double *)at(o_grid), u, st);
    int h_err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h_err, at(o_err), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_fail(YK_ERR_CUDA, "launch: ", cudaGetErrorString(e));
    if (h_err & yk::ERR_POINT_OUTSIDE)
        return static_fail(YK_ERR_ARG, "a source or target lies outside the box");
    return YK_OK;
}
