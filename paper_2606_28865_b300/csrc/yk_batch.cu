/*
 * yk_batch.cu — many uneven evaluations in one persistent launch.
 *
 * A batch holds plans whose points are set.  Their stages become one work list in topological
 * order: every spread item of every instance, then every row-FFT item, then every column, every
 * inverse-row item and every interpolation item (instances ordered by decreasing cost inside each
 * stage).  One persistent kernel per precision pulls items from the list with an atomic counter;
 * an item of stage s of instance i first waits until all items of stage s-1 of instance i have
 * finished (a per-instance counter).  Items are taken in list order by running CTAs only, so every
 * item a CTA waits for is already held by a running CTA that waits only for earlier items: the
 * waits always end.  Each wait is still bounded (a poll limit, then an error bit and the CTA moves
 * on) so a broken invariant reports YK_ERR_TIMEOUT instead of hanging the GPU.  The launch (two
 * memsets and one kernel per precision) is captured once into a CUDA graph and replayed.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "yk_stages.cuh"

namespace {

using yk::Inst;

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

/* items[q] = (instance, stage << 24 | index); one kernel per precision and window width */
template <typename R, int W>
__global__ void __launch_bounds__(256)
    k_batch(const Inst *__restrict__ insts, const int *__restrict__ need,
            const int2 *__restrict__ items, int total, int *head, int *done, int *status,
            long long spin_limit)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_q, s_go;
    /* the item's instance descriptor, copied into shared memory: the stage bodies index its
     * tables (FFT stage lists) dynamically, which from global memory cost registers and spills */
    __shared__ __align__(16) Inst s_inst;
    static_assert(sizeof(Inst) % 16 == 0, "Inst is copied in 16-byte words");
    int held = -1; /* the instance whose descriptor s_inst holds (items of one instance and stage
                      are consecutive in the list, so a CTA mostly takes the same one again) */
    /* items are claimed two at a time (one atomic for both) and run in list order; the second
     * waits like any other item, and only for items earlier in the list, so the waits still end */
    int q0 = 0, nq = 0; /* the claimed pair [q0, q0 + nq) */
    for (;;) {
        if (nq == 0) {
            if (threadIdx.x == 0) s_q = atomicAdd(head, 2);
            __syncthreads();
            q0 = s_q;
            nq = 2;
            __syncthreads(); /* s_q is rewritten below */
        }
        const int q = q0 + (2 - nq);
        --nq;
        if (q >= total) return; /* uniform */
        if (threadIdx.x == 0) {
            int go = 1;
            const int2 it = items[q];
            const int stage = it.y >> 24;
            if (stage > 0) {
                const int *cnt = done + it.x * yk::ST_COUNT + stage - 1;
                const int want = need[it.x * yk::ST_COUNT + stage - 1];
                long long k = 0;
                while (ld_acquire(cnt) < want) {
                    if (*(volatile int *)status) {
                        go = 0;
                        break;
                    }
                    if (++k > spin_limit) {
                        atomicOr(status, yk::ERR_WAIT_TIMEOUT);
                        go = 0;
                        break;
                    }
                    __nanosleep(200);
                }
                __threadfence();
            }
            if (*(volatile int *)status) go = 0;
            s_go = go;
        }
        __syncthreads();
        const int2 it = items[q];
        const int inst = it.x, stage = it.y >> 24, idx = it.y & 0xffffff;
        if (s_go) {
            if (inst != held) { /* uniform: every thread read the same item */
                const int4 *src = reinterpret_cast<const int4 *>(insts + inst);
                int4 *dst = reinterpret_cast<int4 *>(&s_inst);
                for (int i = threadIdx.x; i < (int)(sizeof(Inst) / 16); i += blockDim.x)
                    dst[i] = src[i];
                held = inst;
                __syncthreads();
            }
            yk::run_stage_w<R, W>(s_inst, stage, idx, sm);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + inst * yk::ST_COUNT + stage, 1);
        }
    }
}

yk_status bfail(yk_status s, const char *fmt, ...)
{
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    yk_set_last_error(buf);
    return s;
}

struct Buf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t b)
    {
        if (ptr && bytes >= b) return cudaSuccess;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        if (b == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&ptr, b);
        if (e == cudaSuccess) bytes = b;
        return e;
    }
    void release()
    {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
};

/* the instances of one precision and window width */
struct Group {
    bool f32 = false;
    int w = 0;
    std::vector<int> members;     /* indices into the batch's plans */
    std::vector<Inst> h_inst;     /* host copies (density/output pointers refreshed per run) */
    Buf insts, need, items, done, head;
    int total = 0, grid = 0, smem = 0;
};

} /* namespace */

struct yk_batch_s {
    std::vector<yk_plan_t> plans;
    std::vector<int64_t> versions;
    std::vector<int> trivial;      /* plans whose output is zero (no kernels) */
    std::vector<int64_t> trivial_n;
    std::vector<Group> grp;        /* one per (precision, window width) */
    Buf status;
    cudaStream_t stream = nullptr;
    bool own_stream = false; /* created here: graphs cannot be captured on the legacy stream */
    bool use_graph = true;
    long long spin_limit = 5000000;
    bool inject_stall = false;
    cudaGraphExec_t exec = nullptr;
    std::vector<const double *> last_dens;
    std::vector<double *> last_u;
    bool built = false;
};

namespace {

void drop_graph(yk_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

/* cost estimate used to put heavy instances first inside every stage */
double inst_cost(const Inst &d)
{
    const double n = d.n;
    return n * n * (std::log2(n) + 4.0) + 50.0 * (d.tile_ptr ? 1.0 : 0.0);
}

/* shared-memory attribute and occupancy of the group's kernel */
template <typename R, int W> cudaError_t setup_one(int smem, int *per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(k_batch<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch<R, W>,
                                                                          256, smem);
    return e;
}

cudaError_t kernel_setup(bool f32, int w, int smem, int *per_sm)
{
    cudaError_t e = cudaSuccess;
#define YK_C(W) e = f32 ? setup_one<float, W>(smem, per_sm) : setup_one<double, W>(smem, per_sm)
    YK_W_SWITCH(w, YK_C)
#undef YK_C
    return e;
}

void launch_group(const Group &g, const yk_batch_s *b)
{
    const Inst *insts = (const Inst *)g.insts.ptr;
    const int *need = (const int *)g.need.ptr;
    const int2 *items = (const int2 *)g.items.ptr;
    int *head = (int *)g.head.ptr, *done = (int *)g.done.ptr, *status = (int *)b->status.ptr;
#define YK_C(W)                                                                                 \
    if (g.f32)                                                                                  \
        k_batch<float, W><<<g.grid, 256, g.smem, b->stream>>>(insts, need, items, g.total, head, \
                                                              done, status, b->spin_limit);     \
    else                                                                                        \
        k_batch<double, W><<<g.grid, 256, g.smem, b->stream>>>(insts, need, items, g.total,      \
                                                               head, done, status, b->spin_limit)
    YK_W_SWITCH(g.w, YK_C)
#undef YK_C
}

yk_status build(yk_batch_s *b)
{
    drop_graph(b);
    b->trivial.clear();
    b->trivial_n.clear();
    for (auto &g : b->grp) {
        g.members.clear();
        g.h_inst.clear();
    }
    const int n = (int)b->plans.size();
    b->versions.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        yk_plan_t p = b->plans[i];
        if (!p) return bfail(YK_ERR_ARG, "plan %d is NULL", i);
        if (!p->points_set) return bfail(YK_ERR_STATE, "plan %d has no points (yk_set_points)", i);
        if (p->status != YK_OK) return bfail((yk_status)p->status, "plan %d is in an error state", i);
        if (p->n_dip > 0)
            return bfail(YK_ERR_UNSUPPORTED,
                         "plan %d has dipole sources: batches take charges only "
                         "(use yk_eval_longrange_dl)", i);
        b->versions[i] = p->layout_version;
        Inst d;
        if (!yk_fill_inst(p, &d)) {
            b->trivial.push_back(i);
            b->trivial_n.push_back(p->n_trg);
            continue;
        }
        /* the row passes in items of as many rows as shared memory takes (see rows_per_item) */
        d.rows = yk::rows_per_item(d.n, d.f32 != 0, false);
        for (int s = 0; s < yk::ST_COUNT; ++s) {
            d.items[s] = yk::stage_items(d, s);
            d.smem[s] = yk::stage_smem(d, s);
        }
        Group *gp = nullptr;
        for (Group &g : b->grp)
            if (g.f32 == (d.f32 != 0) && g.w == d.g.w) gp = &g;
        if (!gp) {
            b->grp.emplace_back();
            gp = &b->grp.back();
            gp->f32 = d.f32 != 0;
            gp->w = d.g.w;
        }
        Group &g = *gp;
        g.members.push_back(i);
        g.h_inst.push_back(d);
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bfail(YK_ERR_CUDA, "device query failed");
    for (Group &g : b->grp) {
        const int m = (int)g.members.size();
        if (m == 0) continue;
        /* heavy instances first inside each stage */
        std::vector<int> ord(m);
        for (int k = 0; k < m; ++k) ord[k] = k;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
            return inst_cost(g.h_inst[x]) > inst_cost(g.h_inst[y]);
        });
        std::vector<int2> items;
        std::vector<int> need(m * yk::ST_COUNT, 0);
        g.smem = 0;
        for (int s = 0; s < yk::ST_COUNT; ++s)
            for (int k : ord) {
                const Inst &d = g.h_inst[k];
                for (int idx = 0; idx < d.items[s]; ++idx) items.push_back(make_int2(k, (s << 24) | idx));
                need[k * yk::ST_COUNT + s] = d.items[s];
                g.smem = std::max(g.smem, d.smem[s]);
            }
        if (b->inject_stall) need[0] += 1; /* test hook: instance 0's first stage never "finishes" */
        g.total = (int)items.size();
        cudaError_t e = g.insts.ensure(sizeof(Inst) * m);
        if (e == cudaSuccess) e = g.need.ensure(sizeof(int) * need.size());
        if (e == cudaSuccess) e = g.items.ensure(sizeof(int2) * items.size());
        if (e == cudaSuccess) e = g.done.ensure(sizeof(int) * m * yk::ST_COUNT);
        if (e == cudaSuccess) e = g.head.ensure(sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g.need.ptr, need.data(), sizeof(int) * need.size(),
                                cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g.items.ptr, items.data(), sizeof(int2) * items.size(),
                                cudaMemcpyHostToDevice, b->stream);
        int per_sm = 0;
        if (e == cudaSuccess) e = kernel_setup(g.f32, g.w, g.smem, &per_sm);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(e == cudaErrorMemoryAllocation ? YK_ERR_OOM : YK_ERR_CUDA,
                         "batch set-up: %s", cudaGetErrorString(e));
        }
        g.grid = std::max(1, std::min(g.total, std::max(1, per_sm) * sms));
    }
    if (b->status.ensure(sizeof(int)) != cudaSuccess) return bfail(YK_ERR_OOM, "status word");
    b->last_dens.assign(n, nullptr);
    b->last_u.assign(n, nullptr);
    b->built = true;
    return YK_OK;
}

cudaError_t enqueue(yk_batch_s *b)
{
    cudaError_t e = cudaMemsetAsync(b->status.ptr, 0, sizeof(int), b->stream);
    for (Group &g : b->grp) {
        if (g.members.empty() || e != cudaSuccess) continue;
        e = cudaMemsetAsync(g.done.ptr, 0, sizeof(int) * g.members.size() * yk::ST_COUNT, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(g.head.ptr, 0, sizeof(int), b->stream);
        if (e != cudaSuccess) break;
        launch_group(g, b);
        e = cudaGetLastError();
    }
    return e;
}

bool is_device(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

} /* namespace */

extern "C" {

YK_API void yk_batch_opts_default(yk_batch_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->use_graph = 1;
}

YK_API yk_status yk_batch_create(yk_plan_t *plans, int n, const yk_batch_opts *o, yk_batch_t *out)
{
    if (!out) return bfail(YK_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n <= 0 || !plans) return bfail(YK_ERR_ARG, "need n > 0 plans");
    yk_batch_opts def;
    yk_batch_opts_default(&def);
    if (!o) o = &def;
    if (o->spin_limit < 0) return bfail(YK_ERR_ARG, "spin_limit must be >= 0");
    yk_batch_s *b = new (std::nothrow) yk_batch_s();
    if (!b) return bfail(YK_ERR_OOM, "host allocation failed");
    b->plans.assign(plans, plans + n);
    b->stream = o->stream ? (cudaStream_t)o->stream : (plans[0] ? plans[0]->stream : nullptr);
    if (!b->stream) {
        /* a blocking stream: it still orders with work on the legacy default stream */
        if (cudaStreamCreate(&b->stream) != cudaSuccess) {
            delete b;
            return bfail(YK_ERR_CUDA, "stream creation failed");
        }
        b->own_stream = true;
    }
    b->use_graph = o->use_graph != 0;
    if (o->spin_limit > 0) b->spin_limit = o->spin_limit;
    b->inject_stall = o->inject_stall != 0;
    yk_status s = build(b);
    if (s != YK_OK) {
        yk_batch_destroy(b);
        return s;
    }
    *out = b;
    return YK_OK;
}

YK_API yk_status yk_batch_set_plans(yk_batch_t b, yk_plan_t *plans, int n)
{
    if (!b) return bfail(YK_ERR_ARG, "batch is NULL");
    if (n <= 0 || !plans) return bfail(YK_ERR_ARG, "need n > 0 plans");
    /* the previous run may still read the work list and instance table: let it finish */
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(YK_ERR_CUDA, "batch stream: %s", cudaGetErrorString(e));
    b->plans.assign(plans, plans + n);
    return build(b);
}

YK_API yk_status yk_batch_run(yk_batch_t b, const double *const *density, double *const *u)
{
    if (!b) return bfail(YK_ERR_ARG, "batch is NULL");
    const int n = (int)b->plans.size();
    if (!density || !u) return bfail(YK_ERR_ARG, "density and u arrays are required");
    bool stale = !b->built;
    for (int i = 0; i < n && !stale; ++i) stale = b->plans[i]->layout_version != b->versions[i];
    if (stale) {
        yk_status s = build(b);
        if (s != YK_OK) return s;
    }
    for (int i = 0; i < n; ++i) {
        yk_plan_t p = b->plans[i];
        if ((p->n_src > 0 && !is_device(density[i])) || (p->n_trg > 0 && !is_device(u[i])))
            return bfail(YK_ERR_ARG, "instance %d: density and u must be device memory", i);
    }
    /* refresh density/output pointers of the instances */
    for (Group &g : b->grp) {
        bool changed = false;
        for (size_t k = 0; k < g.members.size(); ++k) {
            const int i = g.members[k];
            if (g.h_inst[k].dens != density[i] || g.h_inst[k].u != u[i]) {
                g.h_inst[k].dens = density[i];
                g.h_inst[k].u = u[i];
                changed = true;
            }
        }
        if (changed && !g.members.empty()) {
            cudaError_t e = cudaMemcpyAsync(g.insts.ptr, g.h_inst.data(),
                                            sizeof(Inst) * g.h_inst.size(),
                                            cudaMemcpyHostToDevice, b->stream);
            if (e != cudaSuccess) return bfail(YK_ERR_CUDA, "instance table: %s", cudaGetErrorString(e));
        }
    }
    for (size_t k = 0; k < b->trivial.size(); ++k)
        if (b->trivial_n[k] > 0) {
            cudaError_t e = cudaMemsetAsync(u[b->trivial[k]], 0, sizeof(double) * b->trivial_n[k],
                                            b->stream);
            if (e != cudaSuccess) return bfail(YK_ERR_CUDA, "zero output: %s", cudaGetErrorString(e));
        }
    cudaError_t e = cudaSuccess;
    if (b->use_graph) {
        if (!b->exec) {
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue(b);
                e = cudaStreamEndCapture(b->stream, &graph);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                cudaGetLastError();
                b->exec = nullptr;
                return bfail(YK_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
            }
        }
        e = cudaGraphLaunch(b->exec, b->stream);
    } else {
        e = enqueue(b);
    }
    if (e != cudaSuccess) return bfail(YK_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
    return YK_OK;
}

YK_API yk_status yk_batch_sync(yk_batch_t b)
{
    if (!b) return bfail(YK_ERR_ARG, "batch is NULL");
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, b->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(YK_ERR_CUDA, "batch sync: %s", cudaGetErrorString(e));
    if (h & yk::ERR_WAIT_TIMEOUT)
        return bfail(YK_ERR_TIMEOUT, "a batch work item waited past its limit for its predecessors");
    return YK_OK;
}

YK_API yk_status yk_batch_destroy(yk_batch_t b)
{
    if (!b) return YK_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (Group &g : b->grp) {
        g.insts.release();
        g.need.release();
        g.items.release();
        g.done.release();
        g.head.release();
    }
    b->status.release();
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return YK_OK;
}

YK_API yk_status yk_batch_eval(yk_plan_t *plans, const double *const *density, double *const *u,
                               int n)
{
    yk_batch_opts o;
    yk_batch_opts_default(&o);
    o.use_graph = 0;
    yk_batch_t b = nullptr;
    yk_status s = yk_batch_create(plans, n, &o, &b);
    if (s == YK_OK) s = yk_batch_run(b, density, u);
    if (s == YK_OK) s = yk_batch_sync(b);
    yk_batch_destroy(b);
    return s;
}

} /* extern "C" */
