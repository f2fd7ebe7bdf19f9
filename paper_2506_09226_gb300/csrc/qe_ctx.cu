// qe_ctx.cu -- context, budgeted allocation, error reporting, and the
// group-table create / compact steps shared by group-by and the pipeline.
#include <cstdio>
#include <cstring>

#include "qe_internal.cuh"

qe_status qe_fail(qe_ctx *ctx, qe_status st, const std::string &msg)
{
    if (ctx) ctx->last_error = msg;
    return st;
}

qe_status qe_cuda_fail(qe_ctx *ctx, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return qe_fail(ctx, QE_ERR_OOM, m);
    return qe_fail(ctx, QE_ERR_CUDA, m);
}

qe_status qe_alloc(qe_ctx *ctx, void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->fail_after > 0 && --ctx->fail_after == 0)
        return qe_fail(ctx, QE_ERR_OOM, "injected allocation failure");
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return qe_fail(ctx, QE_ERR_OOM, "HBM budget exceeded: need " + std::to_string(bytes) + " bytes, " +
                                            std::to_string(ctx->budget - ctx->in_use) + " left");
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return qe_fail(ctx, QE_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    ctx->in_use += bytes;
    ctx->live[*p] = bytes;
    return QE_OK;
}

void qe_free(qe_ctx *ctx, void *p, cudaStream_t s)
{
    if (!p) return;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->live.find(p);
    if (it != ctx->live.end()) {
        ctx->in_use -= it->second;
        ctx->live.erase(it);
    }
    cudaFreeAsync(p, s);
}

extern "C" qe_status qe_create(qe_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) return QE_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return QE_ERR_NO_DEVICE;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return QE_ERR_NO_DEVICE;
    if (!(prop.major == 10 && prop.minor == 3)) return QE_ERR_NO_DEVICE;  // built for sm_103a only
    if (cudaSetDevice(device) != cudaSuccess) return QE_ERR_NO_DEVICE;
    qe_ctx *c = new qe_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;  // keep freed blocks cached in this process
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (cudaMalloc(&c->dstat, sizeof(qe_dev_status)) != cudaSuccess ||
        cudaMallocHost(&c->hstat, sizeof(qe_dev_status)) != cudaSuccess ||
        cudaMemset(c->dstat, 0, sizeof(qe_dev_status)) != cudaSuccess) {
        cudaGetLastError();
        if (c->dstat) cudaFree(c->dstat);
        if (c->hstat) cudaFreeHost(c->hstat);
        delete c;
        return QE_ERR_CUDA;
    }
    *out = c;
    return QE_OK;
}

extern "C" qe_status qe_destroy(qe_ctx *ctx)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    qe_profile_reset(ctx);
    for (auto &kv : ctx->live) cudaFree(kv.first);
    cudaFree(ctx->dstat);
    cudaFreeHost(ctx->hstat);
    delete ctx;
    return QE_OK;
}

extern "C" qe_status qe_set_tuning(qe_ctx *ctx, const char *name, int64_t value)
{
    if (!ctx || !name) return QE_ERR_INVALID_ARG;
    const std::string n(name);
    if (n == "star_items") {
        if (value != 0 && value != 2 && value != 3) return qe_fail(ctx, QE_ERR_INVALID_ARG, "star_items must be 0, 2 or 3");
        ctx->tune_star_items = static_cast<int>(value);
    } else if (n == "force_generic") {
        ctx->tune_force_generic = value != 0;
    } else if (n == "part_general") {
        ctx->tune_part_general = value != 0;
    } else if (n == "part_span") {
        if (value < 0 || value > 1024) return qe_fail(ctx, QE_ERR_INVALID_ARG, "part_span must be in [0, 1024]");
        ctx->tune_part_span = static_cast<int>(value);
    } else if (n == "l2_hint") {
        ctx->tune_l2_hint = value != 0;
    } else if (n == "gb_partition") {
        if (value < 0 || value > 2) return qe_fail(ctx, QE_ERR_INVALID_ARG, "gb_partition must be 0, 1 or 2");
        ctx->tune_gb_partition = static_cast<int>(value);
    } else if (n == "gb_fold2") {
        ctx->tune_gb_fold2 = value != 0;
    } else if (n == "gb_part_log2q") {
        if (value < -1 || value > 8) return qe_fail(ctx, QE_ERR_INVALID_ARG, "gb_part_log2q must be in [-1, 8]");
        ctx->tune_gb_part_log2q = static_cast<int>(value);
    } else if (n == "gb_part_log2p") {
        if (value < 0 || value > 10) return qe_fail(ctx, QE_ERR_INVALID_ARG, "gb_part_log2p must be in [0, 10]");
        ctx->tune_gb_part_log2p = static_cast<int>(value);
    } else if (n == "join_partition") {
        if (value < 0 || value > 2) return qe_fail(ctx, QE_ERR_INVALID_ARG, "join_partition must be 0, 1 or 2");
        ctx->tune_join_partition = static_cast<int>(value);
    } else if (n == "join_part_log2") {
        if (value < 0 || value > 8) return qe_fail(ctx, QE_ERR_INVALID_ARG, "join_part_log2 must be in [0, 8]");
        ctx->tune_join_part_log2 = static_cast<int>(value);
    } else {
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "unknown tuning knob " + n);
    }
    return QE_OK;
}

extern "C" int64_t qe_launch_count(const qe_ctx *ctx) { return ctx ? ctx->launches.load() : 0; }

extern "C" int qe_build_checked(void)
{
#ifdef QE_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" qe_status qe_profile_enable(qe_ctx *ctx, int on)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    ctx->profiling = on != 0;
    return QE_OK;
}

extern "C" qe_status qe_profile_reset(qe_ctx *ctx)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    for (auto &kv : ctx->prof)
        for (auto &ev : kv.second) {
            cudaEventSynchronize(ev.second);
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
    ctx->prof.clear();
    return QE_OK;
}

extern "C" qe_status qe_profile_read(qe_ctx *ctx, const char *name, int64_t *launches, double *total_ms)
{
    if (!ctx || !name || !launches || !total_ms) return QE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    *launches = 0;
    *total_ms = 0;
    auto it = ctx->prof.find(name);
    if (it == ctx->prof.end()) return QE_OK;
    for (auto &ev : it->second) {
        QE_CUDA(ctx, cudaEventSynchronize(ev.second));
        float ms = 0;
        QE_CUDA(ctx, cudaEventElapsedTime(&ms, ev.first, ev.second));
        *total_ms += ms;
        *launches += 1;
    }
    return QE_OK;
}

extern "C" const char *qe_last_error(const qe_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->last_error.c_str();
}

extern "C" size_t qe_bytes_in_use(const qe_ctx *ctx) { return ctx ? ctx->in_use : 0; }

extern "C" void qe_debug_fail_alloc(qe_ctx *ctx, int n)
{
    if (ctx) ctx->fail_after = n;
}

extern "C" void qe_debug_set_spin_limit(qe_ctx *ctx, int64_t iterations)
{
    if (ctx) ctx->spin_limit = iterations > 0 ? iterations : (1 << 22);
}

static const char *status_name(int c)
{
    switch (c) {
    case QE_ERR_CAPACITY: return "output capacity too small";
    case QE_ERR_DUPLICATE_KEY: return "duplicate build key";
    case QE_ERR_RESERVED_KEY: return "key equals the reserved empty-slot marker";
    case QE_ERR_TIMEOUT: return "bounded device wait expired";
    case QE_ERR_INVALID_ARG: return "build key outside the stated range";
    case QE_ERR_DEVICE_CHECK: return "bounds check failed (index + 1 as required)";
    default: return "device error";
    }
}

extern "C" qe_status qe_sync_status(qe_ctx *ctx, void *stream, int64_t *required)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    QE_CUDA(ctx, cudaMemcpyAsync(ctx->hstat, ctx->dstat, sizeof(qe_dev_status), cudaMemcpyDeviceToHost, s));
    QE_CUDA(ctx, cudaStreamSynchronize(s));
    int code = ctx->hstat->code;
    if (required) *required = ctx->hstat->required;
    if (code != 0) {
        QE_CUDA(ctx, cudaMemsetAsync(ctx->dstat, 0, sizeof(qe_dev_status), s));
        QE_CUDA(ctx, cudaStreamSynchronize(s));
        return qe_fail(ctx, static_cast<qe_status>(code),
                       std::string(status_name(code)) + " (required " + std::to_string(ctx->hstat->required) + ")");
    }
    return QE_OK;
}

// ------------------------------------------------------------ group tables

// Index of the COUNT aggregate (the divisor of derived averages), or -1.
int agg_count_index(const AggOps &ops)
{
    for (int a = 0; a < ops.n; a++)
        if (ops.op[a] == QE_COUNT) return a;
    return -1;
}

qe_status gt_check_out(qe_ctx *ctx, const qe_groups_out *out, const AggOps &ops)
{
    if (!out || out->capacity < 0 || !out->ngroups) return qe_fail(ctx, QE_ERR_INVALID_ARG, "bad group output");
    if (out->capacity > 0 && !out->keys) return qe_fail(ctx, QE_ERR_INVALID_ARG, "group output keys missing");
    for (int a = 0; a < ops.n; a++)
        if (out->capacity > 0 && !out->aggs[a]) return qe_fail(ctx, QE_ERR_INVALID_ARG, "group output aggs missing");
    // derived averages: over a SUM, with a COUNT among the aggregates
    for (int a = 0; a < QE_MAX_AGGS; a++) {
        if (!out->avg[a]) continue;
        if (a >= ops.n || ops.op[a] != QE_SUM)
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "group output: an average needs a SUM aggregate");
        if (agg_count_index(ops) < 0)
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "group output: an average needs a COUNT aggregate");
    }
    return QE_OK;
}

qe_status gt_create(qe_ctx *ctx, int64_t capacity, int naggs, GroupTableHost &t, cudaStream_t s)
{
    uint64_t want = static_cast<uint64_t>(capacity > 32 ? capacity : 32) * 2;
    uint64_t slots = 64;
    while (slots < want) slots <<= 1;
    t.slots = slots;
    t.stride = 1 + naggs;
    // table words, then a reserved word and the count of groups emitted
    t.bytes = (slots * t.stride + 2) * sizeof(unsigned long long);
    void *p = nullptr;
    qe_status st = qe_alloc(ctx, &p, t.bytes, s);
    if (st != QE_OK) return st;
    t.words = static_cast<unsigned long long *>(p);
    QE_CUDA(ctx, cudaMemsetAsync(t.words, 0, t.bytes, s));
    return QE_OK;
}

struct CompactArgs {
    const unsigned long long *words;
    uint64_t slots;
    int stride;
    int cnt;             // index of the COUNT aggregate (averages), or -1
    AggOps ops;
    qe_groups_out out;
    unsigned long long *emitted;
};

__global__ void __launch_bounds__(256) k_gt_compact(CompactArgs A)
{
    const int lane = threadIdx.x & 31;
    const uint64_t step = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * blockDim.x; base < A.slots; base += step) {
        uint64_t i = base + threadIdx.x;
        unsigned long long kx = i < A.slots ? A.words[i * A.stride] : 0ull;
        unsigned m = __ballot_sync(QE_FULL_MASK, kx != 0);
        if (!m) continue;
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(A.emitted, static_cast<unsigned long long>(__popc(m)));
        first = __shfl_sync(QE_FULL_MASK, first, 0);
        if (kx != 0) {
            int64_t pos = static_cast<int64_t>(first) + __popc(m & ((1u << lane) - 1));
            if (pos < A.out.capacity) {
                A.out.keys[pos] = static_cast<int64_t>(kx ^ GB_SIGN);
                _Pragma("unroll") for (int a = 0; a < QE_MAX_AGGS; a++) if (a < A.ops.n)
                    A.out.aggs[a][pos] = agg_decode(A.ops.op[a], A.words[i * A.stride + 1 + a]);
                if (A.cnt >= 0)
                    write_avgs(A.out, pos, A.ops.n, A.cnt, [&](int a) { return agg_decode(A.ops.op[a], A.words[i * A.stride + 1 + a]); });
            }
        }
    }
}

__global__ void k_gt_count(const unsigned long long *emitted, int64_t capacity, int64_t *ngroups,
                           qe_dev_status *st)
{
    int64_t n = static_cast<int64_t>(*emitted);
    *ngroups = n;
    if (n > capacity) dev_report(st, QE_ERR_CAPACITY, n);
}

struct DenseCompactArgs {
    const unsigned long long *dense;
    DenseKey d;
    int cnt;             // index of the COUNT aggregate (averages), or -1
    AggOps ops;
    qe_groups_out out;
    unsigned long long *emitted;
};

__global__ void __launch_bounds__(256) k_gd_compact(DenseCompactArgs A)
{
    const int lane = threadIdx.x & 31;
    const uint64_t step = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * blockDim.x; base < A.d.nslots; base += step) {
        const uint64_t i = base + threadIdx.x;
        const bool occ = i < A.d.nslots && A.dense[i * A.d.stride + A.d.occ] != 0;
        const unsigned m = __ballot_sync(QE_FULL_MASK, occ);
        if (!m) continue;
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(A.emitted, static_cast<unsigned long long>(__popc(m)));
        first = __shfl_sync(QE_FULL_MASK, first, 0);
        if (occ) {
            const int64_t pos = static_cast<int64_t>(first) + __popc(m & ((1u << lane) - 1));
            if (pos < A.out.capacity) {
                A.out.keys[pos] = dense_key(A.d, i);
                for (int a = 0; a < A.ops.n; a++)
                    A.out.aggs[a][pos] = agg_decode(A.ops.op[a], A.dense[i * A.d.stride + a]);
                if (A.cnt >= 0)
                    write_avgs(A.out, pos, A.ops.n, A.cnt, [&](int a) { return agg_decode(A.ops.op[a], A.dense[i * A.d.stride + a]); });
            }
        }
    }
}

qe_status gt_finalize_dense(qe_ctx *ctx, const GroupTableHost &t, const AggOps &ops, const DenseKey &d,
                            const unsigned long long *dense, const qe_groups_out *out, cudaStream_t s)
{
    DenseCompactArgs A;
    A.dense = dense;
    A.d = d;
    A.cnt = agg_count_index(ops);
    A.ops = ops;
    A.out = *out;
    A.emitted = t.words + t.slots * t.stride + 1;
    int64_t blocks = qe_ceil_div(static_cast<int64_t>(d.nslots), 256);
    const int64_t cap = static_cast<int64_t>(ctx->num_sms) * 8;
    if (blocks > cap) blocks = cap;
    k_gd_compact<<<static_cast<unsigned>(blocks), 256, 0, s>>>(A);
    QE_LAUNCHED(ctx);
    QE_CHECK_LAUNCH(ctx);
    return gt_finalize(ctx, t, ops, out, s);
}

qe_status gt_finalize(qe_ctx *ctx, const GroupTableHost &t, const AggOps &ops, const qe_groups_out *out,
                      cudaStream_t s)
{
    CompactArgs A;
    A.words = t.words;
    A.slots = t.slots;
    A.stride = t.stride;
    A.cnt = agg_count_index(ops);
    A.ops = ops;
    A.out = *out;
    A.emitted = t.words + t.slots * t.stride + 1;
    int64_t blocks = qe_ceil_div(static_cast<int64_t>(t.slots), 256);
    int64_t cap = static_cast<int64_t>(ctx->num_sms) * 8;
    k_gt_compact<<<static_cast<unsigned>(blocks < cap ? blocks : cap), 256, 0, s>>>(A);
    QE_LAUNCHED(ctx);
    QE_CHECK_LAUNCH(ctx);
    k_gt_count<<<1, 1, 0, s>>>(A.emitted, out->capacity, out->ngroups, ctx->dstat);
    QE_LAUNCHED(ctx);
    QE_CHECK_LAUNCH(ctx);
    return QE_OK;
}
