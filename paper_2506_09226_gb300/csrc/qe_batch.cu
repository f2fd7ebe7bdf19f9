// qe_batch.cu -- many pipelines in one persistent launch.
//
// The batched form runs thousands of pipelines of uneven size (each one
// group-by(join(filter(fact), dim)), Sec. 2.4) as work items of a single
// persistent kernel, captured with the table clearing in one CUDA graph:
//   - build items insert a slice of one pipeline's dimension rows into its
//     dense join table;
//   - probe items run a slice of one pipeline's fact rows through the fused
//     filter / probe / aggregate path into a per-block shared-memory group
//     table, flushed into the pipeline's HBM tables at the end of the item;
//   - the block that finishes a pipeline's last probe item compacts that
//     pipeline's groups into its output.
// Blocks claim items in order from one atomic counter; a pipeline's build
// items are placed a little ahead of its probe items (so its table is still
// in L2 when probed) and always before them, so a probe item waits (bounded,
// QE_ERR_TIMEOUT on expiry) only for builds that running blocks already hold.
// Tables built inside the kernel are read with L2-only loads.
#include <vector>

#include "qe_pipe_core.cuh"

qe_status pipeline_prepare(qe_ctx *ctx, const qe_pipeline_desc *d, PipeSpec &P);

namespace {

constexpr int BT = 1024;            // threads per block
constexpr int B_ITEMS = 2;          // rows per thread per tile
constexpr int BUILD_ROWS = 1 << 16; // dimension rows per build item

struct BatchItem {
    int32_t pipe;
    int32_t kind;                   // 0 build: dimension rows [row0, row1)
    int64_t row0, row1;             // 1 probe: item row0 of the pipeline's nprobe, over fact rows [0, row1)
};

struct BatchPipe {
    PipeSpec P;
    TableCfg T;
    int32_t nbuild, nprobe;
    const int32_t *dim_key, *dim_pay;  // build source (in-kernel build)
    int32_t *ht_pay;                   // writable dense join table
    uint32_t *ht_bm;
    qe_groups_out out;
    unsigned long long *emitted;       // groups written to `out`
    unsigned *build_done, *probe_done;
    uint64_t hslots;                   // HBM hash table slots
    int32_t star;                      // star kind + 1 (0: the generic row loop)
    int32_t cnt;                       // COUNT aggregate of derived averages, or -1
};

static_assert(sizeof(PipeSpec) % 4 == 0, "the spec is copied to shared memory in 4-byte words");

struct BatchArgs {
    const BatchPipe *pipes;
    const BatchItem *items;
    int64_t nitems;
    unsigned long long *counter;
    int64_t spin_limit;
    qe_dev_status *st;
};

__device__ void batch_build(const BatchPipe &B, const BatchItem &I, qe_dev_status *st)
{
    const HtView &h = B.P.ht;
    // BB_ROWS rows per thread and step: their bitmap atomics (whose old value
    // decides whether the payload is written) are in flight together
    constexpr int BB_ROWS = 4;
    for (int64_t r0 = I.row0 + threadIdx.x; r0 < I.row1; r0 += BT * BB_ROWS) {
        uint32_t sl[BB_ROWS], old[BB_ROWS];
        int32_t v[BB_ROWS];
#pragma unroll
        for (int j = 0; j < BB_ROWS; j++) {
            const int64_t r = r0 + j * BT;
            sl[j] = r < I.row1 ? static_cast<uint32_t>(__ldcs(B.dim_key + r)) - static_cast<uint32_t>(h.key_min)
                               : 0xffffffffu;
            v[j] = r < I.row1 && B.ht_pay ? __ldcs(B.dim_pay + r) : 0;
        }
#pragma unroll
        for (int j = 0; j < BB_ROWS; j++) {
            old[j] = 0;
            if (sl[j] < h.range) old[j] = atomicOr(B.ht_bm + (sl[j] >> 5), 1u << (sl[j] & 31));
        }
#pragma unroll
        for (int j = 0; j < BB_ROWS; j++) {
            if (r0 + j * BT >= I.row1) continue;
            if (sl[j] >= h.range) {
                dev_report(st, QE_ERR_INVALID_ARG, 0);
                continue;
            }
            if (!B.ht_pay) continue;          // a key set (semi- or anti-join): repeats are fine
            if ((old[j] >> (sl[j] & 31)) & 1u) {
                dev_report(st, QE_ERR_DUPLICATE_KEY, 0);
                continue;
            }
            B.ht_pay[sl[j]] = v[j];
        }
    }
}

// Compact one pipeline's groups (HBM dense table, then the hash table) into
// its output.  Runs in the block that finished the pipeline's last item;
// other blocks' updates are read through L2.
__device__ void batch_finalize(const BatchPipe &B, qe_dev_status *st)
{
    const PipeSpec &P = B.P;
    const int lane = threadIdx.x & 31;
    if (P.gdense) {
        const uint64_t ns = P.dk.nslots;
        for (uint64_t base = 0; base < ns; base += BT) {
            const uint64_t i = base + threadIdx.x;
            const bool occ = i < ns && __ldcg(P.gdense + i * P.dk.stride + P.dk.occ) != 0;
            const unsigned m = __ballot_sync(QE_FULL_MASK, occ);
            if (!m) continue;
            unsigned long long first = 0;
            if (lane == 0) first = atomicAdd(B.emitted, static_cast<unsigned long long>(__popc(m)));
            first = __shfl_sync(QE_FULL_MASK, first, 0);
            if (occ) {
                const int64_t pos = static_cast<int64_t>(first) + __popc(m & ((1u << lane) - 1));
                if (pos < B.out.capacity) {
                    B.out.keys[pos] = dense_key(P.dk, i);
                    for (int a = 0; a < P.ops.n; a++)
                        B.out.aggs[a][pos] = agg_decode(P.ops.op[a], __ldcg(P.gdense + i * P.dk.stride + a));
                    if (B.cnt >= 0)
                        write_avgs(B.out, pos, P.ops.n, B.cnt,
                                   [&](int a) { return agg_decode(P.ops.op[a], __ldcg(P.gdense + i * P.dk.stride + a)); });
                }
            }
        }
    }
    for (uint64_t base = 0; base < B.hslots; base += BT) {
        const uint64_t i = base + threadIdx.x;
        const unsigned long long kx = i < B.hslots ? __ldcg(P.g.words + i * P.g.stride) : 0ull;
        const unsigned m = __ballot_sync(QE_FULL_MASK, kx != 0);
        if (!m) continue;
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(B.emitted, static_cast<unsigned long long>(__popc(m)));
        first = __shfl_sync(QE_FULL_MASK, first, 0);
        if (kx != 0) {
            const int64_t pos = static_cast<int64_t>(first) + __popc(m & ((1u << lane) - 1));
            if (pos < B.out.capacity) {
                B.out.keys[pos] = static_cast<int64_t>(kx ^ GB_SIGN);
                for (int a = 0; a < P.ops.n; a++)
                    B.out.aggs[a][pos] = agg_decode(P.ops.op[a], __ldcg(P.g.words + i * P.g.stride + 1 + a));
                if (B.cnt >= 0)
                    write_avgs(B.out, pos, P.ops.n, B.cnt,
                               [&](int a) { return agg_decode(P.ops.op[a], __ldcg(P.g.words + i * P.g.stride + 1 + a)); });
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t n = static_cast<int64_t>(atomicAdd(B.emitted, 0ull));
        *B.out.ngroups = n;
        if (n > B.out.capacity) dev_report(st, QE_ERR_CAPACITY, n);
    }
}

// The row paths of a probe item, each out of line so that each gets its own
// register allocation.  Item j of a pipeline's m probe items takes the tiles
// j, j + m, j + 2m, ... of its fact rows [0, n), one tile per call: the blocks
// working on one pipeline read neighbouring tiles at any moment.  Measured on
// GB300 this beats contiguous item ranges (4.39 vs 4.79 ms for 300 pipelines
// of 1K-10M rows, 4.85 vs 5.48 ms for one of 400M rows) and also one strided
// pass that prefetches the next tile across the stride (4.67 / 5.32 ms).
constexpr int64_t STAR_TR = static_cast<int64_t>(BT) * 3;

template <int JK>
__device__ __noinline__ void item_star_smem(const PipeSpec &P, unsigned long long *sm, int64_t j, int64_t m, int64_t n)
{
    for (int64_t t = j * STAR_TR; t < n; t += m * STAR_TR)
        star_range<false, 3, BT, true, JK>(P, sm, t, t + STAR_TR < n ? t + STAR_TR : n, STAR_TR);
}

template <int JK>
__device__ __noinline__ void item_star_global(const PipeSpec &P, unsigned long long *sm, int64_t j, int64_t m,
                                              int64_t n)
{
    for (int64_t t = j * STAR_TR; t < n; t += m * STAR_TR)
        star_range<true, 3, BT, false, JK>(P, sm, t, t + STAR_TR < n ? t + STAR_TR : n, STAR_TR);
}

// A star item of kind JK: the direct array in shared memory or in HBM.
template <int JK>
__device__ __forceinline__ void item_star(const PipeSpec &P, const TableCfg &T, unsigned long long *sm, int64_t j,
                                          int64_t m, int64_t n)
{
    if (T.mode == TM_SMEM_DENSE) item_star_smem<JK>(P, sm, j, m, n);
    else item_star_global<JK>(P, sm, j, m, n);
}

__device__ __noinline__ void item_generic(const PipeSpec &P, const TableCfg T, unsigned long long *sm, int64_t j,
                                          int64_t m, int64_t r1)
{
    constexpr int TR = BT * B_ITEMS;
    for (int64_t t0 = j * TR; t0 < r1; t0 += m * TR) {
        RowVals v[B_ITEMS];
#pragma unroll
        for (int k = 0; k < B_ITEMS; k++) {
            const int64_t r = t0 + k * BT + threadIdx.x;
            v[k] = row_load(P, r, r < r1);
        }
        int64_t hi[B_ITEMS], lo[B_ITEMS];
        bool ok[B_ITEMS];
#pragma unroll
        for (int k = 0; k < B_ITEMS; k++) ok[k] = row_probe(P, v[k], hi[k], lo[k]);
#pragma unroll
        for (int k = 0; k < B_ITEMS; k++)
            if (ok[k]) fold_row(P, T, sm, hi[k], lo[k], v[k]);
    }
}

__global__ void __launch_bounds__(BT, 1) k_batch(BatchArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *sm = reinterpret_cast<unsigned long long *>(smem);
    __shared__ long long s_item;
    __shared__ int s_flag;
    // the current item's pipeline spec, read by the row loop as shared-memory
    // broadcasts instead of global loads
    __shared__ __align__(16) unsigned char s_spec_raw[sizeof(PipeSpec)];
    const PipeSpec &SP = *reinterpret_cast<const PipeSpec *>(s_spec_raw);
    while (true) {
        if (threadIdx.x == 0) s_item = static_cast<long long>(atomicAdd(A.counter, 1ull));
        __syncthreads();
        const int64_t it = s_item;
        if (it >= A.nitems) break;
        const BatchItem I = A.items[it];
        const BatchPipe &B = A.pipes[I.pipe];
        if (I.kind == 0) {
            batch_build(B, I, A.st);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(B.build_done, 1u);
            }
            continue;
        }
        if (threadIdx.x == 0) {
            s_flag = 0;
            if (B.nbuild > 0) {
                int64_t spins = 0;
                while (*reinterpret_cast<volatile unsigned *>(B.build_done) < static_cast<unsigned>(B.nbuild)) {
                    if (++spins > A.spin_limit) {
                        dev_report(A.st, QE_ERR_TIMEOUT, 0);
                        s_flag = 1;
                        break;
                    }
                    __nanosleep(64);
                }
                __threadfence();
            }
        }
        {
            const unsigned *src = reinterpret_cast<const unsigned *>(&B.P);
            unsigned *dst = reinterpret_cast<unsigned *>(s_spec_raw);
            for (int i = threadIdx.x; i < static_cast<int>(sizeof(PipeSpec) / 4); i += BT) dst[i] = src[i];
        }
        __syncthreads();
        const PipeSpec &P = SP;
        const TableCfg T = B.T;
        if (!s_flag) {
            table_zero(P, T, sm);
            __syncthreads();
            switch (B.star) {
            case 1 + STAR_INNER: item_star<STAR_INNER>(P, T, sm, I.row0, B.nprobe, I.row1); break;
            case 1 + STAR_SEMI: item_star<STAR_SEMI>(P, T, sm, I.row0, B.nprobe, I.row1); break;
            case 1 + STAR_ANTI: item_star<STAR_ANTI>(P, T, sm, I.row0, B.nprobe, I.row1); break;
            case 1 + STAR_NONE: item_star<STAR_NONE>(P, T, sm, I.row0, B.nprobe, I.row1); break;
            default: item_generic(P, T, sm, I.row0, B.nprobe, I.row1);
            }
            __syncthreads();
            table_flush(P, T, sm, B.star ? 2 : 0);   // star items: 32-bit COUNT and SUM halves
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_flag = atomicAdd(B.probe_done, 1u) == static_cast<unsigned>(B.nprobe) - 1;
        }
        __syncthreads();
        if (s_flag) batch_finalize(B, A.st);
        __syncthreads();
    }
}

}  // namespace

struct qe_batch {
    int n = 0;
    std::vector<BatchPipe> host_pipes;   // sources of the uploads, alive until destroy
    std::vector<BatchItem> host_items;
    void *arena = nullptr;          // library-owned device memory
    size_t arena_bytes = 0;
    size_t zero_off = 0, zero_bytes = 0;
    BatchArgs args{};
    size_t smem = 0;
    unsigned grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static qe_status batch_enqueue(qe_ctx *ctx, qe_batch *b, cudaStream_t s)
{
    QE_CUDA(ctx, cudaMemsetAsync(static_cast<char *>(b->arena) + b->zero_off, 0, b->zero_bytes, s));
    {
        ProfScope prof(ctx, "batch", s);
        k_batch<<<b->grid, BT, b->smem, s>>>(b->args);
        QE_LAUNCHED(ctx);
    }
    QE_CHECK_LAUNCH(ctx);
    return QE_OK;
}

extern "C" qe_status qe_batch_create(qe_ctx *ctx, const qe_pipeline_desc *descs, const qe_groups_out *outs, int n,
                                     const qe_batch_opts *opts, qe_batch **out, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!descs || !outs || !out || n <= 0) return qe_fail(ctx, QE_ERR_INVALID_ARG, "batch: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qe_batch_opts o{};
    if (opts) o = *opts;
    const int64_t item_rows = o.tile_rows > 0 ? o.tile_rows : (1 << 16);
    if (item_rows % (BT * B_ITEMS) != 0)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "batch: tile_rows must be a multiple of 2048");
    const size_t budget = ctx->smem_optin > 1024 ? ctx->smem_optin - 1024 : 0;
    const size_t smem_cap = o.smem_slots < 0 ? 0 : budget;   // smem_slots < 0: HBM tables only
    cudaSetDevice(ctx->device);

    std::vector<BatchPipe> pipes(n);
    std::vector<BatchItem> items;
    // arena layout: [non-zeroed: dense join payloads][zeroed: join bitmaps,
    // dense group tables, hash tables + counters, done counters, item counter]
    struct Sizes {
        size_t pay = 0, bm = 0, gd = 0, gh = 0;
    };
    std::vector<Sizes> sz(n);
    size_t nz_bytes = 0, z_bytes = 0;
    size_t max_table = 0;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    for (int i = 0; i < n; i++) {
        const qe_pipeline_desc &d = descs[i];
        BatchPipe &B = pipes[i];
        qe_status st = pipeline_prepare(ctx, &d, B.P);
        if (st != QE_OK) return st;
        st = gt_check_out(ctx, &outs[i], B.P.ops);
        if (st != QE_OK) return st;
        B.out = outs[i];
        B.cnt = -1;
        for (int a = 0; a < QE_MAX_AGGS; a++)
            if (B.out.avg[a]) B.cnt = agg_count_index(B.P.ops);
        int64_t pay_min = 1, pay_max = 0;
        if (B.P.has_join) {
            const bool inner = B.P.join_kind == QE_JOIN_INNER;
            if (d.ht) {
                if (d.ht->multi || d.ht->pair)
                    return qe_fail(ctx, QE_ERR_INVALID_ARG,
                                   "batch: pipeline " + std::to_string(i) + ": a multimap or pair-key table is not a pipeline table");
                if (inner && d.ht->set)
                    return qe_fail(ctx, QE_ERR_INVALID_ARG,
                                   "batch: pipeline " + std::to_string(i) + ": an inner join needs a table with payloads");
                B.P.ht = ht_view(d.ht);
                if (d.ht->have_pay) {
                    pay_min = d.ht->pay_min;
                    pay_max = d.ht->pay_max;
                }
            } else {
                if (!d.build.have_range || d.n_dim < 0 || (d.n_dim > 0 && (!d.dim_key || (inner && !d.dim_payload))))
                    return qe_fail(ctx, QE_ERR_INVALID_ARG,
                                   "batch: pipeline " + std::to_string(i) + " needs a prebuilt table or a key range");
                const uint64_t range = static_cast<uint64_t>(static_cast<int64_t>(d.build.key_max) - d.build.key_min + 1);
                if (d.build.key_min > d.build.key_max || range >= (1ull << 31))
                    return qe_fail(ctx, QE_ERR_INVALID_ARG, "batch: bad dimension key range");
                B.dim_key = d.dim_key;
                B.dim_pay = d.dim_payload;
                B.P.ht = HtView{};
                B.P.ht.layout = QE_HT_DENSE;
                B.P.ht.key_min = d.build.key_min;
                B.P.ht.range = static_cast<uint32_t>(range);
                B.P.ht.full = inner && static_cast<uint64_t>(d.n_dim) == range ? 1 : 0;
                B.P.ht.coherent = 1;
                sz[i].pay = inner ? up(range * 4) : 0;      // a key set is its bitmap alone
                sz[i].bm = up(((range + 31) / 32) * 4);
                B.nbuild = static_cast<int32_t>(qe_ceil_div(d.n_dim, BUILD_ROWS));
            }
        }
        // group tables: dense when the key ranges are known
        const bool has_hi = B.P.hi_slot >= 0;
        int64_t lo_min = d.have_key_range ? d.key_lo_min : 1, lo_max = d.have_key_range ? d.key_lo_max : 0;
        if (lo_min > lo_max && B.P.lo_slot == QE_JOIN_PAYLOAD) {
            lo_min = pay_min;
            lo_max = pay_max;
        }
        B.P.dk = DenseKey{};
        if (lo_min <= lo_max && (!has_hi || d.have_key_range))
            B.P.dk = dense_plan(has_hi, d.key_hi_min, d.key_hi_max, lo_min, lo_max, B.P.ops, uint64_t(1) << 24);
        B.T = TableCfg{};
        if (B.P.dk.on) {
            const size_t tb = B.P.dk.nslots * B.P.dk.stride * 8;
            B.T.mode = tb <= smem_cap ? TM_SMEM_DENSE : TM_GLOBAL_DENSE;
            if (B.T.mode == TM_SMEM_DENSE && tb > max_table) max_table = tb;
            sz[i].gd = up(tb);
        } else {
            const int64_t groups = d.expected_groups > 0 ? d.expected_groups : outs[i].capacity;
            const int S = o.smem_slots < 0 ? 0 : st_slots_for(groups, B.P.ops.n, smem_cap);
            if (S) {
                B.T.mode = TM_SMEM_HASH;
                B.T.S = S;
                while ((1 << B.T.log2S) < S) B.T.log2S++;
                const size_t tb = static_cast<size_t>(S) * 8 * (1 + B.P.ops.n);
                if (tb > max_table) max_table = tb;
            } else {
                B.T.mode = TM_GLOBAL_HASH;
            }
        }
        B.star = ctx->tune_force_generic ? 0 : 1 + star_kind(B.P, B.T);
        if (B.star) star_predicate(B.P);
        uint64_t hs = 64;
        while (hs < static_cast<uint64_t>(2 * (outs[i].capacity > 32 ? outs[i].capacity : 32))) hs <<= 1;
        B.hslots = hs;
        sz[i].gh = up((hs * (1 + B.P.ops.n) + 2) * 8);
        nz_bytes += sz[i].pay;
        z_bytes += sz[i].bm + sz[i].gd + sz[i].gh;
        B.nprobe = static_cast<int32_t>(qe_ceil_div(d.n_fact, item_rows));
        if (B.nprobe == 0) B.nprobe = 1;   // one empty item still finalizes
    }
    const size_t counters_off = z_bytes;
    z_bytes += up(static_cast<size_t>(n) * 2 * sizeof(unsigned)) + 256;
    // Item order.  Build items run ahead of their pipeline's probe items by
    // at most `ahead` bytes of join tables built but not yet probed (and at
    // least one pipeline), so a table is probed while it still sits in L2
    // instead of being written to and read back from DRAM: with every build
    // first, 10,000 small tables would all be evicted before any probe.
    // Every build item of a pipeline precedes its probe items, so a probe
    // item waits only for items claimed before it.
    auto push_builds = [&](int i) {
        for (int j = 0; j < pipes[i].nbuild; j++) {
            const int64_t r0 = static_cast<int64_t>(j) * BUILD_ROWS;
            items.push_back({i, 0, r0, std::min<int64_t>(descs[i].n_dim, r0 + BUILD_ROWS)});
        }
    };
    const size_t ahead = o.build_ahead_bytes > 0 ? static_cast<size_t>(o.build_ahead_bytes) : (size_t(32) << 20);
    int next_build = 0;
    size_t pending = 0;             // table bytes built and not yet probed
    for (int i = 0; i < n; i++) {
        while (next_build < n && (next_build <= i || pending + sz[next_build].pay + sz[next_build].bm <= ahead)) {
            push_builds(next_build);
            pending += sz[next_build].pay + sz[next_build].bm;
            next_build++;
        }
        for (int j = 0; j < pipes[i].nprobe; j++) items.push_back({i, 1, j, descs[i].n_fact});
        pending -= sz[i].pay + sz[i].bm;
    }
    const size_t pipes_bytes = up(sizeof(BatchPipe) * n), items_bytes = up(sizeof(BatchItem) * items.size());

    qe_batch *b = new qe_batch();
    b->n = n;
    b->arena_bytes = nz_bytes + z_bytes + pipes_bytes + items_bytes;
    qe_status st = qe_alloc(ctx, &b->arena, b->arena_bytes, s);
    if (st != QE_OK) {
        delete b;
        return st;
    }
    char *base = static_cast<char *>(b->arena);
    b->zero_off = nz_bytes;
    b->zero_bytes = z_bytes;
    size_t nzo = 0, zo = nz_bytes;
    for (int i = 0; i < n; i++) {
        BatchPipe &B = pipes[i];
        if (sz[i].pay) {
            B.ht_pay = reinterpret_cast<int32_t *>(base + nzo);
            nzo += sz[i].pay;
            B.P.ht.payload = B.ht_pay;
        }
        if (sz[i].bm) {
            B.ht_bm = reinterpret_cast<uint32_t *>(base + zo);
            zo += sz[i].bm;
            B.P.ht.bitmap = B.ht_bm;
        }
        if (sz[i].gd) {
            B.P.gdense = B.T.mode == TM_GLOBAL_DENSE || B.T.mode == TM_SMEM_DENSE
                             ? reinterpret_cast<unsigned long long *>(base + zo)
                             : nullptr;
            zo += sz[i].gd;
        }
        unsigned long long *gh = reinterpret_cast<unsigned long long *>(base + zo);
        zo += sz[i].gh;
        B.P.g.words = gh;
        B.P.g.mask = B.hslots - 1;
        B.P.g.stride = 1 + B.P.ops.n;
        B.P.g.capacity = B.out.capacity;
        B.P.g.st = ctx->dstat;
        B.emitted = gh + B.hslots * B.P.g.stride + 1;
        B.build_done = reinterpret_cast<unsigned *>(base + nz_bytes + counters_off) + 2 * i;
        B.probe_done = B.build_done + 1;
    }
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(
        base + nz_bytes + counters_off + up(static_cast<size_t>(n) * 2 * sizeof(unsigned)));
    BatchPipe *dpipes = reinterpret_cast<BatchPipe *>(base + nz_bytes + z_bytes);
    BatchItem *ditems = reinterpret_cast<BatchItem *>(base + nz_bytes + z_bytes + pipes_bytes);
    b->host_pipes = std::move(pipes);
    b->host_items = std::move(items);
    cudaError_t e = cudaMemcpyAsync(dpipes, b->host_pipes.data(), sizeof(BatchPipe) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ditems, b->host_items.data(), sizeof(BatchItem) * b->host_items.size(),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        qe_free(ctx, b->arena, s);
        delete b;
        return qe_cuda_fail(ctx, e, "batch: upload");
    }
    b->args.pipes = dpipes;
    b->args.items = ditems;
    b->args.nitems = static_cast<int64_t>(b->host_items.size());
    b->args.counter = counter;
    b->args.spin_limit = ctx->spin_limit;
    b->args.st = ctx->dstat;
    b->smem = max_table;
    b->grid = static_cast<unsigned>(ctx->num_sms);
    e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(b->smem));
    if (e == cudaSuccess && o.use_graph) {
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaMemsetAsync(static_cast<char *>(b->arena) + b->zero_off, 0, b->zero_bytes, cs);
                k_batch<<<b->grid, BT, b->smem, cs>>>(b->args);
                e = cudaStreamEndCapture(cs, &b->graph);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            cudaStreamDestroy(cs);
        }
    }
    if (e != cudaSuccess) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        qe_free(ctx, b->arena, s);
        delete b;
        return qe_cuda_fail(ctx, e, "batch: graph");
    }
    *out = b;
    return QE_OK;
}

extern "C" qe_status qe_batch_launch(qe_ctx *ctx, qe_batch *batch, void *stream)
{
    if (!ctx || !batch) return QE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (batch->exec) {
        ProfScope prof(ctx, "batch", s);
        QE_CUDA(ctx, cudaGraphLaunch(batch->exec, s));
        QE_LAUNCHED(ctx);
        return QE_OK;
    }
    return batch_enqueue(ctx, batch, s);
}

extern "C" qe_status qe_batch_destroy(qe_ctx *ctx, qe_batch *batch, void *stream)
{
    if (!ctx || !batch) return QE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the host arrays back the uploads issued at create time
    cudaStreamSynchronize(s);
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    qe_free(ctx, batch->arena, s);
    delete batch;
    return QE_OK;
}

extern "C" qe_status qe_batch_run(qe_ctx *ctx, const qe_pipeline_desc *descs, const qe_groups_out *outs, int n,
                                  const qe_batch_opts *opts, void *stream)
{
    qe_batch *b = nullptr;
    qe_batch_opts o{};
    if (opts) o = *opts;
    o.use_graph = 0;
    qe_status st = qe_batch_create(ctx, descs, outs, n, &o, &b, stream);
    if (st != QE_OK) return st;
    st = qe_batch_launch(ctx, b, stream);
    qe_status st2 = qe_batch_destroy(ctx, b, stream);
    return st != QE_OK ? st : st2;
}
