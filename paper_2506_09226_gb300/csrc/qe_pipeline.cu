// qe_pipeline.cu -- the fused per-GPU operator pipeline (Sec. 2.4: each GPU
// runs one program over its local columns): group-by(join(filter(fact), dim)).
//
// After the dimension table is built (qe_join.cu), one persistent kernel,
// one 1024-thread block per SM, makes a single pass over the fact columns.
// Each thread owns ITEMS rows of a tile, 1024 rows apart, so every column
// read is a coalesced warp access; per row it evaluates the predicates,
// probes the join table (dense tables: one L2 read, the table staying
// resident while the fact columns stream through with an evict-first hint)
// and folds the row into the block's group table (additive aggregates as
// reductions, MIN/MAX as max over an order-preserving code).  Blocks merge
// their tables into the HBM tables at the end and the HBM tables are
// compacted into the output.
//
// Group tables, by preference: a direct (perfect-hash) array when the key's
// parts have known small ranges, in shared memory or else in HBM; a hash
// table in shared memory; a hash table in HBM.  Keys outside a direct
// array's range go to the HBM hash table.
//
// The star shape (one int32 predicate, [SUM(x*y), COUNT, MIN(x), MAX(x)]
// and a direct group array, with the key (column, join payload) of a dense
// inner join, or a key of fact columns with a dense semi- / anti-join or no
// join) has its own kernel: all columns of the next tile are loaded into
// registers while the current tile is processed, which keeps about 100 KB of
// loads in flight per SM from the register file.  (A variant that staged tiles in shared memory with
// bulk TMA copies ran at half this speed: the stages shared the 227 KB with
// the group table and a stage could only be refilled once every warp had
// read it.)
//
// Aggregate values are drawn from at most two fact columns X and Y (each
// aggregate is X, Y or X*Y); other shapes are rejected with
// QE_ERR_INVALID_ARG.
#include <climits>
#include <cstdlib>

#include "qe_pipe_core.cuh"

namespace {

constexpr int PT = 1024;          // threads per block (one block per SM)

// Generic pass: any column types, predicates and aggregate plan.
template <int ITEMS>
__global__ void __launch_bounds__(PT, 1) k_pipeline(PipeSpec P, TableCfg T)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *sm = reinterpret_cast<unsigned long long *>(smem);
    table_zero(P, T, sm);
    __syncthreads();
    constexpr int TR = PT * ITEMS;
    const int64_t ntiles = (P.n + TR - 1) / TR;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        RowVals v[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int64_t r = tile * TR + k * PT + threadIdx.x;
            v[k] = row_load(P, r, r < P.n);
        }
        int64_t hi[ITEMS], lo[ITEMS];
        bool ok[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) ok[k] = row_probe(P, v[k], hi[k], lo[k]);
        if (T.mode == TM_GLOBAL_HASH) {
            fold_rows_ghash<ITEMS>(P, ok, hi, lo, v);
        } else {
#pragma unroll
            for (int k = 0; k < ITEMS; k++)
                if (ok[k]) fold_row(P, T, sm, hi[k], lo[k], v[k]);
        }
    }
    __syncthreads();
    table_flush(P, T, sm);
}

// Star shape (see the file comment).  GLOBAL: the direct array lives in HBM (AoS, 4 words per slot)
// instead of shared memory (SoA).
// NSUM: the shared-memory direct array keeps SUM as 32-bit halves (small
// arrays, where many rows hit each slot and 64-bit atomics collide most).
// JK: the star kind (STAR_INNER, STAR_SEMI, STAR_ANTI, STAR_NONE).
template <bool GLOBAL, int ITEMS, bool NSUM, int JK, bool L2H = false>
__global__ void __launch_bounds__(PT, 1) k_pipeline_star(PipeSpec P, TableCfg T)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *sm = reinterpret_cast<unsigned long long *>(smem);
    if (!GLOBAL) table_zero(P, T, sm);
    __syncthreads();
    // grid-stride tiles: at any moment the blocks read neighbouring tiles
    constexpr int64_t TR = static_cast<int64_t>(PT) * ITEMS;
    star_range<GLOBAL, ITEMS, PT, NSUM, JK, L2H>(P, sm, static_cast<int64_t>(blockIdx.x) * TR, P.n, TR * gridDim.x);
    __syncthreads();
    if (!GLOBAL) table_flush(P, T, sm, NSUM ? 2 : 1);
}

template <class K>
qe_status launch(qe_ctx *ctx, K kern, const PipeSpec &P, const TableCfg &T, size_t smem, int64_t rows_per_tile,
                 cudaStream_t s)
{
    QE_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    const int64_t ntiles = qe_ceil_div(P.n, rows_per_tile);
    int64_t grid = ctx->num_sms;
    if (grid > ntiles) grid = ntiles;
    {
        ProfScope prof(ctx, "pipeline", s);
        kern<<<static_cast<unsigned>(grid), PT, smem, s>>>(P, T);
        QE_LAUNCHED(ctx);
    }
    QE_CHECK_LAUNCH(ctx);
    return QE_OK;
}

}  // namespace

// Validate a pipeline description and build its device view (everything but
// the join table and the group table).
qe_status pipeline_prepare(qe_ctx *ctx, const qe_pipeline_desc *d, PipeSpec &P)
{
    if (!d) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: null desc");
    if (d->n_fact < 0 || d->n_fact >= (int64_t(1) << 31) || d->n_fact_cols < 0 || d->n_fact_cols > QE_MAX_COLS ||
        d->n_preds < 0 || d->n_preds > QE_MAX_PREDS || d->n_aggs < 0 || d->n_aggs > QE_MAX_AGGS)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad sizes");
    P = PipeSpec{};
    P.n = d->n_fact;
    const int nc = d->n_fact_cols;
    for (int c = 0; c < nc; c++) {
        const qe_col &col = d->fact[c];
        if (!qe_valid_type(col.type) || col.gather || (P.n > 0 && !col.data) || !qe_aligned(col.data, col.type))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad fact column " + std::to_string(c));
    }
    auto colok = [&](int c) { return c >= 0 && c < nc; };
    int slot_of[QE_MAX_COLS];
    for (int c = 0; c < QE_MAX_COLS; c++) slot_of[c] = -1;
    auto use = [&](int c) -> int {
        if (slot_of[c] < 0) {
            slot_of[c] = P.ncol;
            P.col[P.ncol] = d->fact[c].data;
            P.type[P.ncol] = d->fact[c].type;
            P.ncol++;
        }
        return slot_of[c];
    };
    P.npreds = d->n_preds;
    for (int p = 0; p < d->n_preds; p++) {
        const qe_pred &pr = d->preds[p];
        if (!colok(pr.col) || pr.op < QE_LT || pr.op > QE_BETWEEN)
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad predicate");
        P.pslot[p] = use(pr.col);
        P.pop[p] = pr.op;
        P.plo[p] = pr.lo;
        P.phi[p] = pr.hi;
    }
    if (d->fk_col >= 0) {
        if (!colok(d->fk_col) || d->fact[d->fk_col].type != QE_I32)
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: join column must be int32");
        P.has_join = 1;
        P.fk_slot = use(d->fk_col);
    } else if (d->fk_col != -1) {
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad join column");
    }
    if (d->join_kind < QE_JOIN_INNER || d->join_kind > QE_JOIN_ANTI)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad join kind");
    if (d->join_kind != QE_JOIN_INNER && !P.has_join)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: a semi- or anti-join needs a join column");
    if (d->join_kind != QE_JOIN_INNER && d->key_lo_col == QE_JOIN_PAYLOAD)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: a semi- or anti-join has no payload to group by");
    P.join_kind = d->join_kind;
    P.hi_slot = -1;
    if (d->key_hi_col != -1) {
        if (!colok(d->key_hi_col)) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad key_hi");
        P.hi_slot = use(d->key_hi_col);
    }
    if (d->key_lo_col == QE_JOIN_PAYLOAD) {
        if (!P.has_join) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: join payload key without a join");
        P.lo_slot = QE_JOIN_PAYLOAD;
    } else if (colok(d->key_lo_col)) {
        P.lo_slot = use(d->key_lo_col);
    } else {
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad key_lo");
    }
    int xc = -1, yc = -1;
    P.ops.n = d->n_aggs;
    for (int a = 0; a < d->n_aggs; a++) {
        const qe_agg_spec &g = d->aggs[a];
        if (g.op < QE_SUM || g.op > QE_MAX) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad aggregate");
        P.ops.op[a] = g.op;
        P.src[a] = SRC_NONE;
        if (g.op == QE_COUNT) continue;
        if (!colok(g.a) || (g.b != -1 && !colok(g.b)))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad aggregate column");
        auto place = [&](int c) -> int {
            if (xc == c) return SRC_X;
            if (yc == c) return SRC_Y;
            if (xc < 0) { xc = c; return SRC_X; }
            if (yc < 0) { yc = c; return SRC_Y; }
            return -1;
        };
        int sa = place(g.a);
        if (sa < 0) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: aggregates use more than two columns");
        if (g.b == -1) {
            P.src[a] = sa;
        } else {
            int sb = place(g.b);
            if (sb < 0 || sb == sa) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: unsupported aggregate shape");
            P.src[a] = SRC_XY;
        }
    }
    P.x_slot = xc >= 0 ? use(xc) : -1;
    P.y_slot = yc >= 0 ? use(yc) : -1;
    return QE_OK;
}

// Table placement of a pipeline.
struct PipePlan {
    TableCfg T{};
    size_t table = 0;     // shared-memory table bytes
    size_t gdense_bytes = 0;
};

// Choose where groups live: a direct array (shared memory, else HBM) when
// the key parts have known small ranges, else a shared-memory hash table,
// else the HBM hash table.
qe_status pipeline_plan(qe_ctx *ctx, PipeSpec &P, const qe_pipeline_desc *d, const qe_hash_table *ht,
                        int64_t capacity, PipePlan &plan)
{
    const size_t static_smem = 1024;
    const size_t budget = ctx->smem_optin > static_smem ? ctx->smem_optin - static_smem : 0;
    const bool has_hi = P.hi_slot >= 0;
    P.dk = DenseKey{};
    int64_t lo_min = 1, lo_max = 0;
    if (d->have_key_range) {
        lo_min = d->key_lo_min;
        lo_max = d->key_lo_max;
    }
    if (lo_min > lo_max && P.lo_slot == QE_JOIN_PAYLOAD && ht && ht->have_pay) {
        lo_min = ht->pay_min;
        lo_max = ht->pay_max;
    }
    if (lo_min <= lo_max && (!has_hi || d->have_key_range))
        P.dk = dense_plan(has_hi, d->key_hi_min, d->key_hi_max, lo_min, lo_max, P.ops, uint64_t(1) << 26);
    if (P.dk.on) {
        const size_t bytes = P.dk.nslots * P.dk.stride * 8;
        if (bytes <= budget) {
            plan.T.mode = TM_SMEM_DENSE;
            plan.table = bytes;
        } else {
            plan.T.mode = TM_GLOBAL_DENSE;
            plan.gdense_bytes = bytes;
        }
    } else {
        const int64_t groups = d->expected_groups > 0 ? d->expected_groups : capacity;
        const int S = st_slots_for(groups, P.ops.n, budget);
        if (S) {
            plan.T.mode = TM_SMEM_HASH;
            plan.T.S = S;
            while ((1 << plan.T.log2S) < S) plan.T.log2S++;
            plan.table = static_cast<size_t>(S) * 8 * (1 + P.ops.n);
        } else {
            plan.T.mode = TM_GLOBAL_HASH;
        }
    }
    return QE_OK;
}

// The star kinds other than the inner join: 3 rows per thread.
template <int JK>
qe_status launch_star_kind(qe_ctx *ctx, const PipeSpec &P, const PipePlan &plan, cudaStream_t s)
{
    if (plan.T.mode == TM_GLOBAL_DENSE)
        return launch(ctx, k_pipeline_star<true, 3, false, JK>, P, plan.T, 0, PT * 3, s);
    if (P.dk.nslots <= STAR_NSUM_SLOTS)
        return launch(ctx, k_pipeline_star<false, 3, true, JK>, P, plan.T, plan.table, PT * 3, s);
    return launch(ctx, k_pipeline_star<false, 3, false, JK>, P, plan.T, plan.table, PT * 3, s);
}

// Bind the HBM tables and launch the fused pass.
qe_status pipeline_launch(qe_ctx *ctx, PipeSpec &P, const PipePlan &plan, const GroupTableHost &t, int64_t capacity,
                          cudaStream_t s)
{
    P.g.words = t.words;
    P.g.mask = t.slots - 1;
    P.g.stride = t.stride;
    P.g.capacity = capacity;
    P.g.st = ctx->dstat;
    if (P.n == 0) return QE_OK;
    const int kind = ctx->tune_force_generic ? -1 : star_kind(P, plan.T);
    if (kind == STAR_SEMI || kind == STAR_ANTI || kind == STAR_NONE) {
        star_predicate(P);
        return kind == STAR_SEMI   ? launch_star_kind<STAR_SEMI>(ctx, P, plan, s)
               : kind == STAR_ANTI ? launch_star_kind<STAR_ANTI>(ctx, P, plan, s)
                                   : launch_star_kind<STAR_NONE>(ctx, P, plan, s);
    }
    if (kind == STAR_INNER) {
        star_predicate(P);
        // rows per thread: 3 by default, 2 when tuned so
        const bool two = ctx->tune_star_items == 2;
        if (ctx->tune_l2_hint && !two) {
            // L2 policies: fact columns evict first, payload lookups evict last
            if (plan.T.mode == TM_GLOBAL_DENSE)
                return launch(ctx, k_pipeline_star<true, 3, false, STAR_INNER, true>, P, plan.T, 0, PT * 3, s);
            if (P.dk.nslots <= STAR_NSUM_SLOTS)
                return launch(ctx, k_pipeline_star<false, 3, true, STAR_INNER, true>, P, plan.T, plan.table, PT * 3, s);
            return launch(ctx, k_pipeline_star<false, 3, false, STAR_INNER, true>, P, plan.T, plan.table, PT * 3, s);
        }
        if (plan.T.mode == TM_GLOBAL_DENSE)
            return two ? launch(ctx, k_pipeline_star<true, 2, false, STAR_INNER>, P, plan.T, 0, PT * 2, s)
                       : launch(ctx, k_pipeline_star<true, 3, false, STAR_INNER>, P, plan.T, 0, PT * 3, s);
        // SUM in 32-bit halves up to STAR_NSUM_SLOTS slots: measured 2.89 against 4.38 ms for a
        // batch of 300 pipelines of 75 groups, and 2.94 against 2.86 ms for 600M rows into 3,000
        if (P.dk.nslots <= STAR_NSUM_SLOTS)
            return two ? launch(ctx, k_pipeline_star<false, 2, true, STAR_INNER>, P, plan.T, plan.table, PT * 2, s)
                       : launch(ctx, k_pipeline_star<false, 3, true, STAR_INNER>, P, plan.T, plan.table, PT * 3, s);
        return two ? launch(ctx, k_pipeline_star<false, 2, false, STAR_INNER>, P, plan.T, plan.table, PT * 2, s)
                   : launch(ctx, k_pipeline_star<false, 3, false, STAR_INNER>, P, plan.T, plan.table, PT * 3, s);
    }
    return launch(ctx, k_pipeline<2>, P, plan.T, plan.table, PT * 2, s);
}

qe_status pipeline_partitioned(qe_ctx *ctx, PipeSpec &P, const qe_groups_out *out, int64_t groups, cudaStream_t s);

// Whether a pipeline whose groups go to the HBM hash table takes the
// partitioned path: when tuned so, or (auto) when that table would be far
// larger than L2 (random read-modify-writes in DRAM) and the input is large
// enough to amortise the extra passes.
static bool use_partitioned(qe_ctx *ctx, const PipeSpec &P, int64_t capacity)
{
    if (ctx->tune_gb_partition == 1 || P.n == 0) return false;
    if (ctx->tune_gb_partition == 2) return true;
    uint64_t want = static_cast<uint64_t>(capacity > 32 ? capacity : 32) * 2, slots = 64;
    while (slots < want) slots <<= 1;
    return slots * (1 + P.ops.n) * 8 > (256ull << 20) && P.n >= (int64_t(1) << 22);
}

extern "C" qe_status qe_pipeline(qe_ctx *ctx, const qe_pipeline_desc *desc, const qe_groups_out *out, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PipeSpec P;
    qe_status st = pipeline_prepare(ctx, desc, P);
    if (st != QE_OK) return st;
    st = gt_check_out(ctx, out, P.ops);
    if (st != QE_OK) return st;
    cudaSetDevice(ctx->device);
    qe_hash_table *built = nullptr;
    if (P.has_join) {
        const qe_hash_table *ht = desc->ht;
        const bool inner = P.join_kind == QE_JOIN_INNER;
        if (!ht) {
            if (desc->n_dim < 0 || (desc->n_dim > 0 && (!desc->dim_key || (inner && !desc->dim_payload))))
                return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad dimension columns");
            // a semi- or anti-join builds a key set (repeated keys allowed)
            st = join_build_impl(ctx, desc->dim_key, desc->dim_payload, desc->n_dim, &desc->build, !inner, &built, s);
            if (st != QE_OK) return st;
            ht = built;
        } else if (inner && ht->set) {
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: an inner join needs a table with payloads");
        } else if (ht->multi || ht->pair) {
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: takes a unique-key table or a key set, not a multimap or pair-key table");
        }
        P.ht = ht_view(ht);
    }
    PipePlan plan;
    st = pipeline_plan(ctx, P, desc, P.has_join ? (desc->ht ? desc->ht : built) : nullptr, out->capacity, plan);
    void *gd = nullptr;
    if (st == QE_OK && plan.gdense_bytes) {
        st = qe_alloc(ctx, &gd, plan.gdense_bytes, s);
        if (st == QE_OK) {
            cudaError_t e = cudaMemsetAsync(gd, 0, plan.gdense_bytes, s);
            if (e != cudaSuccess) st = qe_cuda_fail(ctx, e, "pipeline: dense table");
        }
        P.gdense = static_cast<unsigned long long *>(gd);
    }
    // Groups that only fit an HBM hash table far larger than L2: partition
    // the rows on the key's hash and aggregate each part in L2 (qe_pipe_part.cu).
    if (st == QE_OK && plan.T.mode == TM_GLOBAL_HASH && use_partitioned(ctx, P, out->capacity)) {
        P.g = GTable{};
        P.g.st = ctx->dstat;
        P.g.capacity = out->capacity;
        st = pipeline_partitioned(ctx, P, out, out->capacity, s);
        if (built) qe_join_destroy(ctx, built, s);
        return st;
    }
    GroupTableHost t;
    if (st == QE_OK) st = gt_create(ctx, out->capacity, P.ops.n, t, s);
    if (st == QE_OK) {
        st = pipeline_launch(ctx, P, plan, t, out->capacity, s);
        if (st == QE_OK) {
            st = P.gdense ? gt_finalize_dense(ctx, t, P.ops, P.dk, P.gdense, out, s)
                          : gt_finalize(ctx, t, P.ops, out, s);
        }
        qe_free(ctx, t.words, s);
    }
    if (gd) qe_free(ctx, gd, s);
    if (built) qe_join_destroy(ctx, built, s);
    return st;
}
