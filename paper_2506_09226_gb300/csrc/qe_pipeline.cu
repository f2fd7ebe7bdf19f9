// qe_pipeline.cu -- the fused per-GPU operator pipeline (Sec. 2.4: each GPU
// runs one program over its local columns): group-by(join(filter(fact), dim)).
//
// After the dimension table is built (qe_join.cu), one persistent kernel
// makes a single pass over the fact columns.  For each tile of rows it
//   1. reads the predicate columns (streaming, coalesced) and evaluates the
//      conjunction;
//   2. reads the foreign key and the group/aggregate columns of survivors;
//   3. probes the join table (dense tables sit in L2);
//   4. folds survivors into the block's shared-memory group table (or the HBM
//      table when the groups do not fit), without any block barrier, so warps
//      overlap these phases.
// Blocks merge their shared-memory tables into the HBM table at the end and
// the HBM table is compacted into the output.
//
// Aggregate values are drawn from at most two fact columns X and Y (each
// aggregate is X, Y or X*Y), which covers SUM(price*qty), MIN(price),
// MAX(price), COUNT(*); other shapes are rejected with QE_ERR_INVALID_ARG.
#include "qe_internal.cuh"

namespace {

enum { SRC_NONE = 0, SRC_X = 1, SRC_Y = 2, SRC_XY = 3 };

struct PipeArgs {
    int64_t n;
    const void *col[QE_MAX_COLS];
    int32_t type[QE_MAX_COLS];
    int npreds;
    int32_t pcol[QE_MAX_PREDS], pop[QE_MAX_PREDS];
    int64_t plo[QE_MAX_PREDS], phi[QE_MAX_PREDS];
    int fk_col;
    HtView ht;
    int key_hi_col, key_lo_col;
    int x_col, y_col;
    int32_t src[QE_MAX_AGGS];
    AggOps ops;
    GTable g;
    int S;
    int max_probe;
};

template <int ITEMS, int BLOCK>
__device__ __forceinline__ void load_col(const void *p, int type, int64_t base, const bool (&ld)[ITEMS],
                                         int64_t (&v)[ITEMS])
{
    switch (type) {
    case QE_I32:
#pragma unroll
        for (int k = 0; k < ITEMS; k++)
            v[k] = ld[k] ? static_cast<int64_t>(__ldcs(static_cast<const int32_t *>(p) + base + k * BLOCK)) : 0;
        break;
    case QE_I64:
#pragma unroll
        for (int k = 0; k < ITEMS; k++) v[k] = ld[k] ? __ldcs(static_cast<const long long *>(p) + base + k * BLOCK) : 0;
        break;
    default:
#pragma unroll
        for (int k = 0; k < ITEMS; k++)
            v[k] = ld[k] ? static_cast<int64_t>(__ldcs(static_cast<const signed char *>(p) + base + k * BLOCK)) : 0;
        break;
    }
}

template <int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) k_pipeline(PipeArgs A)
{
    extern __shared__ unsigned long long sm[];
    if (A.S) st_zero(sm, A.S, A.ops.n);
    __syncthreads();
    const int64_t tile_rows = static_cast<int64_t>(BLOCK) * ITEMS;
    const int64_t ntiles = (A.n + tile_rows - 1) / tile_rows;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * tile_rows + threadIdx.x;
        bool ok[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) ok[k] = base + k * BLOCK < A.n;
        // 1. selection
        for (int p = 0; p < A.npreds; p++) {
            int64_t v[ITEMS];
            load_col<ITEMS, BLOCK>(A.col[A.pcol[p]], A.type[A.pcol[p]], base, ok, v);
#pragma unroll
            for (int k = 0; k < ITEMS; k++) ok[k] = ok[k] && dev_cmp(v[k], A.pop[p], A.plo[p], A.phi[p]);
        }
        // 2. columns of survivors
        int64_t lo[ITEMS], hi[ITEMS], x[ITEMS], y[ITEMS];
        if (A.fk_col >= 0) load_col<ITEMS, BLOCK>(A.col[A.fk_col], QE_I32, base, ok, lo);
        else load_col<ITEMS, BLOCK>(A.col[A.key_lo_col], A.type[A.key_lo_col], base, ok, lo);
        if (A.key_hi_col >= 0) load_col<ITEMS, BLOCK>(A.col[A.key_hi_col], A.type[A.key_hi_col], base, ok, hi);
        if (A.x_col >= 0) load_col<ITEMS, BLOCK>(A.col[A.x_col], A.type[A.x_col], base, ok, x);
        if (A.y_col >= 0) load_col<ITEMS, BLOCK>(A.col[A.y_col], A.type[A.y_col], base, ok, y);
        // 3. join probe: the low key half becomes the dimension payload
        if (A.fk_col >= 0) {
#pragma unroll
            for (int k = 0; k < ITEMS; k++) {
                int32_t pay = 0;
                if (ok[k]) ok[k] = ht_lookup(A.ht, static_cast<int32_t>(lo[k]), pay);
                if (A.key_lo_col == QE_JOIN_PAYLOAD) lo[k] = pay;
            }
            if (A.key_lo_col != QE_JOIN_PAYLOAD)
                load_col<ITEMS, BLOCK>(A.col[A.key_lo_col], A.type[A.key_lo_col], base, ok, lo);
        }
        // 4. aggregate
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            if (!ok[k]) continue;
            int64_t key = lo[k];
            if (A.key_hi_col >= 0)
                key = static_cast<int64_t>((static_cast<uint64_t>(hi[k]) << 32) | static_cast<uint32_t>(lo[k]));
            const unsigned long long kx = static_cast<unsigned long long>(key) ^ GB_SIGN;
            if (kx == 0) {
                dev_report(A.g.st, QE_ERR_RESERVED_KEY, 0);
                continue;
            }
            unsigned long long e[QE_MAX_AGGS];
            _Pragma("unroll") for (int a = 0; a < QE_MAX_AGGS; a++) if (a < A.ops.n) {
                const int src = A.src[a];
                int64_t v = src == SRC_X ? x[k]
                          : src == SRC_Y ? y[k]
                          : src == SRC_XY ? static_cast<int64_t>(static_cast<uint64_t>(x[k]) * static_cast<uint64_t>(y[k]))
                                          : 0;
                e[a] = agg_encode(A.ops.op[a], v);
            }
            st_fold_row(sm, A.S, A.ops, A.g, kx, e, A.max_probe);
        }
    }
    if (A.S) {
        __syncthreads();
        st_flush(sm, A.S, A.ops, A.g);
    }
}

template <int BLOCK, int ITEMS>
qe_status launch_pipeline(qe_ctx *ctx, const PipeArgs &A, size_t smem, cudaStream_t s)
{
    auto kern = k_pipeline<BLOCK, ITEMS>;
    QE_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    QE_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(ctx->num_sms) * per_sm;
    int64_t need = qe_ceil_div(A.n, static_cast<int64_t>(BLOCK) * ITEMS);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    {
        ProfScope prof(ctx, "pipeline", s);
        kern<<<static_cast<unsigned>(grid), BLOCK, smem, s>>>(A);
        QE_LAUNCHED(ctx);
    }
    QE_CHECK_LAUNCH(ctx);
    return QE_OK;
}

}  // namespace

// Validate a pipeline description and translate it to kernel arguments
// (everything but the join table and the group table).
qe_status pipeline_prepare(qe_ctx *ctx, const qe_pipeline_desc *d, PipeArgs &A);

qe_status pipeline_prepare(qe_ctx *ctx, const qe_pipeline_desc *d, PipeArgs &A)
{
    if (!d) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: null desc");
    if (d->n_fact < 0 || d->n_fact >= (int64_t(1) << 31) || d->n_fact_cols < 0 || d->n_fact_cols > QE_MAX_COLS ||
        d->n_preds < 0 || d->n_preds > QE_MAX_PREDS || d->n_aggs < 0 || d->n_aggs > QE_MAX_AGGS)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad sizes");
    A = PipeArgs{};
    A.n = d->n_fact;
    const int nc = d->n_fact_cols;
    for (int c = 0; c < nc; c++) {
        const qe_col &col = d->fact[c];
        if (!qe_valid_type(col.type) || col.gather || (A.n > 0 && !col.data) || !qe_aligned(col.data, col.type))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad fact column " + std::to_string(c));
        A.col[c] = col.data;
        A.type[c] = col.type;
    }
    auto colok = [&](int c) { return c >= 0 && c < nc; };
    A.npreds = d->n_preds;
    for (int p = 0; p < d->n_preds; p++) {
        const qe_pred &pr = d->preds[p];
        if (!colok(pr.col) || pr.op < QE_LT || pr.op > QE_BETWEEN)
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad predicate");
        A.pcol[p] = pr.col;
        A.pop[p] = pr.op;
        A.plo[p] = pr.lo;
        A.phi[p] = pr.hi;
    }
    A.fk_col = d->fk_col;
    if (A.fk_col >= 0 && (!colok(A.fk_col) || A.type[A.fk_col] != QE_I32))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: join column must be int32");
    if (A.fk_col < 0 && A.fk_col != -1) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad join column");
    A.key_hi_col = d->key_hi_col;
    A.key_lo_col = d->key_lo_col;
    if (A.key_hi_col != -1 && !colok(A.key_hi_col)) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad key_hi");
    if (A.key_lo_col == QE_JOIN_PAYLOAD) {
        if (A.fk_col < 0) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: join payload key without a join");
    } else if (!colok(A.key_lo_col)) {
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad key_lo");
    }
    A.x_col = A.y_col = -1;
    A.ops.n = d->n_aggs;
    for (int a = 0; a < d->n_aggs; a++) {
        const qe_agg_spec &g = d->aggs[a];
        if (g.op < QE_SUM || g.op > QE_MAX) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad aggregate");
        A.ops.op[a] = g.op;
        A.src[a] = SRC_NONE;
        if (g.op == QE_COUNT) continue;
        if (!colok(g.a) || (g.b != -1 && !colok(g.b)))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad aggregate column");
        auto place = [&](int c) -> int {
            if (A.x_col == c) return SRC_X;
            if (A.y_col == c) return SRC_Y;
            if (A.x_col < 0) { A.x_col = c; return SRC_X; }
            if (A.y_col < 0) { A.y_col = c; return SRC_Y; }
            return -1;
        };
        int sa = place(g.a);
        if (sa < 0) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: aggregates use more than two columns");
        if (g.b == -1) {
            A.src[a] = sa;
        } else {
            int sb = place(g.b);
            if (sb < 0 || sb == sa) return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: unsupported aggregate shape");
            A.src[a] = SRC_XY;
        }
    }
    return QE_OK;
}

// Launch the fused pass with the join table and group table in place.
qe_status pipeline_launch(qe_ctx *ctx, PipeArgs &A, const GroupTableHost &t, int64_t capacity,
                          int64_t expected_groups, cudaStream_t s)
{
    A.g.words = t.words;
    A.g.mask = t.slots - 1;
    A.g.stride = t.stride;
    A.g.nkeys = t.words + t.slots * t.stride;
    A.g.capacity = capacity;
    A.g.st = ctx->dstat;
    A.max_probe = 32;
    const size_t budget = ctx->smem_optin > 4096 ? ctx->smem_optin - 4096 : 0;
    const int64_t groups = expected_groups > 0 ? expected_groups : capacity;
    A.S = st_slots_for(groups, A.ops.n, budget);
    if (A.n == 0) return QE_OK;
    const size_t smem = static_cast<size_t>(A.S) * 8 * (1 + A.ops.n);
    if (smem > 48 * 1024) return launch_pipeline<1024, 4>(ctx, A, smem, s);
    return launch_pipeline<256, 8>(ctx, A, smem, s);
}

extern "C" qe_status qe_pipeline(qe_ctx *ctx, const qe_pipeline_desc *desc, const qe_groups_out *out, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PipeArgs A;
    qe_status st = pipeline_prepare(ctx, desc, A);
    if (st != QE_OK) return st;
    st = gt_check_out(ctx, out, desc->n_aggs);
    if (st != QE_OK) return st;
    cudaSetDevice(ctx->device);
    qe_hash_table *built = nullptr;
    if (A.fk_col >= 0) {
        const qe_hash_table *ht = desc->ht;
        if (!ht) {
            if (desc->n_dim < 0 || (desc->n_dim > 0 && (!desc->dim_key || !desc->dim_payload)))
                return qe_fail(ctx, QE_ERR_INVALID_ARG, "pipeline: bad dimension columns");
            st = join_build_impl(ctx, desc->dim_key, desc->dim_payload, desc->n_dim, &desc->build, &built, s);
            if (st != QE_OK) return st;
            ht = built;
        }
        A.ht = ht_view(ht);
    }
    GroupTableHost t;
    st = gt_create(ctx, out->capacity, A.ops.n, t, s);
    if (st == QE_OK) {
        st = pipeline_launch(ctx, A, t, out->capacity, desc->expected_groups, s);
        if (st == QE_OK) st = gt_finalize(ctx, t, A.ops, out, s);
        qe_free(ctx, t.words, s);
    }
    if (built) qe_join_destroy(ctx, built, s);
    return st;
}
