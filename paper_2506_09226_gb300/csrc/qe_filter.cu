// qe_filter.cu -- selection with stable stream compaction (Sec. 2.1).
#include "qe_compact.cuh"

namespace {

constexpr int FILTER_ITEMS = 16;

struct FilterOp {
    const void *col[QE_MAX_PREDS];
    int32_t type[QE_MAX_PREDS];
    int32_t cmp[QE_MAX_PREDS];
    int64_t lo[QE_MAX_PREDS], hi[QE_MAX_PREDS];
    int npreds;
    int32_t *out;

    struct Slot {};

    template <int ITEMS>
    __device__ __forceinline__ void eval(int64_t pos0, bool (&ok)[ITEMS], Slot &) const
    {
        for (int p = 0; p < npreds; p++) {
            const void *c = col[p];
            const int op = cmp[p];
            const int64_t l = lo[p], h = hi[p];
            int64_t x[ITEMS];
            switch (type[p]) {
            case QE_I32:
#pragma unroll
                for (int k = 0; k < ITEMS; k++)
                    x[k] = ok[k] ? static_cast<int64_t>(__ldcs(static_cast<const int32_t *>(c) + pos0 + 32 * k)) : 0;
                break;
            case QE_I64:
#pragma unroll
                for (int k = 0; k < ITEMS; k++)
                    x[k] = ok[k] ? __ldcs(static_cast<const long long *>(c) + pos0 + 32 * k) : 0;
                break;
            default:
#pragma unroll
                for (int k = 0; k < ITEMS; k++)
                    x[k] = ok[k] ? static_cast<int64_t>(__ldcs(static_cast<const signed char *>(c) + pos0 + 32 * k)) : 0;
                break;
            }
#pragma unroll
            for (int k = 0; k < ITEMS; k++) ok[k] = ok[k] && dev_cmp(x[k], op, l, h);
        }
    }

    __device__ __forceinline__ void emit(int64_t o, int64_t pos, int, const Slot &) const
    {
        __stcs(out + o, static_cast<int32_t>(pos));
    }
};

}  // namespace

extern "C" qe_status qe_filter(qe_ctx *ctx, const qe_col *cols, int ncols, const qe_pred *preds, int npreds,
                               int64_t nrows, int32_t *out_sel, int64_t sel_capacity, int64_t *out_count,
                               void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (nrows < 0 || nrows >= (int64_t(1) << 31)) return qe_fail(ctx, QE_ERR_INVALID_ARG, "filter: nrows out of range");
    if (npreds < 0 || npreds > QE_MAX_PREDS || (npreds > 0 && !preds))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "filter: bad predicate list");
    if (ncols < 0 || ncols > QE_MAX_COLS || (ncols > 0 && !cols))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "filter: bad column list");
    if (!out_count || sel_capacity < 0 || (sel_capacity > 0 && !out_sel))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "filter: bad output");
    FilterOp op{};
    op.npreds = npreds;
    op.out = out_sel;
    for (int p = 0; p < npreds; p++) {
        const qe_pred &pr = preds[p];
        if (pr.col < 0 || pr.col >= ncols || pr.op < QE_LT || pr.op > QE_BETWEEN)
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "filter: bad predicate");
        const qe_col &c = cols[pr.col];
        if (!qe_valid_type(c.type) || c.gather || (nrows > 0 && !c.data) || !qe_aligned(c.data, c.type))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "filter: bad predicate column");
        op.col[p] = c.data;
        op.type[p] = c.type;
        op.cmp[p] = pr.op;
        op.lo[p] = pr.lo;
        op.hi[p] = pr.hi;
    }
    cudaSetDevice(ctx->device);
    return launch_compact<FILTER_ITEMS>(ctx, "filter", nrows, sel_capacity, out_count, op, static_cast<cudaStream_t>(stream));
}
