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

// ------------------------------------------------------------------------
// qe_filter_noalloc: the same selection kernel, with its scratch (the tile
// counter and the look-back status words) in a fixed static device array
// instead of memory allocated per call.  For callers that must not
// allocate device memory from inside the call (see qe.h).
//
// The array below is a host-side stand-in in host code, not a device
// address: host code must never pass `g_filter_scratch` itself to a kernel.
// Its device address is looked up with cudaGetSymbolAddress once per
// device (with that device current) on the first call made on that device.

namespace {

constexpr int64_t NOALLOC_TILES = QE_FILTER_NOALLOC_MAX_ROWS / (256 * FILTER_ITEMS);
static_assert(NOALLOC_TILES * 256 * FILTER_ITEMS == QE_FILTER_NOALLOC_MAX_ROWS, "max rows must be whole tiles");

// word 0: tile counter; words 1..NOALLOC_TILES: tile status words
static __device__ __align__(256) unsigned long long g_filter_scratch[1 + NOALLOC_TILES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

qe_status noalloc_scratch(qe_ctx *ctx, unsigned long long **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "qe_filter_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "qe_filter_noalloc: device index too large");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_filter_scratch);
        if (e != cudaSuccess || !p) return qe_cuda_fail(ctx, e, "qe_filter_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned long long *>(g_noalloc_ptr[dev]);
    return QE_OK;
}

}  // namespace

extern "C" qe_status qe_filter_noalloc(qe_ctx *ctx, const qe_col *cols, int ncols, const qe_pred *preds, int npreds,
                                       int64_t nrows, int32_t *out_sel, int64_t sel_capacity, int64_t *out_count,
                                       void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (nrows < 0) return qe_fail(ctx, QE_ERR_INVALID_ARG, "qe_filter_noalloc: nrows out of range");
    if (nrows > QE_FILTER_NOALLOC_MAX_ROWS)
        return qe_fail(ctx, QE_ERR_INVALID_ARG,
                       "qe_filter_noalloc: nrows " + std::to_string(nrows) + " exceeds the static scratch limit of " +
                           std::to_string(static_cast<long long>(QE_FILTER_NOALLOC_MAX_ROWS)) + " rows");
    if (npreds < 0 || npreds > QE_MAX_PREDS || (npreds > 0 && !preds))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "qe_filter_noalloc: bad predicate list");
    if (ncols < 0 || ncols > QE_MAX_COLS || (ncols > 0 && !cols))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "qe_filter_noalloc: bad column list");
    if (!out_count || sel_capacity < 0 || (sel_capacity > 0 && !out_sel))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "qe_filter_noalloc: bad output");
    FilterOp op{};
    op.npreds = npreds;
    op.out = out_sel;
    for (int p = 0; p < npreds; p++) {
        const qe_pred &pr = preds[p];
        if (pr.col < 0 || pr.col >= ncols || pr.op < QE_LT || pr.op > QE_BETWEEN)
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "qe_filter_noalloc: bad predicate");
        const qe_col &c = cols[pr.col];
        if (!qe_valid_type(c.type) || c.gather || (nrows > 0 && !c.data) || !qe_aligned(c.data, c.type))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "qe_filter_noalloc: bad predicate column");
        op.col[p] = c.data;
        op.type[p] = c.type;
        op.cmp[p] = pr.op;
        op.lo[p] = pr.lo;
        op.hi[p] = pr.hi;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "qe_filter_noalloc: cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nrows == 0) {
        QE_CUDA(ctx, cudaMemsetAsync(out_count, 0, sizeof(int64_t), s));
        return QE_OK;
    }
    unsigned long long *scratch = nullptr;
    qe_status st = noalloc_scratch(ctx, &scratch);
    if (st != QE_OK) return st;
    constexpr int TILE = 256 * FILTER_ITEMS;
    CompactCommon C;
    C.n = nrows;
    C.ntiles = qe_ceil_div(nrows, TILE);
    C.capacity = sel_capacity;
    C.out_count = out_count;
    C.st = ctx->dstat;
    C.spin_limit = ctx->spin_limit;
    C.tile_counter = scratch;
    C.tile_state = scratch + 1;
    // the counter and the status words of this call's tiles must start at zero
    QE_CUDA(ctx, cudaMemsetAsync(scratch, 0, (static_cast<size_t>(C.ntiles) + 1) * sizeof(unsigned long long), s));
    int per_sm = 0;
    QE_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compact<FILTER_ITEMS, FilterOp>, 256, 0));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(ctx->num_sms) * per_sm;
    if (grid > C.ntiles) grid = C.ntiles;
    {
        ProfScope prof(ctx, "filter", s);
        k_compact<FILTER_ITEMS, FilterOp><<<static_cast<unsigned>(grid), 256, 0, s>>>(C, op);
        QE_LAUNCHED(ctx);
    }
    QE_CHECK_LAUNCH(ctx);
    return QE_OK;
}
