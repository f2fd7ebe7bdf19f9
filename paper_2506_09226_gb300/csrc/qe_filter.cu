// qe_filter.cu -- selection with stable stream compaction (Sec. 2.1).
#include <type_traits>

#include "qe_compact.cuh"

namespace {

constexpr int FILTER_ITEMS = 16;

struct FilterSpec {
    const void *col[QE_MAX_PREDS];
    int32_t type[QE_MAX_PREDS];
    int32_t cmp[QE_MAX_PREDS];
    int64_t lo[QE_MAX_PREDS], hi[QE_MAX_PREDS];
    int npreds;
    int32_t *out;
    // each predicate as a range test: row passes iff ((uint64)(x - ra) <=
    // rw) != rneg, or iff rconst when the range is empty (rempty); for the
    // first predicate also at its column's width (ra0 / rw0 clamped to it)
    int64_t ra[QE_MAX_PREDS];
    uint64_t rw[QE_MAX_PREDS];
    uint8_t rneg[QE_MAX_PREDS], rempty[QE_MAX_PREDS];
    int64_t ra0;
    uint64_t rw0;
    uint8_t rconst0, rempty0, rneg0, pad0;
};

// Predicate p of a row whose value is x (any width, sign-extended).
__device__ __forceinline__ bool spec_pred(const FilterSpec &f, int p, int64_t x)
{
    const bool in = static_cast<uint64_t>(x - f.ra[p]) <= f.rw[p];
    return f.rempty[p] ? f.rneg[p] != 0 : in != (f.rneg[p] != 0);
}

// The first predicate at its column's own width.
template <class T0>
__device__ __forceinline__ bool spec_pred0(const FilterSpec &f, T0 x)
{
    using U = typename std::conditional<sizeof(T0) == 8, uint64_t, uint32_t>::type;
    const bool in = static_cast<U>(static_cast<U>(x) - static_cast<U>(f.ra0)) <= static_cast<U>(f.rw0);
    return f.rempty0 ? f.rconst0 != 0 : in != (f.rneg0 != 0);
}

// T0: element type of the first predicate's column, held in registers at
// its own width.
template <class T0>
struct FilterOp : FilterSpec {
    struct Slot {};
    struct Pre {
        T0 x[FILTER_ITEMS];
    };

    template <int ITEMS>
    __device__ __forceinline__ void load_col(int p, int64_t pos0, const bool (&in)[ITEMS], long long (&x)[ITEMS]) const
    {
        const void *c = col[p];
        switch (type[p]) {
        case QE_I32:
#pragma unroll
            for (int k = 0; k < ITEMS; k++)
                x[k] = in[k] ? static_cast<long long>(__ldcs(static_cast<const int32_t *>(c) + pos0 + 32 * k)) : 0;
            break;
        case QE_I64:
#pragma unroll
            for (int k = 0; k < ITEMS; k++) x[k] = in[k] ? __ldcs(static_cast<const long long *>(c) + pos0 + 32 * k) : 0;
            break;
        default:
#pragma unroll
            for (int k = 0; k < ITEMS; k++)
                x[k] = in[k] ? static_cast<long long>(__ldcs(static_cast<const signed char *>(c) + pos0 + 32 * k)) : 0;
            break;
        }
    }

    template <int ITEMS>
    __device__ __forceinline__ void load(int64_t pos0, const bool (&in)[ITEMS], Pre &p) const
    {
        if (npreds > 0) {
            const T0 *c = static_cast<const T0 *>(col[0]);
#pragma unroll
            for (int k = 0; k < ITEMS; k++) p.x[k] = in[k] ? __ldcs(c + pos0 + 32 * k) : T0(0);
        }
    }

    template <int ITEMS>
    __device__ __forceinline__ void eval(int64_t pos0, bool (&ok)[ITEMS], const Pre &pre, Slot &) const
    {
        if (npreds > 0) {
#pragma unroll
            for (int k = 0; k < ITEMS; k++) ok[k] = ok[k] && spec_pred0<T0>(*this, pre.x[k]);
        }
        for (int p = 1; p < npreds; p++) {
            long long x[ITEMS];
            load_col<ITEMS>(p, pos0, ok, x);
#pragma unroll
            for (int k = 0; k < ITEMS; k++) ok[k] = ok[k] && spec_pred(*this, p, x[k]);
        }
    }

    __device__ __forceinline__ void emit(int64_t o, int64_t pos, int, const Slot &) const
    {
        __stcs(out + o, static_cast<int32_t>(pos));
    }
};

// ---------------------------------------------------------------------------
// Two-pass filter for large inputs.  There is no dependency between blocks,
// so both passes keep as many loads in flight as registers allow; the
// price is a second read of the predicate columns.
//
// The segment counts are scanned by the generic two-pass kernels of
// qe_compact.cuh.
// Layout: a warp segment is IT items x 32 lanes x 4 rows; lane l of item k
// holds the 4 consecutive rows seg*SEGR + 128k + 4l + v (v = 0..3), read
// with one vector load of the first predicate's column, so row order is
// (item, lane, v).  Pass 1 counts each segment's survivors, a two-level scan
// turns the counts into offsets, and pass 2 re-evaluates each segment and
// writes its survivors item by item: the rank of row (l, v) in its item is
// the survivors of rows v' of lanes before l plus rows v' < v of lane l.
template <class T0>
struct Vec4;
template <>
struct Vec4<int32_t> {
    static constexpr int IT = 8;              // 128 bytes of loads in flight per thread
    __device__ static void load(const int32_t *p, int32_t (&v)[4])
    {
        const int4 x = __ldcs(reinterpret_cast<const int4 *>(p));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
};
template <>
struct Vec4<long long> {
    static constexpr int IT = 4;
    __device__ static void load(const long long *p, long long (&v)[4])
    {
        const longlong2 a = __ldcs(reinterpret_cast<const longlong2 *>(p));
        const longlong2 b = __ldcs(reinterpret_cast<const longlong2 *>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <>
struct Vec4<signed char> {
    static constexpr int IT = 16;
    __device__ static void load(const signed char *p, signed char (&v)[4])
    {
        const char4 x = __ldcs(reinterpret_cast<const char4 *>(p));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
};

// Survivor flags of lane's 4 rows of item k (bit v), for rows < n.
template <class T0>
__device__ __forceinline__ void seg_load(const FilterSpec &f, int64_t row, int64_t n, T0 (&x)[4])
{
    const T0 *c = static_cast<const T0 *>(f.col[0]);
    if (row + 3 < n) {
        Vec4<T0>::load(c + row, x);
    } else {
#pragma unroll
        for (int v = 0; v < 4; v++) x[v] = row + v < n ? __ldcs(c + row + v) : T0(0);
    }
}

template <class T0>
__device__ __forceinline__ unsigned seg_eval(const FilterSpec &f, int64_t row, int64_t n, const T0 (&x)[4], bool full)
{
    unsigned bits = 0;
#pragma unroll
    for (int v = 0; v < 4; v++) {
        bool ok = (full || row + v < n) && (f.npreds == 0 || spec_pred0<T0>(f, x[v]));
        for (int p = 1; p < f.npreds && ok; p++) ok = spec_pred(f, p, dev_col(f.col[p], f.type[p], row + v));
        bits |= ok ? (1u << v) : 0u;
    }
    return bits;
}

template <class T0>
__global__ void __launch_bounds__(256) k_filter_count(FilterSpec f, int64_t n, int64_t nseg, uint32_t *cnt)
{
    constexpr int IT = Vec4<T0>::IT;
    constexpr int SEGR = IT * 128;
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * 8;
    for (int64_t seg = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); seg < nseg; seg += warps) {
        const int64_t row0 = seg * SEGR + 4 * lane;
        T0 x[IT][4];
#pragma unroll
        for (int k = 0; k < IT; k++) seg_load<T0>(f, row0 + 128 * k, n, x[k]);
        const bool full = (seg + 1) * SEGR <= n;
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < IT; k++) c += __popc(seg_eval<T0>(f, row0 + 128 * k, n, x[k], full));
        c = warp_sum(c);
        if (lane == 0) cnt[seg] = c;
    }
}

template <class T0>
__global__ void __launch_bounds__(256) k_filter_write(FilterSpec f, int64_t n, int64_t nseg, const uint32_t *loc,
                                                     const int64_t *bsum, int64_t capacity)
{
    constexpr int IT = Vec4<T0>::IT;
    constexpr int SEGR = IT * 128;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * 8;
    for (int64_t seg = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); seg < nseg; seg += warps) {
        const int64_t row0 = seg * SEGR + 4 * lane;
        T0 x[IT][4];
#pragma unroll
        for (int k = 0; k < IT; k++) seg_load<T0>(f, row0 + 128 * k, n, x[k]);
        const bool full = (seg + 1) * SEGR <= n;
        int64_t pos = bsum[seg / TP_SCAN_B] + loc[seg];
#pragma unroll
        for (int k = 0; k < IT; k++) {
            const int64_t row = row0 + 128 * k;
            const unsigned bits = seg_eval<T0>(f, row, n, x[k], full);
            int before = 0, total = 0;
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const unsigned m = __ballot_sync(QE_FULL_MASK, (bits >> v) & 1u);
                before += __popc(m & lt);
                total += __popc(m);
            }
            int64_t o = pos + before;
#pragma unroll
            for (int v = 0; v < 4; v++) {
                if ((bits >> v) & 1u) {
                    if (o < capacity) __stcs(f.out + o, static_cast<int32_t>(row + v));
                    o++;
                }
            }
            pos += total;
        }
    }
}

template <class T0>
static qe_status filter_two_pass(qe_ctx *ctx, const FilterSpec &spec, int64_t n, int64_t capacity, int64_t *out_count,
                                 cudaStream_t s)
{
    const int64_t nseg = qe_ceil_div(n, static_cast<int64_t>(Vec4<T0>::IT) * 128);
    const int64_t nblk = qe_ceil_div(nseg, TP_SCAN_B);  // <= 1024 for n < 2^31 (segments >= 512 rows)
    void *scratch = nullptr;
    const size_t cnt_bytes = ((static_cast<size_t>(nseg) * 4 + 255) / 256) * 256;
    qe_status st = qe_alloc(ctx, &scratch, 2 * cnt_bytes + static_cast<size_t>(nblk) * 8, s);
    if (st != QE_OK) return st;
    uint32_t *cnt = static_cast<uint32_t *>(scratch);
    uint32_t *loc = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + cnt_bytes);
    int64_t *bsum = reinterpret_cast<int64_t *>(static_cast<char *>(scratch) + 2 * cnt_bytes);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_write<T0>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(ctx->num_sms) * per_sm;
    if (grid > qe_ceil_div(nseg, 8)) grid = qe_ceil_div(nseg, 8);
    cudaError_t e;
    {
        ProfScope prof(ctx, "filter", s);
        k_filter_count<T0><<<static_cast<unsigned>(grid), 256, 0, s>>>(spec, n, nseg, cnt);
        QE_LAUNCHED(ctx);
        k_tp_scan_local<<<static_cast<unsigned>(nblk), 1024, 0, s>>>(cnt, loc, nseg, bsum);
        QE_LAUNCHED(ctx);
        k_tp_scan_top<<<1, 1024, 0, s>>>(bsum, static_cast<int>(nblk), out_count, capacity, ctx->dstat);
        QE_LAUNCHED(ctx);
        k_filter_write<T0><<<static_cast<unsigned>(grid), 256, 0, s>>>(spec, n, nseg, loc, bsum, capacity);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    qe_free(ctx, scratch, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "filter launch");
    return QE_OK;
}

// Inputs from this size on take the two-pass filter; smaller ones the
// single-pass compaction (one launch).
constexpr int64_t TWO_PASS_ROWS = int64_t(1) << 22;

}  // namespace

// Checks the predicate list and fills the filter's description.
static qe_status filter_spec(qe_ctx *ctx, const qe_col *cols, int ncols, const qe_pred *preds, int npreds,
                             int64_t nrows, int32_t *out_sel, FilterSpec &spec)
{
    spec.npreds = npreds;
    spec.out = out_sel;
    for (int p = 0; p < npreds; p++) {
        const qe_pred &pr = preds[p];
        if (pr.col < 0 || pr.col >= ncols || pr.op < QE_LT || pr.op > QE_BETWEEN)
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "filter: bad predicate");
        const qe_col &c = cols[pr.col];
        if (!qe_valid_type(c.type) || c.gather || (nrows > 0 && !c.data) || !qe_aligned(c.data, c.type))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "filter: bad predicate column");
        spec.col[p] = c.data;
        spec.type[p] = c.type;
        spec.cmp[p] = pr.op;
        spec.lo[p] = pr.lo;
        spec.hi[p] = pr.hi;
        int64_t a, b;
        bool neg;
        const bool nonempty = qe_pred_range(pr.op, pr.lo, pr.hi, a, b, neg);
        spec.ra[p] = a;
        spec.rw[p] = static_cast<uint64_t>(b) - static_cast<uint64_t>(a);
        spec.rneg[p] = neg;
        spec.rempty[p] = !nonempty;
        if (p == 0) {
            // clamp to the column's own range, where the width test runs
            const int64_t tmin = c.type == QE_I8 ? INT8_MIN : (c.type == QE_I32 ? INT32_MIN : INT64_MIN);
            const int64_t tmax = c.type == QE_I8 ? INT8_MAX : (c.type == QE_I32 ? INT32_MAX : INT64_MAX);
            const int64_t ca = a < tmin ? tmin : a, cb = b > tmax ? tmax : b;
            const bool empty0 = !nonempty || ca > cb;
            spec.ra0 = empty0 ? 0 : ca;
            spec.rw0 = empty0 ? 0 : static_cast<uint64_t>(cb) - static_cast<uint64_t>(ca);
            spec.rneg0 = neg;
            spec.rempty0 = empty0;
            spec.rconst0 = neg;            // an empty range: every row fails, or passes when negated
        }
    }
    return QE_OK;
}

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
    FilterSpec spec{};
    qe_status st = filter_spec(ctx, cols, ncols, preds, npreds, nrows, out_sel, spec);
    if (st != QE_OK) return st;
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the two-pass filter reads the first predicate's column in 4-row vectors
    const int esz = npreds > 0 ? spec.type[0] : 4;
    if (nrows >= TWO_PASS_ROWS && (npreds == 0 || qe_aligned(spec.col[0], 4 * esz))) {
        switch (npreds > 0 ? spec.type[0] : QE_I32) {
        case QE_I64:
            return filter_two_pass<long long>(ctx, spec, nrows, sel_capacity, out_count, s);
        case QE_I8:
            return filter_two_pass<signed char>(ctx, spec, nrows, sel_capacity, out_count, s);
        default:
            return filter_two_pass<int32_t>(ctx, spec, nrows, sel_capacity, out_count, s);
        }
    }
    switch (npreds > 0 ? spec.type[0] : QE_I32) {
    case QE_I64:
        return launch_compact<FILTER_ITEMS>(ctx, "filter", nrows, sel_capacity, out_count, FilterOp<long long>{spec}, s);
    case QE_I8:
        return launch_compact<FILTER_ITEMS>(ctx, "filter", nrows, sel_capacity, out_count, FilterOp<signed char>{spec}, s);
    default:
        return launch_compact<FILTER_ITEMS>(ctx, "filter", nrows, sel_capacity, out_count, FilterOp<int32_t>{spec}, s);
    }
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

template <class Op>
static void noalloc_launch(qe_ctx *ctx, const CompactCommon &C, const Op &op, cudaStream_t s)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compact<FILTER_ITEMS, Op>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(ctx->num_sms) * per_sm;
    if (grid > C.ntiles) grid = C.ntiles;
    ProfScope prof(ctx, "filter", s);
    k_compact<FILTER_ITEMS, Op><<<static_cast<unsigned>(grid), 256, 0, s>>>(C, op);
    QE_LAUNCHED(ctx);
}

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
    FilterSpec spec{};
    qe_status sst = filter_spec(ctx, cols, ncols, preds, npreds, nrows, out_sel, spec);
    if (sst != QE_OK) return sst;
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
    switch (npreds > 0 ? spec.type[0] : QE_I32) {
    case QE_I64:
        noalloc_launch(ctx, C, FilterOp<long long>{spec}, s);
        break;
    case QE_I8:
        noalloc_launch(ctx, C, FilterOp<signed char>{spec}, s);
        break;
    default:
        noalloc_launch(ctx, C, FilterOp<int32_t>{spec}, s);
        break;
    }
    QE_CHECK_LAUNCH(ctx);
    return QE_OK;
}
