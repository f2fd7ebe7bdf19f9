// qe_pipe_part.cu -- partition-then-aggregate for pipelines whose groups do
// not fit on chip.
//
// The paper names hash tables with hundreds of millions of keys as too large
// to handle efficiently (Sec. 7.2) and, for its exchange, applies one
// partitioning function to every row before the local operator runs on each
// part (Sec. 2.2).  Here the same idea keeps a group-by with tens of
// millions of groups out of random DRAM read-modify-writes: the surviving
// rows are partitioned on the hash of their group key, so that each part's
// groups fit a hash table that stays in L2, and each part is aggregated in
// turn.
//
//   count    one contiguous row range per block; each row's part p (top
//            log2p bits of fmix64 of the stored key) is counted in a shared
//            histogram.  When the group key is made of fact columns only,
//            every row is counted from the key columns alone (the filter and
//            join run once, in the scatter); otherwise the survivors of the
//            filter and join are counted.
//   scan     exclusive scan of the counts, part-major: segment (p, b) of
//            block b starts after every row of the parts before p and of
//            the blocks before b in part p.
//   scatter  the same ranges again: filter, join, key; each survivor
//            appends (stored key, X, Y) -- 24 bytes -- to its segment
//            through a shared-memory cursor, and the final cursors give each
//            segment's fill.  A block writes one run per part, so at most
//            2^log2p pages per block are open.
//   fold     one persistent kernel over an ordered list of work items:
//            stage s holds the fold items (s, b) of part s -- one per
//            segment -- and then the compaction chunks of part s - 1.  Part
//            p aggregates into window p mod R of a ring of R hash tables
//            (linear probing on the low hash bits, atomics), which together
//            stay resident in L2.  A compaction chunk waits (bounded) for
//            every fold item of its part, emits its slots' groups straight
//            into the caller's output and zeroes them; a fold item of part p
//            waits (bounded) for the compaction of part p - R, the previous
//            user of its window.  Items are claimed in order from one
//            counter and every wait is on an earlier item, so running blocks
//            always hold what is waited for.
//
// Aggregates are exact whatever order rows fold in (wrapping sums, counts,
// min / max), so the parts need no stable order.
#include "qe_pipe_core.cuh"

namespace {

constexpr int PPT = 1024;          // threads per block (all phases)
constexpr int PP_ITEMS = 2;        // rows per thread per tile (count / scatter)
constexpr int PF_ITEMS = 4;        // rows per thread per round (fold)

struct PartRow {
    unsigned long long kx;         // stored key: key ^ INT64_MIN (0 is reserved)
    long long x, y;                // the aggregate sources X and Y
};
static_assert(sizeof(PartRow) == 24, "scratch rows are 24 bytes");

struct PartArgs {
    PipeSpec P;
    int32_t log2p;                 // parts = 1 << log2p (1 .. 10)
    int32_t nblk;                  // blocks of the count and scatter phases
    int64_t rows_per_blk;          // contiguous fact rows per block
    int32_t count_all;             // count every row from its key columns
    int32_t pad;
    uint32_t *cnt;                 // [parts][nblk] counted rows
    int64_t *seg;                  // [parts][nblk] segment starts
    uint32_t *fill;                // [parts][nblk] rows written
    PartRow *rows;                 // scratch, one row per fact row at most
};

__device__ __forceinline__ unsigned long long pp_key(const PipeSpec &P, int64_t hi, int64_t lo)
{
    int64_t key = lo;
    if (P.hi_slot >= 0) key = static_cast<int64_t>((static_cast<uint64_t>(hi) << 32) | static_cast<uint32_t>(lo));
    return static_cast<unsigned long long>(key) ^ GB_SIGN;
}

__device__ __forceinline__ uint32_t pp_part(unsigned long long kx, int log2p)
{
    return static_cast<uint32_t>(dev_fmix64(kx) >> (64 - log2p));
}

// Key parts of fact row r from the key columns alone (the low part is a
// fact column here).
__device__ __forceinline__ bool pp_key_only(const PipeSpec &P, int64_t r, bool in, int64_t &hi, int64_t &lo)
{
    if (!in) return false;
    lo = ld_slot(P, P.lo_slot, r);
    hi = P.hi_slot >= 0 ? ld_slot(P, P.hi_slot, r) : 0;
    return true;
}

__global__ void __launch_bounds__(PPT) k_pp_count(PartArgs A)
{
    extern __shared__ unsigned hist[];
    const int parts = 1 << A.log2p;
    for (int i = threadIdx.x; i < parts; i += PPT) hist[i] = 0;
    __syncthreads();
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * A.rows_per_blk;
    const int64_t r1 = r0 + A.rows_per_blk < A.P.n ? r0 + A.rows_per_blk : A.P.n;
    for (int64_t t = r0; t < r1; t += PPT * PP_ITEMS) {
        int64_t hi[PP_ITEMS], lo[PP_ITEMS];
        bool ok[PP_ITEMS];
        if (A.count_all) {
#pragma unroll
            for (int k = 0; k < PP_ITEMS; k++) {
                const int64_t r = t + k * PPT + threadIdx.x;
                ok[k] = pp_key_only(A.P, r, r < r1, hi[k], lo[k]);
            }
        } else {
            RowVals v[PP_ITEMS];
#pragma unroll
            for (int k = 0; k < PP_ITEMS; k++) {
                const int64_t r = t + k * PPT + threadIdx.x;
                v[k] = row_load(A.P, r, r < r1);
            }
#pragma unroll
            for (int k = 0; k < PP_ITEMS; k++) ok[k] = row_probe(A.P, v[k], hi[k], lo[k]);
        }
#pragma unroll
        for (int k = 0; k < PP_ITEMS; k++) {
            if (!ok[k]) continue;
            const unsigned long long kx = pp_key(A.P, hi[k], lo[k]);
            if (kx == 0) continue;         // reserved key: reported by the scatter
            atomicAdd(&hist[pp_part(kx, A.log2p)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < parts; i += PPT) A.cnt[static_cast<int64_t>(i) * A.nblk + blockIdx.x] = hist[i];
}

// Exclusive scan of m counts into seg (one block): each thread sums a
// contiguous run, the run sums are scanned across the block, then each
// thread writes its run's starts.
__global__ void __launch_bounds__(PPT) k_pp_scan(const uint32_t *cnt, int64_t m, int64_t *seg)
{
    __shared__ int64_t warp_tot[PPT / 32];
    const int64_t per = (m + PPT - 1) / PPT;
    const int64_t a = threadIdx.x * per, b = a + per < m ? a + per : m;
    int64_t s = 0;
    for (int64_t i = a; i < b; i++) s += cnt[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t inc = warp_incl_scan<int64_t>(s);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int64_t t = warp_tot[lane];
        const int64_t ti = warp_incl_scan<int64_t>(t);
        warp_tot[lane] = ti - t;
    }
    __syncthreads();
    int64_t run = warp_tot[w] + inc - s;
    for (int64_t i = a; i < b; i++) {
        seg[i] = run;
        run += cnt[i];
    }
}

__global__ void __launch_bounds__(PPT) k_pp_scatter(PartArgs A)
{
    extern __shared__ __align__(16) unsigned char pp_smem[];
    const int parts = 1 << A.log2p;
    int64_t *base = reinterpret_cast<int64_t *>(pp_smem);
    unsigned *cur = reinterpret_cast<unsigned *>(base + parts);
    unsigned *cap = cur + parts;
    for (int i = threadIdx.x; i < parts; i += PPT) {
        const int64_t j = static_cast<int64_t>(i) * A.nblk + blockIdx.x;
        base[i] = A.seg[j];
        cap[i] = A.cnt[j];
        cur[i] = 0;
    }
    __syncthreads();
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * A.rows_per_blk;
    const int64_t r1 = r0 + A.rows_per_blk < A.P.n ? r0 + A.rows_per_blk : A.P.n;
    for (int64_t t = r0; t < r1; t += PPT * PP_ITEMS) {
        RowVals v[PP_ITEMS];
#pragma unroll
        for (int k = 0; k < PP_ITEMS; k++) {
            const int64_t r = t + k * PPT + threadIdx.x;
            v[k] = row_load(A.P, r, r < r1);
        }
        int64_t hi[PP_ITEMS], lo[PP_ITEMS];
        bool ok[PP_ITEMS];
#pragma unroll
        for (int k = 0; k < PP_ITEMS; k++) ok[k] = row_probe(A.P, v[k], hi[k], lo[k]);
#pragma unroll
        for (int k = 0; k < PP_ITEMS; k++) {
            if (!ok[k]) continue;
            const unsigned long long kx = pp_key(A.P, hi[k], lo[k]);
            if (kx == 0) {
                dev_report(A.P.g.st, QE_ERR_RESERVED_KEY, 0);
                continue;
            }
            const uint32_t p = pp_part(kx, A.log2p);
            const unsigned pos = atomicAdd(&cur[p], 1u);
            if (pos >= cap[p]) {           // the count pass saw fewer rows: never write past a segment
                dev_report(A.P.g.st, QE_ERR_INVALID_ARG, 0);
                continue;
            }
            PartRow *d = A.rows + base[p] + pos;
            d->kx = kx;
            d->x = v[k].x;
            d->y = v[k].y;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < parts; i += PPT) {
        const unsigned f = cur[i] < cap[i] ? cur[i] : cap[i];
        A.fill[static_cast<int64_t>(i) * A.nblk + blockIdx.x] = f;
    }
}

// ------------------------------------------------------------ fold
struct FoldArgs {
    AggOps ops;
    int32_t src[QE_MAX_AGGS];
    int32_t log2p, nblk;
    int32_t log2w;                 // window slots = 1 << log2w
    int32_t ring;                  // windows in the ring (power of two)
    int32_t chunks;                // compaction chunks per window
    int32_t stride;                // words per slot: key + aggregates
    int32_t cnt;                   // COUNT aggregate (averages), or -1
    int32_t pad;
    const int64_t *seg;
    const uint32_t *fill;
    const PartRow *rows;
    unsigned long long *win;       // ring * (1 << log2w) * stride words
    unsigned *done_fold, *done_comp;   // [parts]
    unsigned long long *items;     // item counter
    unsigned long long *emitted;   // groups written to `out`
    qe_groups_out out;
    int64_t nitems;
    int64_t spin_limit;
    qe_dev_status *st;
};

__device__ __forceinline__ unsigned long long pp_value(const FoldArgs &A, int a, long long x, long long y)
{
    const int s = A.src[a];
    const int64_t v = s == SRC_X ? x : s == SRC_Y ? y
                    : s == SRC_XY ? static_cast<int64_t>(static_cast<uint64_t>(x) * static_cast<uint64_t>(y)) : 0;
    return agg_encode(A.ops.op[a], v);
}

// Slot of kx in a window (inserting it), starting from its home slot; -1
// when a probe chain of GT_MAX_PROBE slots holds neither the key nor an
// empty slot (more groups in the part than the window can take).
static __device__ __noinline__ int64_t pp_find_insert(unsigned long long *win, uint64_t wmask, int stride,
                                                      unsigned long long kx, uint64_t i)
{
    const uint64_t limit = wmask < GT_MAX_PROBE ? wmask : GT_MAX_PROBE;
    for (uint64_t probes = 0; probes <= limit; probes++) {
        unsigned long long *cell = win + i * stride;
        const unsigned long long c = __ldcg(cell);
        if (c == kx) return static_cast<int64_t>(i);
        if (c == 0) {
            const unsigned long long old = atomicCAS(cell, 0ull, kx);
            if (old == 0 || old == kx) return static_cast<int64_t>(i);
        }
        i = (i + 1) & wmask;
    }
    return -1;
}

// Fold the n rows of one segment into a window.  Each thread holds
// PF_ITEMS rows; their home slots are read before any of them folds, so the
// rows' L2 round trips overlap.
__device__ void pp_fold_segment(const FoldArgs &A, unsigned long long *win, const PartRow *rows, int64_t n)
{
    const uint64_t wmask = (uint64_t(1) << A.log2w) - 1;
    for (int64_t b0 = 0; b0 < n; b0 += PPT * PF_ITEMS) {
        unsigned long long kx[PF_ITEMS], cur[PF_ITEMS];
        long long x[PF_ITEMS], y[PF_ITEMS];
        uint64_t home[PF_ITEMS];
#pragma unroll
        for (int k = 0; k < PF_ITEMS; k++) {
            const int64_t i = b0 + k * PPT + threadIdx.x;
            kx[k] = 0;
            x[k] = y[k] = 0;
            if (i < n) {
                kx[k] = __ldcs(&rows[i].kx);
                x[k] = __ldcs(&rows[i].x);
                y[k] = __ldcs(&rows[i].y);
            }
        }
#pragma unroll
        for (int k = 0; k < PF_ITEMS; k++) {
            home[k] = dev_fmix64(kx[k]) & wmask;
            cur[k] = kx[k] ? __ldcg(win + home[k] * A.stride) : 0;
        }
#pragma unroll
        for (int k = 0; k < PF_ITEMS; k++) {
            if (!kx[k]) continue;
            const int64_t s = cur[k] == kx[k] ? static_cast<int64_t>(home[k])
                                              : pp_find_insert(win, wmask, A.stride, kx[k], home[k]);
            if (s < 0) {
                dev_report(A.st, QE_ERR_CAPACITY, A.out.capacity + 1);
                continue;
            }
            unsigned long long *cell = win + s * A.stride + 1;
#pragma unroll
            for (int a = 0; a < QE_MAX_AGGS; a++)
                if (a < A.ops.n) agg_fold(cell + a, A.ops.op[a], pp_value(A, a, x[k], y[k]));
        }
    }
}

// Emit the groups of slots [s0, s1) of a window into the output and zero
// those slots.
__device__ void pp_compact_chunk(const FoldArgs &A, unsigned long long *win, int64_t s0, int64_t s1)
{
    const int lane = threadIdx.x & 31;
    for (int64_t b = s0; b < s1; b += PPT) {
        const int64_t i = b + threadIdx.x;
        const bool in = i < s1;
        unsigned long long *cell = win + i * A.stride;
        const unsigned long long kx = in ? __ldcg(cell) : 0ull;
        const unsigned m = __ballot_sync(QE_FULL_MASK, kx != 0);
        if (m) {
            unsigned long long first = 0;
            if (lane == 0) first = atomicAdd(A.emitted, static_cast<unsigned long long>(__popc(m)));
            first = __shfl_sync(QE_FULL_MASK, first, 0);
            if (kx) {
                const int64_t pos = static_cast<int64_t>(first) + __popc(m & ((1u << lane) - 1));
                if (pos < A.out.capacity) {
                    A.out.keys[pos] = static_cast<int64_t>(kx ^ GB_SIGN);
                    for (int a = 0; a < A.ops.n; a++) A.out.aggs[a][pos] = agg_decode(A.ops.op[a], __ldcg(cell + 1 + a));
                    if (A.cnt >= 0)
                        write_avgs(A.out, pos, A.ops.n, A.cnt,
                                   [&](int a) { return agg_decode(A.ops.op[a], __ldcg(cell + 1 + a)); });
                }
            }
        }
        if (in)
            for (int w = 0; w < A.stride; w++) __stcg(cell + w, 0ull);
    }
}

// Bounded wait (thread 0) until *ctr reaches want; false on expiry.
__device__ __forceinline__ bool pp_wait(const unsigned *ctr, unsigned want, int64_t limit)
{
    int64_t spins = 0;
    while (*reinterpret_cast<const volatile unsigned *>(ctr) < want) {
        if (++spins > limit) return false;
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

__global__ void __launch_bounds__(PPT, 1) k_pp_fold(FoldArgs A)
{
    __shared__ long long s_item;
    __shared__ int s_ok;
    const int parts = 1 << A.log2p;
    const int64_t per_stage = static_cast<int64_t>(A.nblk) + A.chunks;
    const int64_t wslots = int64_t(1) << A.log2w;
    while (true) {
        if (threadIdx.x == 0) s_item = static_cast<long long>(atomicAdd(A.items, 1ull));
        __syncthreads();
        const int64_t it = s_item;
        if (it >= A.nitems) break;
        const int64_t stage = it / per_stage, r = it % per_stage;
        if (r < A.nblk) {
            // fold segment (stage, r) into window stage mod ring
            const int p = static_cast<int>(stage);
            if (p < parts) {
                if (threadIdx.x == 0)
                    s_ok = p < A.ring || pp_wait(A.done_comp + (p - A.ring), static_cast<unsigned>(A.chunks), A.spin_limit);
                __syncthreads();
                if (s_ok) {
                    const int64_t j = static_cast<int64_t>(p) * A.nblk + r;
                    pp_fold_segment(A, A.win + static_cast<int64_t>(p & (A.ring - 1)) * wslots * A.stride,
                                    A.rows + A.seg[j], A.fill[j]);
                } else if (threadIdx.x == 0) {
                    dev_report(A.st, QE_ERR_TIMEOUT, 0);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    atomicAdd(A.done_fold + p, 1u);
                }
            }
        } else if (stage >= 1) {
            // compaction chunk c of part stage - 1
            const int q = static_cast<int>(stage - 1);
            const int64_t c = r - A.nblk;
            if (threadIdx.x == 0) s_ok = pp_wait(A.done_fold + q, static_cast<unsigned>(A.nblk), A.spin_limit);
            __syncthreads();
            if (s_ok) {
                const int64_t span = wslots / A.chunks;
                pp_compact_chunk(A, A.win + static_cast<int64_t>(q & (A.ring - 1)) * wslots * A.stride, c * span,
                                 (c + 1) * span);
            } else if (threadIdx.x == 0) {
                dev_report(A.st, QE_ERR_TIMEOUT, 0);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(A.done_comp + q, 1u);
            }
        }
        __syncthreads();
    }
}

__global__ void k_pp_count_out(const unsigned long long *emitted, int64_t capacity, int64_t *ngroups, qe_dev_status *st)
{
    const int64_t n = static_cast<int64_t>(*emitted);
    *ngroups = n;
    if (n > capacity) dev_report(st, QE_ERR_CAPACITY, n);
}

}  // namespace

// Parameters of the partitioned group-by for `groups` expected groups with
// `stride` words per slot: parts (log2p), window slots (log2w) and ring
// windows, so that every window takes its part's groups at a load of at
// most about 2/3 and the whole ring stays within `ring_bytes` of L2.
struct PartPlan {
    int log2p = 0, log2w = 0, ring = 0, chunks = 0;
};

static PartPlan part_plan(int64_t groups, int stride, int log2p_hint)
{
    PartPlan pl;
    const uint64_t ring_bytes = 48ull << 20;
    pl.ring = 4;
    for (int lp = 1; lp <= 10; lp++) {
        const uint64_t per = static_cast<uint64_t>(groups + (int64_t(1) << lp) - 1) >> lp;
        int lw = 12;
        while ((uint64_t(1) << lw) < per + per / 2) lw++;
        pl.log2p = lp;
        pl.log2w = lw;
        if (log2p_hint > 0 ? lp == log2p_hint
                           : (uint64_t(1) << lw) * stride * 8 * static_cast<uint64_t>(pl.ring) <= ring_bytes)
            break;
    }
    pl.chunks = static_cast<int>((int64_t(1) << pl.log2w) / 2048);
    if (pl.chunks < 1) pl.chunks = 1;
    return pl;
}

// The partitioned path for a pipeline `P` whose group table would be an
// HBM hash table.  `P` must have its join table bound.  Writes `out`.
qe_status pipeline_partitioned(qe_ctx *ctx, PipeSpec &P, const qe_groups_out *out, int64_t groups, cudaStream_t s)
{
    const int stride = 1 + P.ops.n;
    const PartPlan pl = part_plan(groups, stride, ctx->tune_gb_part_log2p);
    const int parts = 1 << pl.log2p;
    const int nblk = ctx->num_sms;
    const int64_t tr = static_cast<int64_t>(PPT) * PP_ITEMS;
    int64_t rpb = qe_ceil_div(qe_ceil_div(P.n > 0 ? P.n : 1, nblk), tr) * tr;
    const int64_t m = static_cast<int64_t>(parts) * nblk;
    const int64_t wslots = int64_t(1) << pl.log2w;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t b_rows = up(static_cast<size_t>(P.n) * sizeof(PartRow));
    const size_t b_cnt = up(m * 4), b_seg = up(m * 8), b_fill = up(m * 4);
    const size_t b_win = up(static_cast<size_t>(pl.ring) * wslots * stride * 8);
    const size_t b_done = up(static_cast<size_t>(parts) * 8);
    const size_t b_ctr = 256;
    void *mem = nullptr;
    qe_status st = qe_alloc(ctx, &mem, b_rows + b_cnt + b_seg + b_fill + b_win + b_done + b_ctr, s);
    if (st != QE_OK) return st;
    char *c = static_cast<char *>(mem);
    PartArgs A{};
    A.P = P;
    A.log2p = pl.log2p;
    A.nblk = nblk;
    A.rows_per_blk = rpb;
    A.count_all = P.lo_slot != QE_JOIN_PAYLOAD;
    A.rows = reinterpret_cast<PartRow *>(c);
    A.cnt = reinterpret_cast<uint32_t *>(c + b_rows);
    A.seg = reinterpret_cast<int64_t *>(c + b_rows + b_cnt);
    A.fill = reinterpret_cast<uint32_t *>(c + b_rows + b_cnt + b_seg);
    char *zero = c + b_rows + b_cnt + b_seg + b_fill;   // window ring, done counters, item and group counters
    cudaError_t e = cudaMemsetAsync(zero, 0, b_win + b_done + b_ctr, s);
    FoldArgs F{};
    F.ops = P.ops;
    for (int a = 0; a < QE_MAX_AGGS; a++) F.src[a] = P.src[a];
    F.log2p = pl.log2p;
    F.nblk = nblk;
    F.log2w = pl.log2w;
    F.ring = pl.ring;
    F.chunks = pl.chunks;
    F.stride = stride;
    F.cnt = -1;
    for (int a = 0; a < QE_MAX_AGGS; a++)
        if (out->avg[a]) F.cnt = agg_count_index(P.ops);
    F.seg = A.seg;
    F.fill = A.fill;
    F.rows = A.rows;
    F.win = reinterpret_cast<unsigned long long *>(zero);
    F.done_fold = reinterpret_cast<unsigned *>(zero + b_win);
    F.done_comp = F.done_fold + parts;
    F.items = reinterpret_cast<unsigned long long *>(zero + b_win + b_done);
    F.emitted = F.items + 1;
    F.out = *out;
    F.nitems = static_cast<int64_t>(parts + 1) * (nblk + pl.chunks);
    F.spin_limit = ctx->spin_limit;
    F.st = ctx->dstat;
    const size_t sm_count = static_cast<size_t>(parts) * 4;
    const size_t sm_scatter = static_cast<size_t>(parts) * 16;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pp_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_scatter));
    if (e == cudaSuccess && P.n > 0) {
        {
            ProfScope prof(ctx, "part_count", s);
            k_pp_count<<<nblk, PPT, sm_count, s>>>(A);
            QE_LAUNCHED(ctx);
        }
        k_pp_scan<<<1, PPT, 0, s>>>(A.cnt, m, A.seg);
        QE_LAUNCHED(ctx);
        {
            ProfScope prof(ctx, "part_scatter_rows", s);
            k_pp_scatter<<<nblk, PPT, sm_scatter, s>>>(A);
            QE_LAUNCHED(ctx);
        }
        {
            ProfScope prof(ctx, "part_fold", s);
            k_pp_fold<<<nblk, PPT, 0, s>>>(F);
            QE_LAUNCHED(ctx);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_pp_count_out<<<1, 1, 0, s>>>(F.emitted, out->capacity, out->ngroups, ctx->dstat);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    qe_free(ctx, mem, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "pipeline: partitioned group-by");
    return QE_OK;
}
