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
//   scatter  the same ranges again, in tiles of 4,096 rows: filter, join,
//            key; the tile's survivors are grouped by part in shared memory
//            (a shared count per part gives each row its rank, a scan gives
//            each part its start) and written as (stored key, X, Y) -- 24
//            bytes -- to the end of their segments, consecutive threads
//            storing consecutive 8-byte words of each part's run.  The final
//            cursors give each segment's fill.
//   fold     one persistent kernel over an ordered list of work items:
//            stage s holds the fold items (s, b) of part s -- one per
//            segment -- and then the compaction chunks of part s - lag.
//            Part p aggregates into window p mod R of a ring of R hash
//            tables (linear probing on the low hash bits, atomics), which
//            together stay resident in L2.  A compaction chunk waits
//            (bounded) for every fold item of its part, emits its slots'
//            groups straight into the caller's output and zeroes them; a
//            fold item of part p waits (bounded) for the compaction of part
//            p - R, the previous user of its window.  With lag = R - 2 both
//            waits are on items claimed a stage or more earlier, so they are
//            rarely felt; items are claimed in order from one counter and
//            every wait is on an earlier item, so running blocks always hold
//            what is waited for.
//
// Aggregates are exact whatever order rows fold in (wrapping sums, counts,
// min / max), so the parts need no stable order.
#include "qe_pipe_core.cuh"

namespace {

constexpr int PPT = 1024;          // threads per block (all phases)
constexpr int PP_ITEMS = 2;        // rows per thread per tile (count / scatter)
constexpr int PF_ITEMS = 4;        // rows per thread per round (fold)
constexpr int FPT = 512;           // threads per fold block; two blocks per SM, so one
                                   // block's item hand-over overlaps the other's rows

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

// Prefetch into L2 the lines of rows [t, t + rows) of the columns a row of
// the pipeline reads (its predicate, join and key columns and X / Y), so
// that the next tile's loads, issued one after another, hit L2.  Lane l of
// each warp takes every 32nd line of the warp's share of the tile.
__device__ __forceinline__ void pp_prefetch_tile(const PipeSpec &P, int64_t t, int64_t r1, int rows, bool key_only)
{
    if (t >= r1) return;
    const int64_t e = t + rows < r1 ? t + rows : r1;
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = 0; c < P.ncol; c++) {
        if (key_only && c != P.lo_slot && c != P.hi_slot) continue;
        const int sz = P.type[c];
        const uintptr_t b0 = reinterpret_cast<uintptr_t>(P.col[c]) + static_cast<uintptr_t>(t) * sz;
        const uintptr_t b1 = reinterpret_cast<uintptr_t>(P.col[c]) + static_cast<uintptr_t>(e) * sz;
        for (uintptr_t a = (b0 & ~uintptr_t(127)) + static_cast<uintptr_t>(w * 32 + lane) * 128; a < b1;
             a += static_cast<uintptr_t>(nw) * 32 * 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

__global__ void __launch_bounds__(PPT) k_pp_count(PartArgs A)
{
    extern __shared__ unsigned hist[];
    const int parts = 1 << A.log2p;
    for (int i = threadIdx.x; i < parts; i += PPT) hist[i] = 0;
    __syncthreads();
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * A.rows_per_blk;
    const int64_t r1 = r0 + A.rows_per_blk < A.P.n ? r0 + A.rows_per_blk : A.P.n;
    if (A.count_all) {
        // key columns only: PC_ITEMS independent loads in flight per thread
        constexpr int PC_ITEMS = 8;
        for (int64_t t = r0; t < r1; t += PPT * PC_ITEMS) {
            int64_t hi[PC_ITEMS], lo[PC_ITEMS];
            bool in[PC_ITEMS];
#pragma unroll
            for (int k = 0; k < PC_ITEMS; k++) {
                const int64_t r = t + k * PPT + threadIdx.x;
                in[k] = r < r1;
                lo[k] = in[k] ? ld_slot(A.P, A.P.lo_slot, r) : 0;
                hi[k] = in[k] && A.P.hi_slot >= 0 ? ld_slot(A.P, A.P.hi_slot, r) : 0;
            }
#pragma unroll
            for (int k = 0; k < PC_ITEMS; k++) {
                if (!in[k]) continue;
                const unsigned long long kx = pp_key(A.P, hi[k], lo[k]);
                if (kx) atomicAdd(&hist[pp_part(kx, A.log2p)], 1u);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < parts; i += PPT) A.cnt[static_cast<int64_t>(i) * A.nblk + blockIdx.x] = hist[i];
        return;
    }
    pp_prefetch_tile(A.P, r0, r1, PPT * PP_ITEMS, false);
    for (int64_t t = r0; t < r1; t += PPT * PP_ITEMS) {
        int64_t hi[PP_ITEMS], lo[PP_ITEMS];
        bool ok[PP_ITEMS];
        pp_prefetch_tile(A.P, t + PPT * PP_ITEMS, r1, PPT * PP_ITEMS, false);
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

// Rows per tile of the scatter (threads x PS_ITEMS) and the words of a
// staged row.
constexpr int PS_ITEMS = 4;
constexpr int PS_TILE = PPT * PS_ITEMS;

// Shared memory of the scatter: the staged tile (3 words per row), each
// staged row's part, and per part the segment base, cursor, capacity, tile
// count and tile start.
static inline size_t pp_scatter_smem(int parts)
{
    return static_cast<size_t>(PS_TILE) * 24 + static_cast<size_t>(PS_TILE) * 2 + static_cast<size_t>(parts) * 24 + 64 * 8;
}

// Shared-memory state of a scatter block (see pp_scatter_smem).
struct PpScatterShared {
    unsigned long long *stage;     // [PS_TILE][3] staged rows
    uint16_t *spart;               // [PS_TILE] part of each staged row
    int64_t *base;                 // [parts] segment start
    unsigned *cur, *cap, *tcnt, *tstart;   // [parts] cursor, capacity, tile count, tile start
};

__device__ __forceinline__ PpScatterShared pp_scatter_shared(unsigned char *smem, int parts)
{
    PpScatterShared S;
    S.stage = reinterpret_cast<unsigned long long *>(smem);
    S.spart = reinterpret_cast<uint16_t *>(S.stage + 3 * PS_TILE);
    S.base = reinterpret_cast<int64_t *>(S.spart + PS_TILE);
    S.cur = reinterpret_cast<unsigned *>(S.base + parts);
    S.cap = S.cur + parts;
    S.tcnt = S.cap + parts;
    S.tstart = S.tcnt + parts;
    return S;
}

__device__ __forceinline__ void pp_scatter_begin(const PartArgs &A, const PpScatterShared &S, int parts)
{
    for (int i = threadIdx.x; i < parts; i += PPT) {
        const int64_t j = static_cast<int64_t>(i) * A.nblk + blockIdx.x;
        S.base[i] = A.seg[j];
        S.cap[i] = A.cnt[j];
        S.cur[i] = 0;
        S.tcnt[i] = 0;
    }
    __syncthreads();
}

__device__ __forceinline__ void pp_scatter_end(const PartArgs &A, const PpScatterShared &S, int parts)
{
    for (int i = threadIdx.x; i < parts; i += PPT) {
        const unsigned f = S.cur[i] < S.cap[i] ? S.cur[i] : S.cap[i];
        A.fill[static_cast<int64_t>(i) * A.nblk + blockIdx.x] = f;
    }
}

// One tile's survivors (kx != 0) to their segments: rank by a shared count
// per part, scan the counts, stage the rows grouped by part, then store the
// staged 8-byte words with consecutive threads on consecutive words of each
// part's run.  The block's threads all call it (it has barriers).
template <int IT>
__device__ __forceinline__ void pp_stage_tile(const PartArgs &A, const PpScatterShared &S, int parts,
                                              const unsigned long long (&kx)[IT], const long long (&xv)[IT],
                                              const long long (&yv)[IT])
{
    __shared__ int s_w[PPT / 32];
    __shared__ unsigned s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t part[IT], rank[IT];
#pragma unroll
    for (int k = 0; k < IT; k++) {
        part[k] = kx[k] ? pp_part(kx[k], A.log2p) : 0;
        rank[k] = kx[k] ? atomicAdd(&S.tcnt[part[k]], 1u) : 0;
    }
    __syncthreads();
    {
        const int per = (parts + PPT - 1) / PPT;
        unsigned loc = 0;
        for (int j = 0; j < per; j++) {
            const int i = threadIdx.x * per + j;
            if (i < parts) loc += S.tcnt[i];
        }
        const unsigned inc = warp_incl_scan(loc);
        if (lane == 31) s_w[warp] = static_cast<int>(inc);
        __syncthreads();
        if (warp == 0) {
            const int w = s_w[lane];
            const int wi = warp_incl_scan(w);
            s_w[lane] = wi - w;
            if (lane == 31) s_total = static_cast<unsigned>(wi);
        }
        __syncthreads();
        unsigned run = static_cast<unsigned>(s_w[warp]) + inc - loc;
        for (int j = 0; j < per; j++) {
            const int i = threadIdx.x * per + j;
            if (i < parts) {
                S.tstart[i] = run;
                run += S.tcnt[i];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < IT; k++) {
        if (!kx[k]) continue;
        const unsigned pos = S.tstart[part[k]] + rank[k];
        S.stage[3 * pos] = kx[k];
        S.stage[3 * pos + 1] = static_cast<unsigned long long>(xv[k]);
        S.stage[3 * pos + 2] = static_cast<unsigned long long>(yv[k]);
        S.spart[pos] = static_cast<uint16_t>(part[k]);
    }
    __syncthreads();
    const unsigned total = s_total;
    for (unsigned w = threadIdx.x; w < 3 * total; w += PPT) {
        const unsigned row = w / 3, word = w - 3 * row;
        const unsigned p = S.spart[row];
        const unsigned pos = S.cur[p] + (row - S.tstart[p]);
        if (pos >= S.cap[p]) {             // the count pass saw fewer rows: never write past a segment
            if (word == 0) dev_report(A.P.g.st, QE_ERR_INVALID_ARG, 0);
            continue;
        }
        if (!QE_DCHECK(A.P.g.st, S.base[p] + pos < A.P.n, S.base[p] + pos)) continue;
        reinterpret_cast<unsigned long long *>(A.rows + S.base[p] + pos)[word] = S.stage[w];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < parts; i += PPT) {
        S.cur[i] += S.tcnt[i];
        S.tcnt[i] = 0;
    }
    __syncthreads();
}

// Any pipeline shape: the generic row loader, the next tile prefetched to L2.
__global__ void __launch_bounds__(PPT, 1) k_pp_scatter(PartArgs A)
{
    extern __shared__ __align__(16) unsigned char pp_smem[];
    const int parts = 1 << A.log2p;
    const PpScatterShared S = pp_scatter_shared(pp_smem, parts);
    pp_scatter_begin(A, S, parts);
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * A.rows_per_blk;
    const int64_t r1 = r0 + A.rows_per_blk < A.P.n ? r0 + A.rows_per_blk : A.P.n;
    pp_prefetch_tile(A.P, r0, r1, PS_TILE, false);
    for (int64_t t = r0; t < r1; t += PS_TILE) {
        pp_prefetch_tile(A.P, t + PS_TILE, r1, PS_TILE, false);
        RowVals v[PS_ITEMS];
#pragma unroll
        for (int k = 0; k < PS_ITEMS; k++) {
            const int64_t r = t + k * PPT + threadIdx.x;
            v[k] = row_load(A.P, r, r < r1);
        }
        unsigned long long kx[PS_ITEMS];
        long long xv[PS_ITEMS], yv[PS_ITEMS];
#pragma unroll
        for (int k = 0; k < PS_ITEMS; k++) {
            int64_t hi = 0, lo = 0;
            kx[k] = 0;
            if (row_probe(A.P, v[k], hi, lo)) {
                kx[k] = pp_key(A.P, hi, lo);
                if (kx[k] == 0) dev_report(A.P.g.st, QE_ERR_RESERVED_KEY, 0);
            }
            xv[k] = v[k].x;
            yv[k] = v[k].y;
        }
        pp_stage_tile<PS_ITEMS>(A, S, parts, kx, xv, yv);
    }
    pp_scatter_end(A, S, parts);
}

// The star shape (one int32 predicate column; no join, or a dense join
// table used for membership; a group key of fact columns: an int8 / int32
// high part or none and an int32 / int64 low part; X an int64 and Y an int32
// column): every column of the next tile is loaded into registers while the
// current tile is staged, as in the fused star pipeline, so the loads of a
// tile are in flight together instead of one dependent round trip after
// another.  JK: STAR_INNER / STAR_SEMI (membership), STAR_ANTI, STAR_NONE.
constexpr int PSS_ITEMS = 2;

template <int JK, bool LO64>
__global__ void __launch_bounds__(PPT, 1) k_pp_scatter_star(PartArgs A)
{
    extern __shared__ __align__(16) unsigned char pp_smem[];
    const int parts = 1 << A.log2p;
    const PpScatterShared S = pp_scatter_shared(pp_smem, parts);
    pp_scatter_begin(A, S, parts);
    const PipeSpec &P = A.P;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * A.rows_per_blk;
    const int64_t r1 = r0 + A.rows_per_blk < P.n ? r0 + A.rows_per_blk : P.n;
    constexpr int TR = PPT * PSS_ITEMS;
    int d[PSS_ITEMS], f[PSS_ITEMS], h[PSS_ITEMS], q[PSS_ITEMS];
    long long l[PSS_ITEMS], x[PSS_ITEMS];
    unsigned inmask = 0;
    auto load = [&](int64_t t0) {
        inmask = 0;
#pragma unroll
        for (int k = 0; k < PSS_ITEMS; k++) {
            const int64_t r = t0 + k * PPT + threadIdx.x;
            const bool in = r < r1;
            inmask |= in ? (1u << k) : 0u;
            d[k] = in ? __ldcs(P.s_pred + r) : 0;
            f[k] = JK != STAR_NONE && in ? __ldcs(P.s_fk + r) : 0;
            h[k] = P.s_has_hi && in ? (P.s_h8 ? static_cast<int>(__ldcs(static_cast<const signed char *>(P.s_hi) + r))
                                              : __ldcs(static_cast<const int32_t *>(P.s_hi) + r))
                                    : 0;
            l[k] = in ? (LO64 ? __ldcs(static_cast<const long long *>(P.s_lo) + r)
                              : static_cast<long long>(__ldcs(static_cast<const int32_t *>(P.s_lo) + r)))
                      : 0;
            x[k] = in ? __ldcs(P.s_x + r) : 0;
            q[k] = in ? __ldcs(P.s_y + r) : 0;
        }
    };
    if (r0 < r1) load(r0);
    for (int64_t t0 = r0; t0 < r1; t0 += TR) {
        unsigned long long kx[PSS_ITEMS];
        long long xv[PSS_ITEMS], yv[PSS_ITEMS];
        const unsigned cin = inmask;
#pragma unroll
        for (int k = 0; k < PSS_ITEMS; k++) {
            const bool pass = ((cin >> k) & 1u) && ((d[k] >= P.p0_lo && d[k] <= P.p0_hi) != static_cast<bool>(P.p0_neg));
            bool keep = pass;
            if (JK != STAR_NONE && pass) {
                const uint32_t ks = static_cast<uint32_t>(f[k]) - static_cast<uint32_t>(P.ht.key_min);
                const bool in = ks < P.ht.range && (P.ht.full || ((ht_ld(P.ht, P.ht.bitmap + (ks >> 5)) >> (ks & 31)) & 1u));
                keep = JK == STAR_ANTI ? !in : in;
            }
            const int64_t key = P.s_has_hi ? static_cast<int64_t>((static_cast<uint64_t>(static_cast<int64_t>(h[k])) << 32) |
                                                                  static_cast<uint32_t>(l[k]))
                                           : static_cast<int64_t>(l[k]);
            kx[k] = keep ? static_cast<unsigned long long>(key) ^ GB_SIGN : 0ull;
            if (keep && kx[k] == 0) dev_report(P.g.st, QE_ERR_RESERVED_KEY, 0);
            xv[k] = x[k];
            yv[k] = q[k];
        }
        load(t0 + TR);                     // the next tile's loads overlap this tile's staging
        pp_stage_tile<PSS_ITEMS>(A, S, parts, kx, xv, yv);
    }
    pp_scatter_end(A, S, parts);
}

// ------------------------------------------------------------ fold
struct FoldArgs {
    AggOps ops;
    int32_t src[QE_MAX_AGGS];
    int32_t log2p, nblk;
    int32_t log2w;                 // window slots = 1 << log2w
    int32_t ring;                  // windows in the ring (power of two)
    int32_t chunks;                // compaction chunks per window
    int32_t lag;                   // stage s compacts part s - lag (1 <= lag < ring)
    int32_t stride;                // words per slot: key + aggregates
    int32_t cnt;                   // COUNT aggregate (averages), or -1
    int32_t pad;
    const int64_t *seg;
    const uint32_t *fill;
    const PartRow *rows;
    unsigned long long *win;       // ring * (1 << log2w) * stride words
    unsigned *done_fold, *done_comp;   // [parts]
    unsigned *abort;               // set when a wait expired: later waits give up at once
    unsigned long long *items;     // item counter
    unsigned long long *emitted;   // groups written to `out`
    qe_groups_out out;
    int64_t nitems;
    int64_t nrows;                 // scratch rows (bounds of the segments)
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
    for (int64_t b0 = 0; b0 < n; b0 += FPT * PF_ITEMS) {
        unsigned long long kx[PF_ITEMS], cur[PF_ITEMS];
        long long x[PF_ITEMS], y[PF_ITEMS];
        uint64_t home[PF_ITEMS];
#pragma unroll
        for (int k = 0; k < PF_ITEMS; k++) {
            const int64_t i = b0 + k * FPT + threadIdx.x;
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
            // fire-and-forget reductions: a group gets only a few rows per
            // part, so reading MIN/MAX cells first would add two dependent
            // L2 round trips per row and save few atomics
            unsigned long long *cell = win + s * A.stride + 1;
#pragma unroll
            for (int a = 0; a < QE_MAX_AGGS; a++) {
                if (a >= A.ops.n) continue;
                const unsigned long long e = pp_value(A, a, x[k], y[k]);
                if (A.ops.op[a] == QE_SUM || A.ops.op[a] == QE_COUNT)
                    atomicAdd(cell + a, e);
                else
                    atomicMax(cell + a, e);
            }
        }
    }
}

// Emit the groups of slots [s0, s1) of a window into the output and zero
// those slots.  The block takes its output positions with one atomic per
// FPT slots (warp counts scanned in shared memory), not one per warp.
__device__ void pp_compact_chunk(const FoldArgs &A, unsigned long long *win, int64_t s0, int64_t s1)
{
    __shared__ unsigned s_wc[FPT / 32];
    __shared__ unsigned long long s_first;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b = s0; b < s1; b += FPT) {
        const int64_t i = b + threadIdx.x;
        const bool in = i < s1;
        unsigned long long *cell = win + i * A.stride;
        const unsigned long long kx = in ? __ldcg(cell) : 0ull;
        const unsigned m = __ballot_sync(QE_FULL_MASK, kx != 0);
        if (lane == 0) s_wc[warp] = __popc(m);
        __syncthreads();
        if (warp == 0) {
            constexpr int NW = FPT / 32;
            const unsigned c = lane < NW ? s_wc[lane] : 0u;
            const unsigned inc = warp_incl_scan(c);
            if (lane < NW) s_wc[lane] = inc - c;
            if (lane == 31) s_first = inc ? atomicAdd(A.emitted, static_cast<unsigned long long>(inc)) : 0ull;
        }
        __syncthreads();
        if (kx) {
            const int64_t pos = static_cast<int64_t>(s_first) + s_wc[warp] + __popc(m & ((1u << lane) - 1));
            if (pos < A.out.capacity) {
                A.out.keys[pos] = static_cast<int64_t>(kx ^ GB_SIGN);
                for (int a = 0; a < A.ops.n; a++) A.out.aggs[a][pos] = agg_decode(A.ops.op[a], __ldcg(cell + 1 + a));
                if (A.cnt >= 0)
                    write_avgs(A.out, pos, A.ops.n, A.cnt,
                               [&](int a) { return agg_decode(A.ops.op[a], __ldcg(cell + 1 + a)); });
            }
            // an empty slot is all zeros already (its aggregate words are
            // only touched once its key is set): zero the occupied ones
            for (int w = 0; w < A.stride; w++) __stcg(cell + w, 0ull);
        }
        __syncthreads();
    }
}

// Bounded wait (thread 0) until *ctr reaches want; false on expiry, or at
// once after any earlier wait of the launch expired.
__device__ __forceinline__ bool pp_wait(const unsigned *ctr, unsigned want, int64_t limit, unsigned *abort)
{
    int64_t spins = 0;
    while (*reinterpret_cast<const volatile unsigned *>(ctr) < want) {
        if (++spins > limit || *reinterpret_cast<const volatile unsigned *>(abort)) {
            atomicExch(abort, 1u);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// Thread 0: claim the next item and wait (bounded) for what it depends on;
// s_ok = 0 when the wait expired.
__device__ __forceinline__ void pp_claim(const FoldArgs &A, long long &s_item, int &s_ok)
{
    const int parts = 1 << A.log2p;
    const int64_t per_stage = static_cast<int64_t>(A.nblk) + A.chunks;
    const int64_t it = static_cast<int64_t>(atomicAdd(A.items, 1ull));
    s_item = it;
    s_ok = 1;
    if (it >= A.nitems) return;
    const int64_t stage = it / per_stage, r = it % per_stage;
    if (r < A.nblk) {
        const int p = static_cast<int>(stage);
        if (p < parts && p >= A.ring)
            s_ok = pp_wait(A.done_comp + (p - A.ring), static_cast<unsigned>(A.chunks), A.spin_limit, A.abort);
    } else if (stage >= A.lag && stage - A.lag < parts) {
        s_ok = pp_wait(A.done_fold + (stage - A.lag), static_cast<unsigned>(A.nblk), A.spin_limit, A.abort);
    }
}

__global__ void __launch_bounds__(FPT, 2) k_pp_fold(FoldArgs A)
{
    __shared__ long long s_item;
    __shared__ int s_ok;
    const int parts = 1 << A.log2p;
    const int64_t per_stage = static_cast<int64_t>(A.nblk) + A.chunks;
    const int64_t wslots = int64_t(1) << A.log2w;
    if (threadIdx.x == 0) pp_claim(A, s_item, s_ok);
    __syncthreads();
    while (true) {
        const int64_t it = s_item;
        const bool ok = s_ok;
        if (it >= A.nitems) break;
        const int64_t stage = it / per_stage, r = it % per_stage;
        unsigned *done = nullptr;
        if (r < A.nblk) {
            // fold segment (stage, r) into window stage mod ring
            const int p = static_cast<int>(stage);
            if (p < parts) {
                const int64_t j = static_cast<int64_t>(p) * A.nblk + r;
                if (ok && QE_DCHECK(A.st, A.seg[j] >= 0 && A.seg[j] + A.fill[j] <= A.nrows, A.seg[j] + A.fill[j]))
                    pp_fold_segment(A, A.win + static_cast<int64_t>(p & (A.ring - 1)) * wslots * A.stride,
                                    A.rows + A.seg[j], A.fill[j]);
                done = A.done_fold + p;
            }
        } else if (stage >= A.lag && stage - A.lag < parts) {
            // compaction chunk c of part stage - lag, whose fold items were
            // claimed lag stages earlier
            const int q = static_cast<int>(stage - A.lag);
            const int64_t c = r - A.nblk, span = wslots / A.chunks;
            if (ok)
                pp_compact_chunk(A, A.win + static_cast<int64_t>(q & (A.ring - 1)) * wslots * A.stride, c * span,
                                 (c + 1) * span);
            done = A.done_comp + q;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (!ok) dev_report(A.st, QE_ERR_TIMEOUT, 0);
            if (done) {
                __threadfence();
                atomicAdd(done, 1u);
            }
            pp_claim(A, s_item, s_ok);
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
    pl.chunks = static_cast<int>((int64_t(1) << pl.log2w) / 8192);
    if (pl.chunks < 1) pl.chunks = 1;
    return pl;
}

// The star-shape scatter's kind for P (see k_pp_scatter_star), or -1.  An
// inner join whose payload is not part of the key only needs membership.
static int pp_star_kind(const PipeSpec &P)
{
    if (P.npreds != 1 || P.type[P.pslot[0]] != QE_I32) return -1;
    if (P.lo_slot < 0 || (P.type[P.lo_slot] != QE_I32 && P.type[P.lo_slot] != QE_I64)) return -1;
    if (P.hi_slot >= 0 && P.type[P.hi_slot] != QE_I32 && P.type[P.hi_slot] != QE_I8) return -1;
    if (P.x_slot < 0 || P.type[P.x_slot] != QE_I64 || P.y_slot < 0 || P.type[P.y_slot] != QE_I32) return -1;
    if (!P.has_join) return STAR_NONE;
    if (P.ht.layout != QE_HT_DENSE) return -1;
    return P.join_kind == QE_JOIN_ANTI ? STAR_ANTI : STAR_SEMI;
}

template <bool LO64>
static const void *pp_star_kernel(int kind)
{
    if (kind == STAR_NONE) return reinterpret_cast<const void *>(k_pp_scatter_star<STAR_NONE, LO64>);
    if (kind == STAR_ANTI) return reinterpret_cast<const void *>(k_pp_scatter_star<STAR_ANTI, LO64>);
    return reinterpret_cast<const void *>(k_pp_scatter_star<STAR_SEMI, LO64>);
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
    F.abort = reinterpret_cast<unsigned *>(F.items + 2);
    F.out = *out;
    F.lag = pl.ring > 2 ? pl.ring - 2 : 1;
    F.nitems = static_cast<int64_t>(parts + F.lag) * (nblk + pl.chunks);
    F.nrows = P.n;
    F.spin_limit = ctx->spin_limit;
    F.st = ctx->dstat;
    const size_t sm_count = static_cast<size_t>(parts) * 4;
    const size_t sm_scatter = pp_scatter_smem(parts);
    // the scatter kernel: the star shape's register-prefetched loop, or the generic one
    const int skind = ctx->tune_force_generic ? -1 : pp_star_kind(P);
    const void *kscatter = reinterpret_cast<const void *>(k_pp_scatter);
    if (skind >= 0) {
        PipeSpec &Q = A.P;
        star_predicate(Q);
        kscatter = Q.type[Q.lo_slot] == QE_I64 ? pp_star_kernel<true>(skind) : pp_star_kernel<false>(skind);
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kscatter, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_scatter));
    if (e == cudaSuccess && P.n > 0) {
        {
            ProfScope prof(ctx, "part_count", s);
            k_pp_count<<<nblk, PPT, sm_count, s>>>(A);
            QE_LAUNCHED(ctx);
        }
        k_pp_scan<<<1, PPT, 0, s>>>(A.cnt, m, A.seg);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            ProfScope prof(ctx, "part_scatter_rows", s);
            void *args[] = {&A};
            e = cudaLaunchKernel(kscatter, dim3(nblk), dim3(PPT), args, sm_scatter, s);
            QE_LAUNCHED(ctx);
        }
        if (e == cudaSuccess) {
            ProfScope prof(ctx, "part_fold", s);
            k_pp_fold<<<2 * nblk, FPT, 0, s>>>(F);
            QE_LAUNCHED(ctx);
            e = cudaGetLastError();
        }
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
