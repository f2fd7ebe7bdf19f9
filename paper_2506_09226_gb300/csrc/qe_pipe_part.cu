// qe_pipe_part.cu -- partition-then-aggregate for pipelines whose groups do
// not fit on chip.
//
// The paper names hash tables with hundreds of millions of keys as too large
// to handle efficiently (Sec. 7.2) and, for its exchange, applies one
// partitioning function to every row before the local operator runs on each
// part (Sec. 2.2).  Here the same idea keeps a group-by with tens of
// millions of groups out of random DRAM read-modify-writes and L2 atomics:
// the surviving rows are partitioned twice on the hash of their group key,
// until each sub-part's groups fit one block's shared-memory hash table, and
// each sub-part is then aggregated on chip and written out once.
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
//            cursors give each segment's fill.  The star shape (one int32
//            predicate, a dense or no join, fact-column keys, int64 X and
//            int32 Y) loads the next tile into registers meanwhile.
//   split    the filled rows of every segment, in chunks of at most 4,096,
//            each sorted by sub-part (the next log2q hash bits) in shared
//            memory and written to a second buffer at the same rows, with
//            the chunk's sub-part offsets.
//   fold     one block per sub-part at a time: its runs (one per chunk of
//            its part) go through a shared-memory hash table (linear
//            probing, shared atomics); the table's groups are written to
//            the output with one global atomic per 1,024 slots, and zeroed.
//            A key that finds no slot within 64 probes (only when a
//            sub-part gets far more groups than planned) goes to an HBM
//            spill table, emitted after the fold.
//
#include "qe_pipe_core.cuh"

namespace {

constexpr int PPT = 1024;          // threads per block (all phases)
constexpr int PP_ITEMS = 2;        // rows per thread per tile (count / scatter)

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
// thread writes its run's starts.  With div > 0 the value scanned is
// ceil(count / div) (chunks of div rows); total (nullable) receives the sum.
__global__ void __launch_bounds__(PPT) k_pp_scan(const uint32_t *cnt, int64_t m, int64_t *seg, int div, int64_t *total)
{
    __shared__ int64_t warp_tot[PPT / 32];
    const int64_t per = (m + PPT - 1) / PPT;
    const int64_t a = threadIdx.x * per, b = a + per < m ? a + per : m;
    auto val = [&](int64_t i) -> int64_t { return div > 0 ? (cnt[i] + div - 1) / div : cnt[i]; };
    int64_t s = 0;
    for (int64_t i = a; i < b; i++) s += val(i);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t inc = warp_incl_scan<int64_t>(s);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int64_t t = warp_tot[lane];
        const int64_t ti = warp_incl_scan<int64_t>(t);
        warp_tot[lane] = ti - t;
        if (lane == 31 && total) *total = ti;
    }
    __syncthreads();
    int64_t run = warp_tot[w] + inc - s;
    for (int64_t i = a; i < b; i++) {
        seg[i] = run;
        run += val(i);
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

// ------------------------------------------------------------ split
// The second partition: every part of the scatter is split once more, into
// 2^log2q sub-parts (the next hash bits), so that a sub-part's groups fit a
// shared-memory hash table.  The part's rows are cut into chunks of at most
// SPLIT_ROWS rows (each inside one segment); a block sorts a chunk by
// sub-part in shared memory and writes it back to the same rows of a second
// buffer, with the chunk's sub-part offsets (16-bit, SPLIT_ROWS < 2^16).
constexpr int SPLIT_ROWS = 4096;
// Two blocks of 512 threads per SM, so that one block's chunk loads overlap
// the other's sorting, and every chunk's successor in its segment fetched
// into L2 while it is split (300M skewed rows, split at 50 / 90 %
// selectivity: 1.76 / 3.01 ms against 2.01 / 3.42 ms for one 1,024-thread
// block per SM without the prefetch).
constexpr int SPT = 512;                        // threads per split block
constexpr int SP_BLOCKS = 2;                    // split blocks per SM
constexpr int SP_ITEMS = SPLIT_ROWS / SPT;

struct SplitArgs {
    int32_t log2p, log2q, nblk, pad;
    int64_t m;                     // segments (parts x nblk)
    int64_t nrows;                 // rows of both buffers
    qe_dev_status *st;
    const int64_t *seg;
    const uint32_t *fill;
    const int64_t *cpre;           // [m + 1] chunks before each segment; cpre[m] = chunks
    const PartRow *rows;           // the scatter's rows
    PartRow *rows2;                // the split rows (same row numbers)
    uint16_t *off2;                // [chunks][2^log2q + 1] sub-part starts inside each chunk
    int64_t *cstart;               // [chunks] first row of each chunk
    unsigned long long *counter;   // chunk claims
};

__device__ __forceinline__ uint32_t pp_subpart(unsigned long long kx, int log2p, int log2q)
{
    return log2q ? static_cast<uint32_t>((dev_fmix64(kx) << log2p) >> (64 - log2q)) : 0u;
}

static inline size_t pp_split_smem(int log2q)
{
    return static_cast<size_t>(SPLIT_ROWS) * 24 + static_cast<size_t>(2 << log2q) * 4 + 64;
}

__global__ void __launch_bounds__(SPT, SP_BLOCKS) k_pp_split(SplitArgs A)
{
    extern __shared__ __align__(16) unsigned char sp_smem[];
    const int Q = 1 << A.log2q;
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(sp_smem);   // [SPLIT_ROWS][3]
    unsigned *tcnt = reinterpret_cast<unsigned *>(stage + 3 * SPLIT_ROWS);         // [Q]
    unsigned *tstart = tcnt + Q;                                                   // [Q]
    __shared__ long long s_j;
    __shared__ int s_w[SPT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < Q; i += SPT) tcnt[i] = 0;
    while (true) {
        // claim a segment; its chunks are cpre[j] .. cpre[j + 1]
        if (threadIdx.x == 0) s_j = static_cast<long long>(atomicAdd(A.counter, 1ull));
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();                   // every thread has read s_j before the next claim
        if (j >= A.m) break;
        const int64_t cA = A.cpre[j], cB = A.cpre[j + 1];
        for (int64_t c = cA; c < cB; c++) {
            const int64_t k = c - cA;
            const int64_t r0 = A.seg[j] + k * SPLIT_ROWS;
            const int64_t rend = A.seg[j] + A.fill[j];
            int n = static_cast<int>(r0 + SPLIT_ROWS < rend ? SPLIT_ROWS : rend - r0);
            if (!QE_DCHECK(A.st, r0 >= 0 && n >= 0 && r0 + n <= A.nrows, r0 + n)) n = 0;
            // the segment's next chunk into L2 while this one is split
            if (c + 1 < cB) {
                const int64_t nr0 = r0 + SPLIT_ROWS;
                const int64_t nn = rend - nr0 < SPLIT_ROWS ? rend - nr0 : SPLIT_ROWS;
                const char *base = reinterpret_cast<const char *>(A.rows + nr0);
                for (int64_t off = static_cast<int64_t>(threadIdx.x) * 128; off < nn * 24; off += SPT * 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
            }
            unsigned long long kx[SP_ITEMS];
            long long xv[SP_ITEMS], yv[SP_ITEMS];
            uint32_t sub[SP_ITEMS], rank[SP_ITEMS];
    #pragma unroll
            for (int t = 0; t < SP_ITEMS; t++) {
                const int i = t * SPT + threadIdx.x;
                kx[t] = 0;
                xv[t] = yv[t] = 0;
                if (i < n) {
                    const PartRow *r = A.rows + r0 + i;
                    kx[t] = __ldcs(&r->kx);
                    xv[t] = __ldcs(&r->x);
                    yv[t] = __ldcs(&r->y);
                }
            }
    #pragma unroll
            for (int t = 0; t < SP_ITEMS; t++) {
                sub[t] = kx[t] ? pp_subpart(kx[t], A.log2p, A.log2q) : 0u;
                rank[t] = kx[t] ? atomicAdd(&tcnt[sub[t]], 1u) : 0u;
            }
            __syncthreads();
            {
                // exclusive scan of the Q sub-part counts
                const int per = (Q + SPT - 1) / SPT;
                unsigned loc = 0;
                for (int q = 0; q < per; q++) {
                    const int i = threadIdx.x * per + q;
                    if (i < Q) loc += tcnt[i];
                }
                const unsigned inc = warp_incl_scan(loc);
                if (lane == 31) s_w[warp] = static_cast<int>(inc);
                __syncthreads();
                if (warp == 0) {
                    constexpr int NW = SPT / 32;
                    const int w = lane < NW ? s_w[lane] : 0;
                    const int wi = warp_incl_scan(w);
                    if (lane < NW) s_w[lane] = wi - w;
                }
                __syncthreads();
                unsigned run = static_cast<unsigned>(s_w[warp]) + inc - loc;
                for (int q = 0; q < per; q++) {
                    const int i = threadIdx.x * per + q;
                    if (i < Q) {
                        tstart[i] = run;
                        run += tcnt[i];
                    }
                }
            }
            __syncthreads();
    #pragma unroll
            for (int t = 0; t < SP_ITEMS; t++) {
                if (!kx[t]) continue;
                const unsigned pos = tstart[sub[t]] + rank[t];
                stage[3 * pos] = kx[t];
                stage[3 * pos + 1] = static_cast<unsigned long long>(xv[t]);
                stage[3 * pos + 2] = static_cast<unsigned long long>(yv[t]);
            }
            __syncthreads();
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(A.rows2 + r0);
            for (int w = threadIdx.x; w < 3 * n; w += SPT) __stcg(dst + w, stage[w]);
            uint16_t *o = A.off2 + c * (Q + 1);
            for (int i = threadIdx.x; i <= Q; i += SPT) o[i] = static_cast<uint16_t>(i < Q ? tstart[i] : n);
            if (threadIdx.x == 0) A.cstart[c] = r0;
            __syncthreads();
            for (int i = threadIdx.x; i < Q; i += SPT) tcnt[i] = 0;
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ fold
// One block per sub-part at a time: the sub-part's runs (one per chunk of
// its part) are folded into a shared-memory hash table, whose groups are
// then written straight to the output; keys that find no slot within the
// probe limit go to an HBM spill table, emitted at the end.
constexpr int FT = 1024;                        // threads per fold (and spill-emit) block
// Rows per lane and step of the fold, the next step's rows prefetched in
// registers (300M skewed rows, fold at 50 / 90 % selectivity: one row per
// lane 2.52 / 4.14 ms; two rows 2.73 / 4.64 ms; two rows with 768 threads
// 3.21 / 5.48 ms; two rows without the prefetch 2.58 / 4.27 ms).
constexpr int FOLD_FI = 1;
constexpr int F_RUNS = 1024;                    // runs described in shared memory at a time
constexpr int F_PROBES = 64;                    // shared-table probe limit before a spill
constexpr int F_EMIT_GROUPS = 128;              // slot groups of 32 in the largest shared table

struct FoldArgs {
    AggOps ops;
    int32_t src[QE_MAX_AGGS];
    int32_t log2p, log2q, nblk, log2s;          // log2s: shared-table slots
    int32_t cnt;                                // COUNT aggregate (averages), or -1
    int32_t pad;
    const int64_t *cpre;
    const uint16_t *off2;
    const int64_t *cstart;
    const PartRow *rows2;
    GTable spill;
    unsigned long long *counter;                // sub-part claims
    unsigned long long *emitted;                // groups written to `out`
    unsigned *spilled;                          // set once any key went to the spill table
    qe_groups_out out;
    qe_dev_status *st;
};

__device__ __forceinline__ unsigned long long pp_value(const FoldArgs &A, int a, long long x, long long y)
{
    const int s = A.src[a];
    const int64_t v = s == SRC_X ? x : s == SRC_Y ? y
                    : s == SRC_XY ? static_cast<int64_t>(static_cast<uint64_t>(x) * static_cast<uint64_t>(y)) : 0;
    return agg_encode(A.ops.op[a], v);
}

static __device__ __noinline__ void pp_spill_ni(const GTable g, const AggOps ops, unsigned long long kx,
                                                unsigned long long e0, unsigned long long e1, unsigned long long e2,
                                                unsigned long long e3, unsigned *spilled)
{
    const unsigned long long e[QE_MAX_AGGS] = {e0, e1, e2, e3};
    gt_fold_row(g, ops, kx, e);
    if (*reinterpret_cast<volatile unsigned *>(spilled) == 0) atomicExch(spilled, 1u);
}

// Emit n words-per-slot table rows [s0, s1) of a table with `stride`
// words per slot laid out as keys[S] then aggs[a][S] (shared) or as
// AoS slots (HBM spill, aos = true): positions come from one atomic per
// FT slots.  Emitted shared slots are zeroed.
template <bool AOS, int T>
__device__ void pp_emit(const FoldArgs &A, unsigned long long *t, uint64_t S, uint64_t s0, uint64_t s1, int stride)
{
    __shared__ unsigned s_wc[32];
    __shared__ unsigned long long s_first;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t b = s0; b < s1; b += T) {
        const uint64_t i = b + threadIdx.x;
        const bool in = i < s1;
        const unsigned long long kx = in ? (AOS ? __ldcg(t + i * stride) : t[i]) : 0ull;
        const unsigned m = __ballot_sync(QE_FULL_MASK, kx != 0);
        if (lane == 0) s_wc[warp] = __popc(m);
        __syncthreads();
        if (warp == 0) {
            const unsigned c = lane < T / 32 ? s_wc[lane] : 0u;
            const unsigned inc = warp_incl_scan(c);
            if (lane < T / 32) s_wc[lane] = inc - c;
            if (lane == 31) s_first = inc ? atomicAdd(A.emitted, static_cast<unsigned long long>(inc)) : 0ull;
        }
        __syncthreads();
        if (kx) {
            const int64_t pos = static_cast<int64_t>(s_first) + s_wc[warp] + __popc(m & ((1u << lane) - 1));
            auto word = [&](int a) -> unsigned long long {
                return AOS ? __ldcg(t + i * stride + 1 + a) : t[(1 + a) * S + i];
            };
            if (pos < A.out.capacity) {
                A.out.keys[pos] = static_cast<int64_t>(kx ^ GB_SIGN);
                for (int a = 0; a < A.ops.n; a++) A.out.aggs[a][pos] = agg_decode(A.ops.op[a], word(a));
                if (A.cnt >= 0)
                    write_avgs(A.out, pos, A.ops.n, A.cnt, [&](int a) { return agg_decode(A.ops.op[a], word(a)); });
            }
            if (!AOS)
                for (int w = 0; w < stride; w++) t[w * S + i] = 0ull;
        }
        __syncthreads();
    }
}

// Emit the groups of a shared-memory table (keys[S], then aggs[a][S]) and
// zero their slots.  Output positions: every warp-sized group of 32 slots
// counts its occupied slots, the S / 32 counts are scanned in shared memory
// and one global atomic reserves the table's run, so the writes stay in slot
// order, as coalesced as the occupancy allows.
template <int T>
__device__ void pp_emit_table(const FoldArgs &A, unsigned long long *t, int log2s, int stride)
{
    constexpr int NW = T / 32;
    __shared__ unsigned s_cnt[F_EMIT_GROUPS];
    __shared__ unsigned long long s_first;
    const int S = 1 << log2s, G = S >> 5;              // slot groups of 32
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int g = warp; g < G; g += NW) {
        const unsigned m = __ballot_sync(QE_FULL_MASK, t[g * 32 + lane] != 0);
        if (lane == 0) s_cnt[g] = __popc(m);
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the G <= F_EMIT_GROUPS counts, G / 32 per lane
        const int per = (G + 31) >> 5;
        unsigned loc = 0;
        for (int j = 0; j < per; j++) {
            const int g = lane * per + j;
            if (g < G) loc += s_cnt[g];
        }
        const unsigned inc = warp_incl_scan(loc);
        unsigned run = inc - loc;
        for (int j = 0; j < per; j++) {
            const int g = lane * per + j;
            if (g < G) {
                const unsigned c = s_cnt[g];
                s_cnt[g] = run;
                run += c;
            }
        }
        if (lane == 31) s_first = inc ? atomicAdd(A.emitted, static_cast<unsigned long long>(inc)) : 0ull;
    }
    __syncthreads();
    for (int g = warp; g < G; g += NW) {
        const int i = g * 32 + lane;
        const unsigned long long kx = t[i];
        const unsigned m = __ballot_sync(QE_FULL_MASK, kx != 0);
        if (!kx) continue;
        const int64_t pos = static_cast<int64_t>(s_first) + s_cnt[g] + __popc(m & ((1u << lane) - 1));
        if (pos < A.out.capacity) {
            A.out.keys[pos] = static_cast<int64_t>(kx ^ GB_SIGN);
            for (int a = 0; a < A.ops.n; a++) A.out.aggs[a][pos] = agg_decode(A.ops.op[a], t[(1 + a) * S + i]);
            if (A.cnt >= 0) write_avgs(A.out, pos, A.ops.n, A.cnt, [&](int a) { return agg_decode(A.ops.op[a], t[(1 + a) * S + i]); });
        }
        for (int w = 0; w < stride; w++) t[w * S + i] = 0ull;
    }
    __syncthreads();
}

// STAR: the aggregates are [SUM(X*Y), COUNT, MIN(X), MAX(X)] (the shared
// COUNT word then holds a 32-bit count, read back whole: its high half stays 0).
template <int T, int MINB, bool STAR, int FI>
__global__ void __launch_bounds__(T, MINB) k_pp_fold(FoldArgs A)
{
    static_assert(T <= F_RUNS, "a block describes at most F_RUNS runs at a time");
    extern __shared__ __align__(16) unsigned char f_smem[];
    const uint64_t S = uint64_t(1) << A.log2s;
    const int stride = 1 + A.ops.n;
    unsigned long long *tab = reinterpret_cast<unsigned long long *>(f_smem);          // keys[S], aggs[a][S]
    int64_t *rstart = reinterpret_cast<int64_t *>(tab + S * stride);                   // [F_RUNS]
    unsigned *rlen = reinterpret_cast<unsigned *>(rstart + F_RUNS);                    // [F_RUNS]
    __shared__ long long s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Q = 1 << A.log2q;
    const int64_t nsub = int64_t(1) << (A.log2p + A.log2q);
    for (uint64_t i = threadIdx.x; i < S * stride; i += T) tab[i] = 0ull;
    while (true) {
        if (threadIdx.x == 0) s_item = static_cast<long long>(atomicAdd(A.counter, 1ull));
        __syncthreads();
        const int64_t f = s_item;
        if (f >= nsub) break;
        const int64_t p = f >> A.log2q, q = f & (Q - 1);
        const int64_t c0 = A.cpre[p * A.nblk], c1 = A.cpre[(p + 1) * A.nblk];
        for (int64_t cb = c0; cb < c1; cb += T) {      // T <= F_RUNS runs at a time
            const int nr = static_cast<int>(c1 - cb < T ? c1 - cb : T);
            // the runs of sub-part q in chunks cb .. cb + nr
            if (threadIdx.x < nr) {
                const int64_t c = cb + threadIdx.x;
                const uint16_t *o = A.off2 + c * (Q + 1);
                const unsigned o0 = o[q], o1 = o[q + 1];
                rlen[threadIdx.x] = o1 - o0;
                rstart[threadIdx.x] = A.cstart[c] + o0;
            }
            __syncthreads();
            // each warp takes whole runs (about 60 rows each at the planned
            // sizes), r = warp, warp + NW, ...: its lanes read consecutive
            // rows of a run, FI rows per lane a step, and the rows of the
            // warp's next step (the run's next rows, or its next run's
            // first) are loaded while the current step's are folded
            constexpr int NW = T / 32;
            int r = warp;
            unsigned i0 = 0;
            while (r < nr && rlen[r] == 0) r += NW;
            unsigned long long kx[FI], nkx[FI];
            long long xv[FI], yv[FI], nxv[FI], nyv[FI];
            auto load_step = [&](int rr, unsigned ii, unsigned long long (&k)[FI], long long (&x)[FI],
                                 long long (&y)[FI]) {
                const int64_t b0 = rstart[rr];
                const unsigned len = rlen[rr];
#pragma unroll
                for (int t = 0; t < FI; t++) {
                    const unsigned i = ii + t * 32 + lane;
                    k[t] = 0;
                    x[t] = y[t] = 0;
                    if (i < len) {
                        const PartRow *row = A.rows2 + b0 + i;
                        k[t] = __ldcs(&row->kx);
                        x[t] = __ldcs(&row->x);
                        y[t] = __ldcs(&row->y);
                    }
                }
            };
            if (r < nr) load_step(r, 0, kx, xv, yv);
            while (r < nr) {
                int r2 = r;
                unsigned i2 = i0 + 32 * FI;
                if (i2 >= rlen[r]) {
                    i2 = 0;
                    r2 = r + NW;
                    while (r2 < nr && rlen[r2] == 0) r2 += NW;
                }
                if (r2 < nr) load_step(r2, i2, nkx, nxv, nyv);
#pragma unroll
                for (int t = 0; t < FI; t++) {
                    if (!kx[t]) continue;
                    const uint32_t mask = static_cast<uint32_t>(S - 1);
                    uint32_t h = static_cast<uint32_t>(dev_fmix64(kx[t])) & mask;
                    int slot = -1;
                    for (int pr = 0; pr < F_PROBES; pr++) {
                        const unsigned long long cur = reinterpret_cast<volatile unsigned long long *>(tab)[h];
                        if (cur == kx[t]) {
                            slot = static_cast<int>(h);
                            break;
                        }
                        if (cur == 0) {
                            const unsigned long long old = atomicCAS(tab + h, 0ull, kx[t]);
                            if (old == 0 || old == kx[t]) {
                                slot = static_cast<int>(h);
                                break;
                            }
                        }
                        h = (h + 1) & mask;
                    }
                    if constexpr (STAR) {
                        // [SUM(X*Y), COUNT, MIN(X), MAX(X)]: the encodings
                        // inline, COUNT as a 32-bit counter in its word's
                        // low half (a sub-part has fewer than 2^32 rows)
                        const unsigned long long v = static_cast<unsigned long long>(xv[t]) *
                                                     static_cast<unsigned long long>(yv[t]);
                        const unsigned long long emin = ~(static_cast<unsigned long long>(xv[t]) ^ GB_SIGN);
                        const unsigned long long emax = static_cast<unsigned long long>(xv[t]) ^ GB_SIGN;
                        if (slot >= 0) {
                            smem_add64(tab + S + slot, v);
                            atomicAdd(reinterpret_cast<unsigned *>(tab + 2 * S + slot), 1u);
                            unsigned long long *cmin = tab + 3 * S + slot, *cmax = tab + 4 * S + slot;
                            if (*cmin < emin) atomicMax(cmin, emin);
                            if (*cmax < emax) atomicMax(cmax, emax);
                        } else {
                            pp_spill_ni(A.spill, A.ops, kx[t], v, 1ull, emin, emax, A.spilled);
                        }
                    } else {
                        unsigned long long e[QE_MAX_AGGS];
#pragma unroll
                        for (int a = 0; a < QE_MAX_AGGS; a++) e[a] = a < A.ops.n ? pp_value(A, a, xv[t], yv[t]) : 0ull;
                        if (slot >= 0) {
#pragma unroll
                            for (int a = 0; a < QE_MAX_AGGS; a++)
                                if (a < A.ops.n) st_update(tab + (1 + a) * S + slot, A.ops.op[a], e[a]);
                        } else {
                            pp_spill_ni(A.spill, A.ops, kx[t], e[0], e[1], e[2], e[3], A.spilled);
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < FI; t++) {
                    kx[t] = nkx[t];
                    xv[t] = nxv[t];
                    yv[t] = nyv[t];
                }
                r = r2;
                i0 = i2;
            }
            __syncthreads();
        }
        pp_emit_table<T>(A, tab, A.log2s, stride);
    }
}

// The spill table's groups, appended to the output.
__global__ void __launch_bounds__(FT) k_pp_spill_emit(FoldArgs A)
{
    if (*A.spilled == 0) return;           // nothing spilled: the table is empty
    const uint64_t slots = A.spill.mask + 1;
    const uint64_t per = (slots + gridDim.x - 1) / gridDim.x;
    const uint64_t s0 = blockIdx.x * per, s1 = s0 + per < slots ? s0 + per : slots;
    pp_emit<true, FT>(A, A.spill.words, 0, s0, s1, A.spill.stride);
}

__global__ void k_pp_count_out(const unsigned long long *emitted, int64_t capacity, int64_t *ngroups, qe_dev_status *st)
{
    const int64_t n = static_cast<int64_t>(*emitted);
    *ngroups = n;
    if (n > capacity) dev_report(st, QE_ERR_CAPACITY, n);
}

}  // namespace

// Parameters of the partitioned group-by for `groups` (at most) groups:
// parts of the scatter (log2p; at most 256, so a block writes few pages at
// a time), sub-parts per part (log2q) and shared-table slots (log2s), so
// that a sub-part's groups fill its shared table to about 60 % on average.
struct PartPlan {
    int log2p = 0, log2q = 0, log2s = 0;
};

static PartPlan part_plan(int64_t groups, int naggs, size_t smem_budget, int log2p_hint, int log2q_hint)
{
    PartPlan pl;
    // shared-table slots: the largest power of two whose table (and the run
    // descriptors) fits the shared-memory budget, at most 4096
    int ls = 12;
    while (ls > 6 && ((size_t(1) << ls) * (1 + naggs) * 8 + F_RUNS * 12 + 64) > smem_budget) ls--;
    pl.log2s = ls;
    const uint64_t per_sub = (uint64_t(1) << ls) * 6 / 10;      // groups per sub-part at ~60 % load
    const uint64_t subs = (static_cast<uint64_t>(groups > 0 ? groups : 1) + per_sub - 1) / per_sub;
    int lt = 0;
    while ((uint64_t(1) << lt) < subs) lt++;
    pl.log2p = log2p_hint > 0 ? log2p_hint : (lt < 8 ? (lt > 1 ? lt : 1) : 8);
    pl.log2q = lt > pl.log2p ? lt - pl.log2p : 0;
    if (pl.log2q > 8) pl.log2q = 8;
    if (log2q_hint >= 0) pl.log2q = log2q_hint;
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
    // fold shape: one 1,024-thread block per SM with the largest shared
    // table, or two 512-thread blocks with half-size tables each, so that
    // one block's hand-over between sub-parts overlaps the other's rows
    const bool fold2 = ctx->tune_gb_fold2 != 0;
    const size_t smem_per_sm = ctx->smem_optin > 2048 ? ctx->smem_optin - 2048 : 0;
    const size_t smem_budget = fold2 ? smem_per_sm / 2 - 1024 : smem_per_sm;
    const PartPlan pl = part_plan(groups, P.ops.n, smem_budget, ctx->tune_gb_part_log2p, ctx->tune_gb_part_log2q);
    const int parts = 1 << pl.log2p, Q = 1 << pl.log2q;
    const int nblk = ctx->num_sms;
    const int64_t tr = static_cast<int64_t>(PPT) * PP_ITEMS;
    int64_t rpb = qe_ceil_div(qe_ceil_div(P.n > 0 ? P.n : 1, nblk), tr) * tr;
    const int64_t m = static_cast<int64_t>(parts) * nblk;
    // chunks: at most one per SPLIT_ROWS rows plus one per segment
    const int64_t max_chunks = P.n / SPLIT_ROWS + m + 1;
    // spill table for keys that find no shared slot (skewed hashes): 1/32 of
    // the groups, at least 128K (it is cleared on every call)
    const int64_t spill_cap = groups / 32 > 131072 ? groups / 32 : 131072;
    uint64_t spill_slots = 64;
    while (spill_slots < static_cast<uint64_t>(2 * spill_cap)) spill_slots <<= 1;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t b_rows = up(static_cast<size_t>(P.n) * sizeof(PartRow));
    const size_t b_cnt = up(m * 4), b_seg = up(m * 8), b_fill = up(m * 4), b_cpre = up((m + 1) * 8);
    const size_t b_off2 = up(static_cast<size_t>(max_chunks) * (Q + 1) * 2), b_cstart = up(max_chunks * 8);
    const size_t b_spill = up(spill_slots * stride * 8);
    const size_t b_ctr = 256;
    void *mem = nullptr;
    qe_status st = qe_alloc(ctx, &mem,
                            2 * b_rows + b_cnt + b_seg + b_fill + b_cpre + b_off2 + b_cstart + b_spill + b_ctr, s);
    if (st != QE_OK) return st;
    char *c = static_cast<char *>(mem);
    PartArgs A{};
    A.P = P;
    A.log2p = pl.log2p;
    A.nblk = nblk;
    A.rows_per_blk = rpb;
    A.count_all = P.lo_slot != QE_JOIN_PAYLOAD;
    A.rows = reinterpret_cast<PartRow *>(c);
    PartRow *rows2 = reinterpret_cast<PartRow *>(c + b_rows);
    char *q = c + 2 * b_rows;
    A.cnt = reinterpret_cast<uint32_t *>(q);
    A.seg = reinterpret_cast<int64_t *>(q + b_cnt);
    A.fill = reinterpret_cast<uint32_t *>(q + b_cnt + b_seg);
    int64_t *cpre = reinterpret_cast<int64_t *>(q + b_cnt + b_seg + b_fill);
    uint16_t *off2 = reinterpret_cast<uint16_t *>(q + b_cnt + b_seg + b_fill + b_cpre);
    int64_t *cstart = reinterpret_cast<int64_t *>(q + b_cnt + b_seg + b_fill + b_cpre + b_off2);
    char *zero = q + b_cnt + b_seg + b_fill + b_cpre + b_off2 + b_cstart;   // spill table, counters
    cudaError_t e = cudaMemsetAsync(zero, 0, b_spill + b_ctr, s);
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(zero + b_spill);

    SplitArgs SA{};
    SA.log2p = pl.log2p;
    SA.log2q = pl.log2q;
    SA.nblk = nblk;
    SA.m = m;
    SA.nrows = P.n;
    SA.st = ctx->dstat;
    SA.seg = A.seg;
    SA.fill = A.fill;
    SA.cpre = cpre;
    SA.rows = A.rows;
    SA.rows2 = rows2;
    SA.off2 = off2;
    SA.cstart = cstart;
    SA.counter = ctr;

    FoldArgs F{};
    F.ops = P.ops;
    for (int a = 0; a < QE_MAX_AGGS; a++) F.src[a] = P.src[a];
    F.log2p = pl.log2p;
    F.log2q = pl.log2q;
    F.nblk = nblk;
    F.log2s = pl.log2s;
    F.cnt = -1;
    for (int a = 0; a < QE_MAX_AGGS; a++)
        if (out->avg[a]) F.cnt = agg_count_index(P.ops);
    F.cpre = cpre;
    F.off2 = off2;
    F.cstart = cstart;
    F.rows2 = rows2;
    F.spill.words = reinterpret_cast<unsigned long long *>(zero);
    F.spill.mask = spill_slots - 1;
    F.spill.stride = stride;
    F.spill.capacity = out->capacity;
    F.spill.st = ctx->dstat;
    F.counter = ctr + 1;
    F.emitted = ctr + 2;
    F.spilled = reinterpret_cast<unsigned *>(ctr + 3);
    F.out = *out;
    F.st = ctx->dstat;

    const size_t sm_count = static_cast<size_t>(parts) * 4;
    const size_t sm_scatter = pp_scatter_smem(parts);
    const size_t sm_split = pp_split_smem(pl.log2q);
    const size_t sm_fold = (size_t(1) << pl.log2s) * stride * 8 + F_RUNS * 12 + 64;
    // the scatter kernel: the star shape's register-prefetched loop, or the generic one
    const int skind = ctx->tune_force_generic ? -1 : pp_star_kind(P);
    const void *kscatter = reinterpret_cast<const void *>(k_pp_scatter);
    if (skind >= 0) {
        PipeSpec &Qs = A.P;
        star_predicate(Qs);
        kscatter = Qs.type[Qs.lo_slot] == QE_I64 ? pp_star_kernel<true>(skind) : pp_star_kernel<false>(skind);
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kscatter, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_scatter));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pp_split, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_split));
    const bool star_aggs = P.ops.n == 4 && P.ops.op[0] == QE_SUM && P.src[0] == SRC_XY && P.ops.op[1] == QE_COUNT &&
                           P.ops.op[2] == QE_MIN && P.src[2] == SRC_X && P.ops.op[3] == QE_MAX && P.src[3] == SRC_X;
    const void *kfold = fold2 ? (star_aggs ? reinterpret_cast<const void *>(k_pp_fold<FT / 2, 2, true, 1>)
                                           : reinterpret_cast<const void *>(k_pp_fold<FT / 2, 2, false, 1>))
                              : (star_aggs ? reinterpret_cast<const void *>(k_pp_fold<FT, 1, true, FOLD_FI>)
                                           : reinterpret_cast<const void *>(k_pp_fold<FT, 1, false, FOLD_FI>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kfold, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm_fold));
    if (e == cudaSuccess && P.n > 0) {
        {
            ProfScope prof(ctx, "part_count", s);
            k_pp_count<<<nblk, PPT, sm_count, s>>>(A);
            QE_LAUNCHED(ctx);
        }
        k_pp_scan<<<1, PPT, 0, s>>>(A.cnt, m, A.seg, 0, nullptr);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            ProfScope prof(ctx, "part_scatter_rows", s);
            void *args[] = {&A};
            e = cudaLaunchKernel(kscatter, dim3(nblk), dim3(PPT), args, sm_scatter, s);
            QE_LAUNCHED(ctx);
        }
        if (e == cudaSuccess) {
            k_pp_scan<<<1, PPT, 0, s>>>(A.fill, m, cpre, SPLIT_ROWS, cpre + m);
            QE_LAUNCHED(ctx);
            ProfScope prof(ctx, "part_split", s);
            k_pp_split<<<nblk * SP_BLOCKS, SPT, sm_split, s>>>(SA);
            QE_LAUNCHED(ctx);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            ProfScope prof(ctx, "part_fold", s);
            void *fargs[] = {&F};
            e = cudaLaunchKernel(kfold, dim3(fold2 ? 2 * nblk : nblk), dim3(fold2 ? FT / 2 : FT), fargs, sm_fold, s);
            QE_LAUNCHED(ctx);
        }
        if (e == cudaSuccess) {
            k_pp_spill_emit<<<nblk, FT, 0, s>>>(F);
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
