// qe_pipe_core.cuh -- the per-row core of the fused pipeline, shared by the
// single-pipeline kernel (qe_pipeline.cu) and the batched persistent kernel
// (qe_batch.cu).
//
// A tile is ITEMS x THREADS consecutive fact rows.  Each thread of a block
// owns ITEMS rows of the tile, THREADS rows apart, so every column read is a
// coalesced warp access straight from global memory with an evict-first
// (streaming) hint; the star-shape loop also loads the next tile's columns
// into registers while the current tile is processed, which keeps the loads
// in flight in the register file rather than in shared memory (shared memory
// holds the group table).
#pragma once

#include <climits>
#include <cstdlib>

#include "qe_internal.cuh"

#define PIPE_THREADS 1024
#define PIPE_WARPS (PIPE_THREADS / 32)

enum { SRC_NONE = 0, SRC_X = 1, SRC_Y = 2, SRC_XY = 3 };

// Device view of one pipeline.  Column slots index the columns it reads.
struct PipeSpec {
    int64_t n;                          // fact rows
    int32_t ncol;                       // columns read
    int32_t pad0;
    const void *col[QE_MAX_COLS];
    int32_t type[QE_MAX_COLS];
    int32_t npreds;
    int32_t pslot[QE_MAX_PREDS], pop[QE_MAX_PREDS];
    int64_t plo[QE_MAX_PREDS], phi[QE_MAX_PREDS];
    int32_t has_join, fk_slot, hi_slot, lo_slot;   // lo_slot == QE_JOIN_PAYLOAD: join payload
    int32_t x_slot, y_slot;
    int32_t src[QE_MAX_AGGS];
    AggOps ops;
    HtView ht;
    GTable g;                           // HBM hash table (spills, hash layouts)
    DenseKey dk;                        // dense layout of the group key
    unsigned long long *gdense;         // HBM dense table (TM_GLOBAL_DENSE), AoS
    // star kernel: direct column pointers and 32-bit bounds, read from the
    // parameter bank as instruction operands instead of held in registers
    const int32_t *s_pred, *s_fk, *s_y;
    const void *s_hi;
    const long long *s_x;
    const void *s_lo;                   // key column of the fact-keyed star kinds
    int32_t p0_lo, p0_hi, p0_neg, s_h8;
    int32_t s_l8, s_has_hi;
    int32_t s_hmin, s_lmin;
    uint32_t s_hspan, s_lspan, s_ns;
    int32_t join_kind;                  // qe_join_kind
};

// Where a block aggregates.
enum { TM_SMEM_HASH = 0, TM_SMEM_DENSE = 1, TM_GLOBAL_DENSE = 2, TM_GLOBAL_HASH = 3 };

struct TableCfg {
    int mode;
    int S;        // shared-memory hash slots (TM_SMEM_HASH)
    int log2S;
};

// ------------------------------------------------------------ row values
// Column slot value of fact row `grow` (streaming load, sign-extended).
__device__ __forceinline__ int64_t ld_slot(const PipeSpec &P, int slot, int64_t grow)
{
    return dev_col_stream(P.col[slot], P.type[slot], grow);
}

struct RowVals {
    int64_t key_a;   // foreign key (join) or low key half
    int64_t lo;      // low key half from a fact column, with a join
    int64_t hi;
    int64_t x, y;
    bool ok;
};

// Predicates and the columns a surviving row needs.
__device__ __forceinline__ RowVals row_load(const PipeSpec &P, int64_t grow, bool in_range)
{
    RowVals v;
    bool ok = in_range;
#pragma unroll
    for (int p = 0; p < QE_MAX_PREDS; p++)
        if (p < P.npreds && ok) ok = dev_cmp(ld_slot(P, P.pslot[p], grow), P.pop[p], P.plo[p], P.phi[p]);
    v.ok = ok;
    v.key_a = 0;
    v.lo = 0;
    v.hi = 0;
    v.x = 0;
    v.y = 0;
    if (ok) {
        v.key_a = ld_slot(P, P.has_join ? P.fk_slot : P.lo_slot, grow);
        if (P.has_join && P.lo_slot >= 0) v.lo = ld_slot(P, P.lo_slot, grow);
        if (P.hi_slot >= 0) v.hi = ld_slot(P, P.hi_slot, grow);
        if (P.x_slot >= 0) v.x = ld_slot(P, P.x_slot, grow);
        if (P.y_slot >= 0) v.y = ld_slot(P, P.y_slot, grow);
    }
    return v;
}

static __device__ __noinline__ bool ht_lookup_open_ni(const HtView h, int32_t key, int32_t *pay)
{
    int32_t p = 0;
    bool hit = ht_lookup(h, key, p);
    *pay = p;
    return hit;
}

// Join probe.  Dense tables are looked up inline (one L2 read), open tables
// out of line.
__device__ __forceinline__ bool probe(const HtView &h, int32_t key, int32_t &pay)
{
    if (h.layout == QE_HT_DENSE) {
        const uint32_t s = static_cast<uint32_t>(key) - static_cast<uint32_t>(h.key_min);
        if (s >= h.range) return false;
        pay = ht_ld(h, h.payload + s);
        if (!h.full && !((ht_ld(h, h.bitmap + (s >> 5)) >> (s & 31)) & 1u)) return false;
        return true;
    }
    return ht_lookup_open_ni(h, key, &pay);
}

// Membership of a key (semi- and anti-join): probe() without the payload,
// open addressing out of line.
__device__ __forceinline__ bool member(const HtView &h, int32_t key)
{
    if (h.layout == QE_HT_DENSE) {
        const uint32_t s = static_cast<uint32_t>(key) - static_cast<uint32_t>(h.key_min);
        return s < h.range && (h.full || ((ht_ld(h, h.bitmap + (s >> 5)) >> (s & 31)) & 1u));
    }
    int32_t pay;
    return ht_lookup_open_ni(h, key, &pay);
}

// ------------------------------------------------------------ group table
// Shared-memory slot hash: multiplicative (Fibonacci) hashing of the
// 64-bit stored key, top log2S bits.
__device__ __forceinline__ uint32_t st_hash(unsigned long long kx, int log2S)
{
    return static_cast<uint32_t>((kx * 0x9E3779B97F4A7C15ull) >> (64 - log2S));
}

static __device__ __noinline__ int st_find_slow(unsigned long long *keys, uint32_t mask, unsigned long long kx, uint32_t h)
{
    for (int p = 0; p < 64; p++) {
        unsigned long long cur = reinterpret_cast<volatile unsigned long long *>(keys)[h];
        if (cur == kx) return static_cast<int>(h);
        if (cur == 0) {
            unsigned long long old = atomicCAS(keys + h, 0ull, kx);
            if (old == 0 || old == kx) return static_cast<int>(h);
        }
        h = (h + 1) & mask;
    }
    return -1;
}

static __device__ __noinline__ void spill_row_ni(const GTable g, const AggOps ops, unsigned long long kx, unsigned long long e0,
                                          unsigned long long e1, unsigned long long e2, unsigned long long e3)
{
    unsigned long long e[QE_MAX_AGGS] = {e0, e1, e2, e3};
    gt_fold_row(g, ops, kx, e);
}

__device__ __forceinline__ unsigned long long agg_value_enc(const PipeSpec &P, int a, const RowVals &v)
{
    const int src = P.src[a];
    const int64_t val = src == SRC_X ? v.x
                      : src == SRC_Y ? v.y
                      : src == SRC_XY ? static_cast<int64_t>(static_cast<uint64_t>(v.x) * static_cast<uint64_t>(v.y))
                                      : 0;
    return agg_encode(P.ops.op[a], val);
}

// 64-bit add into a shared-memory cell as 32-bit atomics: the low half,
// then the high half plus the carry out of the low half (read from the value
// the first atomic replaced).  32-bit shared atomics cost far less than
// 64-bit ones; the cell is read whole only after a barrier.
__device__ __forceinline__ void smem_add64(unsigned long long *cell, unsigned long long e)
{
    unsigned *w = reinterpret_cast<unsigned *>(cell);   // little-endian: w[0] low, w[1] high
    const uint32_t lo = static_cast<uint32_t>(e), hi = static_cast<uint32_t>(e >> 32);
    const uint32_t old = atomicAdd(w, lo);
    const uint32_t up = hi + (old + lo < old ? 1u : 0u);
    if (up) atomicAdd(w + 1, up);
}

// Update of one shared-memory aggregate cell: ADD kinds add (in 32-bit
// halves); MAX kinds read the cell first (a stale read can only cause a
// redundant atomic, never a lost update, since cells only grow).
__device__ __forceinline__ void st_update(unsigned long long *cell, int op, unsigned long long e)
{
    if (op == QE_SUM || op == QE_COUNT) {
        smem_add64(cell, e);
    } else if (*cell < e) {
        atomicMax(cell, e);
    }
}

// Update of one HBM aggregate cell (same rule as st_update).
__device__ __forceinline__ void gd_update(unsigned long long *cell, int op, unsigned long long e)
{
    if (op == QE_SUM || op == QE_COUNT) {
        atomicAdd(cell, e);
    } else if (*cell < e) {
        atomicMax(cell, e);
    }
}

// Fold a surviving row (key parts hi / lo) into the block's table.
__device__ __forceinline__ void fold_row(const PipeSpec &P, const TableCfg &T, unsigned long long *sm, int64_t hi,
                                         int64_t lo, const RowVals &v)
{
    int64_t key = lo;
    if (P.hi_slot >= 0) key = static_cast<int64_t>((static_cast<uint64_t>(hi) << 32) | static_cast<uint32_t>(lo));
    const unsigned long long kx = static_cast<unsigned long long>(key) ^ GB_SIGN;
    if (kx == 0) {
        dev_report(P.g.st, QE_ERR_RESERVED_KEY, 0);
        return;
    }
    unsigned long long e[QE_MAX_AGGS];
#pragma unroll
    for (int a = 0; a < QE_MAX_AGGS; a++) e[a] = a < P.ops.n ? agg_value_enc(P, a, v) : 0;
    if (T.mode == TM_SMEM_DENSE || T.mode == TM_GLOBAL_DENSE) {
        const int64_t idx = dense_index(P.dk, hi, lo);
        if (idx >= 0) {
            if (T.mode == TM_SMEM_DENSE) {
                const uint64_t ns = P.dk.nslots;
#pragma unroll
                for (int a = 0; a < QE_MAX_AGGS; a++)
                    if (a < P.ops.n) st_update(sm + a * ns + idx, P.ops.op[a], e[a]);
                if (P.dk.hidden) smem_add64(sm + P.ops.n * ns + idx, 1ull);
            } else {
                unsigned long long *cell = P.gdense + idx * P.dk.stride;
#pragma unroll
                for (int a = 0; a < QE_MAX_AGGS; a++)
                    if (a < P.ops.n) gd_update(cell + a, P.ops.op[a], e[a]);
                if (P.dk.hidden) atomicAdd(cell + P.ops.n, 1ull);
            }
            return;
        }
    } else if (T.mode == TM_SMEM_HASH) {
        const uint32_t mask = static_cast<uint32_t>(T.S - 1);
        const uint32_t h = st_hash(kx, T.log2S);
        const int slot = sm[h] == kx ? static_cast<int>(h) : st_find_slow(sm, mask, kx, h);
        if (slot >= 0) {
#pragma unroll
            for (int a = 0; a < QE_MAX_AGGS; a++)
                if (a < P.ops.n) st_update(sm + (a + 1) * T.S + slot, P.ops.op[a], e[a]);
            return;
        }
    }
    spill_row_ni(P.g, P.ops, kx, e[0], e[1], e[2], e[3]);
}

static __device__ __noinline__ int64_t gt_find_insert_ni(const GTable g, unsigned long long kx)
{
    return gt_find_insert(g, kx);
}

// Fold ITEMS rows into the HBM hash table: every row's first probe is read
// before any row is folded, so the rows' DRAM round trips overlap (a row
// whose key is not in its home slot takes the out-of-line probe loop).
template <int ITEMS>
__device__ __forceinline__ void fold_rows_ghash(const PipeSpec &P, const bool (&ok)[ITEMS], const int64_t (&hi)[ITEMS],
                                                const int64_t (&lo)[ITEMS], const RowVals (&v)[ITEMS])
{
    unsigned long long kx[ITEMS], cur[ITEMS];
    uint64_t home[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        int64_t key = lo[k];
        if (P.hi_slot >= 0)
            key = static_cast<int64_t>((static_cast<uint64_t>(hi[k]) << 32) | static_cast<uint32_t>(lo[k]));
        kx[k] = static_cast<unsigned long long>(key) ^ GB_SIGN;
        home[k] = gb_hash(kx[k]) & P.g.mask;
        cur[k] = ok[k] ? __ldcg(P.g.words + home[k] * P.g.stride) : 0;
    }
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        if (!ok[k]) continue;
        if (kx[k] == 0) {
            dev_report(P.g.st, QE_ERR_RESERVED_KEY, 0);
            continue;
        }
        const int64_t s = cur[k] == kx[k] ? static_cast<int64_t>(home[k]) : gt_find_insert_ni(P.g, kx[k]);
        if (s < 0) continue;
        unsigned long long *cell = P.g.words + s * P.g.stride + 1;
#pragma unroll
        for (int a = 0; a < QE_MAX_AGGS; a++)
            if (a < P.ops.n) agg_fold(cell + a, P.ops.op[a], agg_value_enc(P, a, v[k]));
    }
}

// Join probe of a loaded row; false when the row does not join.  Sets the
// key parts.
__device__ __forceinline__ bool row_probe(const PipeSpec &P, const RowVals &v, int64_t &hi, int64_t &lo)
{
    if (!v.ok) return false;
    hi = v.hi;
    lo = v.key_a;
    if (P.has_join) {
        const int32_t key = static_cast<int32_t>(v.key_a);
        if (P.join_kind != QE_JOIN_INNER) {
            // the semi-join keeps rows with a match, the anti-join rows without one
            if (member(P.ht, key) == (P.join_kind == QE_JOIN_ANTI)) return false;
            lo = v.lo;
        } else {
            int32_t pay = 0;
            if (!probe(P.ht, key, pay)) return false;
            lo = P.lo_slot == QE_JOIN_PAYLOAD ? static_cast<int64_t>(pay) : v.lo;
        }
    }
    return true;
}

// Zero the block table.
__device__ __forceinline__ void table_zero(const PipeSpec &P, const TableCfg &T, unsigned long long *sm)
{
    if (T.mode == TM_SMEM_HASH) st_zero(sm, T.S, P.ops.n);
    if (T.mode == TM_SMEM_DENSE)
        for (uint64_t i = threadIdx.x; i < P.dk.nslots * P.dk.stride; i += blockDim.x) sm[i] = 0;
}

// Merge the block table into the HBM tables (after a __syncthreads()).  In
// a direct array word w of slot i is sm[w * nslots + i].  The star kernels
// keep the COUNT word (word 1) as 32-bit counters (narrow >= 1) and, for
// small arrays, the SUM word (word 0) as two 32-bit halves, low halves then
// high halves (narrow == 2), each at the start of the word's region:
// 32-bit shared-memory atomics cost much less than 64-bit ones.
__device__ __forceinline__ unsigned long long dense_word(const unsigned long long *sm, uint64_t ns, int w, uint64_t i,
                                                        int narrow)
{
    if (narrow == 2 && w == 0) {
        const unsigned *h = reinterpret_cast<const unsigned *>(sm);
        return static_cast<unsigned long long>(h[i]) | (static_cast<unsigned long long>(h[ns + i]) << 32);
    }
    if (narrow && w == 1) return reinterpret_cast<const unsigned *>(sm + ns)[i];
    return sm[w * ns + i];
}

__device__ __forceinline__ void table_flush(const PipeSpec &P, const TableCfg &T, unsigned long long *sm,
                                            int narrow = 0)
{
    if (T.mode == TM_SMEM_HASH) st_flush(sm, T.S, P.ops, P.g);
    if (T.mode != TM_SMEM_DENSE) return;
    const uint64_t ns = P.dk.nslots;
    for (uint64_t i = threadIdx.x; i < ns; i += blockDim.x) {
        if (dense_word(sm, ns, P.dk.occ, i, narrow) == 0) continue;
        if (P.gdense) {
            unsigned long long *cell = P.gdense + i * P.dk.stride;
            for (int w = 0; w < P.dk.stride; w++)
                gd_update(cell + w, w < P.ops.n ? P.ops.op[w] : QE_COUNT, dense_word(sm, ns, w, i, narrow));
        } else {
            unsigned long long e[QE_MAX_AGGS];
#pragma unroll
            for (int a = 0; a < QE_MAX_AGGS; a++) e[a] = a < P.ops.n ? dense_word(sm, ns, a, i, narrow) : 0;
            const unsigned long long kx = static_cast<unsigned long long>(dense_key(P.dk, i)) ^ GB_SIGN;
            gt_fold_row(P.g, P.ops, kx, e);
        }
    }
}

// ------------------------------------------------------------ star shape
// One int32 predicate column, an int32 foreign key joined through a dense
// table, the group key (hi column, join payload) in a direct array and the
// aggregates [SUM(x*y), COUNT, MIN(x), MAX(x)] with x int64, y int32.  One
// block processes the tiles of THREADS x ITEMS rows starting at r0, r0 +
// stride, ... below r1; all columns of the next tile are loaded into
// registers while the current tile is processed, so the register file holds
// the loads in flight.
// Largest direct array (slots) whose SUM the star kernels keep in 32-bit halves.
constexpr uint64_t STAR_NSUM_SLOTS = 1024;

// Kinds of the star shape: the group key's low part is the inner join's
// payload; or it is a fact column and the join is a semi- or anti-join
// (membership in a dense key set), or there is no join.
enum { STAR_INNER = 0, STAR_SEMI = 1, STAR_ANTI = 2, STAR_NONE = 3 };

// The row work of one star tile, in two steps: star_lookup (predicate and
// dense lookup or membership test of the ITEMS rows a thread holds; bit k
// of cin marks row k as inside the range; cl holds the key column of the
// kinds other than STAR_INNER) and star_fold (direct-array, or spilled
// hash, update of the rows that pass).
template <int ITEMS, int JK = STAR_INNER, bool L2H = false>
__device__ __forceinline__ void star_lookup(const PipeSpec &P, const int (&cd)[ITEMS], const int (&cf)[ITEMS],
                                            const int (&cl)[ITEMS], unsigned cin, uint64_t pol_keep, bool (&ok)[ITEMS],
                                            int32_t (&pay)[ITEMS])
{
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        const bool pass = (cd[k] >= P.p0_lo && cd[k] <= P.p0_hi) != static_cast<bool>(P.p0_neg);
        if constexpr (JK == STAR_INNER) {
            const uint32_t ks = static_cast<uint32_t>(cf[k]) - static_cast<uint32_t>(P.ht.key_min);
            const bool hit = ((cin >> k) & 1u) && pass && ks < P.ht.range;
            if constexpr (L2H)
                pay[k] = hit ? ld_lookup_i32(P.ht.payload + ks, pol_keep) : 0;
            else
                pay[k] = hit ? ht_ld(P.ht, P.ht.payload + ks) : 0;
            ok[k] = hit && (P.ht.full || ((ht_ld(P.ht, P.ht.bitmap + (ks >> 5)) >> (ks & 31)) & 1u));
        } else if constexpr (JK == STAR_NONE) {
            pay[k] = cl[k];
            ok[k] = ((cin >> k) & 1u) && pass;
        } else {
            // membership: in the key range and (a full range or) its bit set
            const uint32_t ks = static_cast<uint32_t>(cf[k]) - static_cast<uint32_t>(P.ht.key_min);
            const bool live = ((cin >> k) & 1u) && pass;
            const bool in = live && ks < P.ht.range &&
                            (P.ht.full || ((ht_ld(P.ht, P.ht.bitmap + (ks >> 5)) >> (ks & 31)) & 1u));
            pay[k] = cl[k];
            ok[k] = live && (JK == STAR_SEMI ? in : !in);
        }
    }
}

template <bool GLOBAL, int ITEMS, bool NSUM, int JK = STAR_INNER>
__device__ __forceinline__ void star_fold(const PipeSpec &P, unsigned long long *sm, const int (&ch)[ITEMS],
                                          const int (&cq)[ITEMS], const long long (&cx)[ITEMS], const bool (&ok)[ITEMS],
                                          const int32_t (&pay)[ITEMS])
{
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        if (!ok[k]) continue;
        const uint32_t hh = static_cast<uint32_t>(ch[k]) - static_cast<uint32_t>(P.s_hmin);
        const uint32_t ll = static_cast<uint32_t>(pay[k]) - static_cast<uint32_t>(P.s_lmin);
        const unsigned long long v = static_cast<unsigned long long>(cx[k]) * static_cast<unsigned long long>(cq[k]);
        const unsigned long long emin = ~(static_cast<unsigned long long>(cx[k]) ^ GB_SIGN);
        const unsigned long long emax = static_cast<unsigned long long>(cx[k]) ^ GB_SIGN;
        if (hh < P.s_hspan && ll < P.s_lspan) {
            const uint32_t idx = hh * P.s_lspan + ll;
            if (!QE_DCHECK(P.g.st, idx < P.s_ns, idx)) continue;
            if (GLOBAL) {
                unsigned long long *cell = P.gdense + static_cast<uint64_t>(idx) * 4;
                atomicAdd(cell, v);
                atomicAdd(cell + 1, 1ull);
                if (cell[2] < emin) atomicMax(cell + 2, emin);
                if (cell[3] < emax) atomicMax(cell + 3, emax);
            } else {
                if (NSUM) {
                    // SUM as 32-bit halves: the low half's carry, read from
                    // the value the atomic replaced, goes into the high half
                    unsigned *slo = reinterpret_cast<unsigned *>(sm);
                    const uint32_t lo = static_cast<uint32_t>(v), hi = static_cast<uint32_t>(v >> 32);
                    const uint32_t old = atomicAdd(slo + idx, lo);
                    const uint32_t up = hi + (old + lo < old ? 1u : 0u);
                    if (up) atomicAdd(slo + P.s_ns + idx, up);
                } else {
                    atomicAdd(sm + idx, v);
                }
                // COUNT as 32 bits: a block's table counts its share of the rows, far below 2^32
                atomicAdd(reinterpret_cast<unsigned *>(sm + P.s_ns) + idx, 1u);
                if (sm[2 * P.s_ns + idx] < emin) atomicMax(sm + 2 * P.s_ns + idx, emin);
                if (sm[3 * P.s_ns + idx] < emax) atomicMax(sm + 3 * P.s_ns + idx, emax);
            }
        } else {
            // the group key: (hi, lo) packed, or lo alone (sign-extended) without a hi part
            const int64_t key = JK == STAR_INNER || P.s_has_hi
                                    ? static_cast<int64_t>((static_cast<uint64_t>(static_cast<int64_t>(ch[k])) << 32) |
                                                           static_cast<uint32_t>(pay[k]))
                                    : static_cast<int64_t>(pay[k]);
            const unsigned long long kx = static_cast<unsigned long long>(key) ^ GB_SIGN;
            if (kx == 0) {
                dev_report(P.g.st, QE_ERR_RESERVED_KEY, 0);
            } else {
                const unsigned long long e[QE_MAX_AGGS] = {v, 1ull, emin, emax};
                gt_fold_row(P.g, P.ops, kx, e);
            }
        }
    }
}

// Star row loop: one block processes the tiles of THREADS x ITEMS rows
// starting at r0, r0 + stride, ... below r1; all columns of the next tile are
// loaded into registers while the current one is processed, so the register
// file holds the loads in flight.
template <bool GLOBAL, int ITEMS, int THREADS, bool NSUM, int JK = STAR_INNER, bool L2H = false>
__device__ __forceinline__ void star_range(const PipeSpec &P, unsigned long long *sm, int64_t r0, int64_t r1,
                                           int64_t stride)
{
    int d[ITEMS], f[ITEMS], h[ITEMS], l[ITEMS], q[ITEMS];
    long long x[ITEMS];
    unsigned inmask = 0;
    // L2H: fact columns evict first, payload lookups evict last
    const uint64_t pol_stream = L2H ? l2_policy_evict_first() : 0;
    const uint64_t pol_keep = L2H ? l2_policy_evict_last() : 0;
    auto ld32 = [&](const int32_t *a) -> int { return L2H ? ld_hint_i32(a, pol_stream) : __ldcs(a); };
    auto ld8 = [&](const signed char *a) -> int {
        return L2H ? ld_hint_s8(a, pol_stream) : static_cast<int>(__ldcs(a));
    };
    auto load = [&](int64_t t0) {
        inmask = 0;
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const int64_t r = t0 + k * THREADS + threadIdx.x;
            const bool in = r < r1;
            inmask |= in ? (1u << k) : 0u;
            d[k] = in ? ld32(P.s_pred + r) : 0;
            f[k] = JK != STAR_NONE && in ? ld32(P.s_fk + r) : 0;
            h[k] = (JK == STAR_INNER || P.s_has_hi) && in
                       ? (P.s_h8 ? ld8(static_cast<const signed char *>(P.s_hi) + r)
                                 : ld32(static_cast<const int32_t *>(P.s_hi) + r))
                       : 0;
            l[k] = JK != STAR_INNER && in
                       ? (P.s_l8 ? ld8(static_cast<const signed char *>(P.s_lo) + r)
                                 : ld32(static_cast<const int32_t *>(P.s_lo) + r))
                       : 0;
            x[k] = in ? (L2H ? ld_hint_i64(P.s_x + r, pol_stream) : __ldcs(P.s_x + r)) : 0;
            q[k] = in ? ld32(P.s_y + r) : 0;
        }
    };
    if (r0 >= r1) return;
    load(r0);
    for (int64_t t0 = r0; t0 < r1; t0 += stride) {
        int cd[ITEMS], cf[ITEMS], ch[ITEMS], cl[ITEMS], cq[ITEMS];
        long long cx[ITEMS];
        const unsigned cin = inmask;
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            cd[k] = d[k];
            cf[k] = f[k];
            ch[k] = h[k];
            cl[k] = l[k];
            cq[k] = q[k];
            cx[k] = x[k];
        }
        // the next tile's loads overlap this tile's work; a tile's dimension
        // reads (payload or membership word) are issued before them, so they
        // do not queue behind them (600M rows: semi-join 3.51 -> 2.73 ms,
        // inner join unchanged; the join-free kind has no such reads)
        bool ok[ITEMS];
        int32_t pay[ITEMS];
        if constexpr (JK == STAR_NONE) {
            load(t0 + stride);
            star_lookup<ITEMS, JK, L2H>(P, cd, cf, cl, cin, pol_keep, ok, pay);
        } else {
            star_lookup<ITEMS, JK, L2H>(P, cd, cf, cl, cin, pol_keep, ok, pay);
            load(t0 + stride);
        }
        star_fold<GLOBAL, ITEMS, NSUM, JK>(P, sm, ch, cq, cx, ok, pay);
    }
}

// The first predicate as x in [lo, hi] (negated for NE), clamped to int32:
// every comparison on an int32 column becomes two compares.
static inline void star_predicate(PipeSpec &P)
{
    const int64_t c = P.plo[0];
    int64_t a = INT64_MIN, b = INT64_MAX;
    int neg = 0;
    switch (P.pop[0]) {
    case QE_LT: b = c == INT64_MIN ? INT64_MIN : c - 1; if (c == INT64_MIN) a = 1; break;
    case QE_LE: b = c; break;
    case QE_GT: a = c == INT64_MAX ? INT64_MAX : c + 1; if (c == INT64_MAX) b = -1; break;
    case QE_GE: a = c; break;
    case QE_EQ: a = b = c; break;
    case QE_NE: a = b = c; neg = 1; break;
    default: a = P.plo[0]; b = P.phi[0]; break;
    }
    // empty ranges become [1, 0]; clamp the rest to int32
    if (a > b || a > INT32_MAX || b < INT32_MIN) {
        a = 1;
        b = 0;
    }
    P.p0_lo = static_cast<int32_t>(a < INT32_MIN ? INT32_MIN : a);
    P.p0_hi = static_cast<int32_t>(b > INT32_MAX ? INT32_MAX : b);
    P.p0_neg = neg;
    P.s_pred = static_cast<const int32_t *>(P.col[P.pslot[0]]);
    P.s_fk = P.has_join ? static_cast<const int32_t *>(P.col[P.fk_slot]) : nullptr;
    P.s_has_hi = P.hi_slot >= 0;
    P.s_hi = P.s_has_hi ? P.col[P.hi_slot] : nullptr;
    P.s_h8 = P.s_has_hi && P.type[P.hi_slot] == QE_I8;
    P.s_lo = P.lo_slot >= 0 ? P.col[P.lo_slot] : nullptr;
    P.s_l8 = P.lo_slot >= 0 && P.type[P.lo_slot] == QE_I8;
    P.s_x = static_cast<const long long *>(P.col[P.x_slot]);
    P.s_y = static_cast<const int32_t *>(P.col[P.y_slot]);
    P.s_hmin = static_cast<int32_t>(P.dk.hi_min);
    P.s_lmin = static_cast<int32_t>(P.dk.lo_min);
    P.s_hspan = static_cast<uint32_t>(P.dk.hi_span);
    P.s_lspan = static_cast<uint32_t>(P.dk.lo_span);
    P.s_ns = static_cast<uint32_t>(P.dk.nslots);
}

// The star kind of a pipeline (see k_pipeline_star), or -1 when the shape
// is not a star: one int32 predicate column, the aggregates [SUM(x*y),
// COUNT, MIN(x), MAX(x)] with x int64 and y int32, a direct array whose key
// parts stay within int32, and either an inner join through a dense table
// keyed (int8/int32 column, payload), or a key (optional int8/int32 column,
// int8/int32 column) with a semi- or anti-join through a dense key set or
// with no join.
static inline int star_kind(const PipeSpec &P, const TableCfg &T)
{
    auto narrow = [&](int slot) { return P.type[slot] == QE_I8 || P.type[slot] == QE_I32; };
    const bool common =
        (T.mode == TM_SMEM_DENSE || T.mode == TM_GLOBAL_DENSE) && P.npreds == 1 && P.type[P.pslot[0]] == QE_I32 &&
        P.ops.n == 4 && P.ops.op[0] == QE_SUM && P.src[0] == SRC_XY && P.ops.op[1] == QE_COUNT &&
        P.ops.op[2] == QE_MIN && P.src[2] == SRC_X && P.ops.op[3] == QE_MAX && P.src[3] == SRC_X &&
        P.type[P.x_slot] == QE_I64 && P.type[P.y_slot] == QE_I32 && P.dk.stride == 4 && P.dk.nslots < (1ull << 31) &&
        P.dk.hi_min >= INT32_MIN && P.dk.hi_min + static_cast<int64_t>(P.dk.hi_span) <= INT32_MAX &&
        P.dk.lo_min >= INT32_MIN && P.dk.lo_min + static_cast<int64_t>(P.dk.lo_span) <= INT32_MAX;
    if (!common) return -1;
    if (P.has_join && P.join_kind == QE_JOIN_INNER)
        return P.ht.layout == QE_HT_DENSE && P.lo_slot == QE_JOIN_PAYLOAD && P.hi_slot >= 0 && narrow(P.hi_slot)
                   ? STAR_INNER : -1;
    if (P.lo_slot < 0 || !narrow(P.lo_slot) || (P.hi_slot >= 0 && !narrow(P.hi_slot))) return -1;
    if (!P.has_join) return STAR_NONE;
    if (P.ht.layout != QE_HT_DENSE) return -1;
    return P.join_kind == QE_JOIN_SEMI ? STAR_SEMI : STAR_ANTI;
}


