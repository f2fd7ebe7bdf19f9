// qe_join_multi.cu -- many-to-many inner equi-join: the local join of
// Sec. 2.2 when build keys repeat.
//
// Build: a multimap from key to the run of its payloads.  Each key (a dense
// slot key - key_min, or an open-addressing slot) counts its build rows; an
// exclusive scan of the counts gives every key the start of its run in one
// payload array; a second pass places each build row at start + an atomic
// cursor, so the order inside a run is unspecified.
//   DENSE  start[range] (int64), cnt[range] (uint32)
//   OPEN   slots (key << 32 | count; INT32_MIN key = empty), start[slots],
//          cnt[slots]; load factor <= 0.5
// Probe: two passes over the probe positions, in segments of 32 x MM_ITEMS
// per warp: count every position's matches and total them per segment; scan
// the segment totals; look up again and write each position's run at its
// offset, so positions stay in ascending order.
#include <climits>

#include "qe_compact.cuh"

namespace {

constexpr int MM_ITEMS = 8;          // probe positions per lane and segment
constexpr int MM_SEG = 32 * MM_ITEMS;

struct MmView {
    int32_t layout;
    int32_t key_min;
    uint32_t range;                  // dense
    uint32_t mask;                   // open: slots - 1
    const unsigned long long *run;   // per slot: start of the run << 32 | its length
    const int32_t *vals;
    const unsigned long long *slots;
};

MmView mm_view(const qe_hash_table *ht)
{
    MmView v{};
    v.layout = ht->layout;
    v.key_min = ht->key_min;
    v.range = ht->layout == QE_HT_DENSE ? static_cast<uint32_t>(ht->slots) : 0;
    v.mask = ht->layout == QE_HT_OPEN ? static_cast<uint32_t>(ht->slots - 1) : 0;
    v.run = reinterpret_cast<const unsigned long long *>(ht->mstart);
    v.vals = ht->payload;
    v.slots = ht->open;
    return v;
}

// Slot of `key` in an open multimap, or -1.
__device__ __forceinline__ int64_t mm_open_find(const unsigned long long *slots, uint32_t mask, int32_t key)
{
    uint32_t i = dev_fmix32(static_cast<uint32_t>(key)) & mask;
    for (uint32_t probes = 0; probes <= mask; probes++) {
        const int32_t k = static_cast<int32_t>(__ldg(slots + i) >> 32);
        if (k == key) return i;
        if (k == HT_EMPTY_KEY) return -1;
        i = (i + 1) & mask;
    }
    return -1;
}

// The run of `key` (start << 32 | number of matches), 0 when it has none.
__device__ __forceinline__ unsigned long long mm_run(const MmView &v, int32_t key)
{
    int64_t s;
    if (v.layout == QE_HT_DENSE) {
        const uint32_t d = static_cast<uint32_t>(key) - static_cast<uint32_t>(v.key_min);
        if (d >= v.range) return 0;
        s = d;
    } else {
        s = mm_open_find(v.slots, v.mask, key);
        if (s < 0) return 0;
    }
    return __ldg(v.run + s);
}

// ---------------------------------------------------------------- build
__global__ void __launch_bounds__(256) k_mm_count_dense(const int32_t *keys, int64_t n, int32_t key_min, uint32_t range,
                                                        uint32_t *cnt, qe_dev_status *st)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) {
        const uint32_t s = static_cast<uint32_t>(__ldcs(keys + i)) - static_cast<uint32_t>(key_min);
        if (s >= range) {
            dev_report(st, QE_ERR_INVALID_ARG, 0);
            continue;
        }
        atomicAdd(cnt + s, 1u);
    }
}

__global__ void __launch_bounds__(256) k_mm_fill_dense(const int32_t *keys, const int32_t *pay, int64_t n,
                                                       int32_t key_min, uint32_t range, const int64_t *start,
                                                       uint32_t *cur, int32_t *vals)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) {
        const uint32_t s = static_cast<uint32_t>(__ldcs(keys + i)) - static_cast<uint32_t>(key_min);
        if (s >= range) continue;
        vals[start[s] + atomicAdd(cur + s, 1u)] = __ldcs(pay + i);
    }
}

// Insert or count: a new key takes an empty slot as (key, 1); a present key
// adds 1 to its slot's low half (counts stay below 2^31, so the key half is
// never touched).
__global__ void __launch_bounds__(256) k_mm_insert_open(const int32_t *keys, int64_t n, unsigned long long *slots,
                                                        uint32_t mask, qe_dev_status *st)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) {
        const int32_t k = __ldcs(keys + i);
        if (k == HT_EMPTY_KEY) {
            dev_report(st, QE_ERR_RESERVED_KEY, 0);
            continue;
        }
        const unsigned long long w = (static_cast<unsigned long long>(static_cast<uint32_t>(k)) << 32) | 1ull;
        uint32_t h = dev_fmix32(static_cast<uint32_t>(k)) & mask;
        bool done = false;
        for (uint32_t probes = 0; probes <= mask && !done; probes++) {
            unsigned long long cur = slots[h];
            if (cur == HT_EMPTY_SLOT) {
                cur = atomicCAS(slots + h, HT_EMPTY_SLOT, w);
                if (cur == HT_EMPTY_SLOT) {
                    done = true;
                    break;
                }
            }
            if (static_cast<int32_t>(cur >> 32) == k) {
                atomicAdd(reinterpret_cast<unsigned *>(slots + h), 1u);   // low half: the count
                done = true;
            } else {
                h = (h + 1) & mask;
            }
        }
        if (!done) dev_report(st, QE_ERR_CAPACITY, n);
    }
}

__global__ void __launch_bounds__(256) k_mm_slot_counts(const unsigned long long *slots, int64_t nslots, uint32_t *cnt)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < nslots; i += static_cast<int64_t>(gridDim.x) * 256) {
        const unsigned long long w = slots[i];
        cnt[i] = static_cast<int32_t>(w >> 32) == HT_EMPTY_KEY ? 0u : static_cast<uint32_t>(w);
    }
}

__global__ void __launch_bounds__(256) k_mm_fill_open(const int32_t *keys, const int32_t *pay, int64_t n,
                                                      const unsigned long long *slots, uint32_t mask,
                                                      const int64_t *start, uint32_t *cur, int32_t *vals)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) {
        const int32_t k = __ldcs(keys + i);
        if (k == HT_EMPTY_KEY) continue;
        const int64_t s = mm_open_find(slots, mask, k);
        if (s < 0) continue;                     // only after a reported capacity error
        vals[start[s] + atomicAdd(cur + s, 1u)] = __ldcs(pay + i);
    }
}

// After the fill: each slot's run as one word, start << 32 | length (both
// below 2^31), so that a probe reads one word per key.
__global__ void __launch_bounds__(256) k_mm_pack_runs(int64_t *start, const uint32_t *cnt, int64_t n)
{
    for (int64_t s = blockIdx.x * 256ll + threadIdx.x; s < n; s += static_cast<int64_t>(gridDim.x) * 256)
        start[s] = static_cast<int64_t>((static_cast<unsigned long long>(start[s]) << 32) | cnt[s]);
}

// ---------------------------------------------------------------- scans
// Exclusive scan of TP_SCAN_B int64 values per block into local offsets and
// block totals (the int64 form of k_tp_scan_local).
__global__ void __launch_bounds__(1024) k_mm_scan_local_i64(const int64_t *in, int64_t *loc, int64_t n, int64_t *bsum)
{
    __shared__ int64_t s_w[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * TP_SCAN_B + 4 * t;
    int64_t v[4], local = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        v[j] = base + j < n ? in[base + j] : 0;
        local += v[j];
    }
    const int64_t inc = warp_incl_scan(local);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int64_t w = s_w[lane];
        const int64_t wi = warp_incl_scan(w);
        s_w[lane] = wi - w;
        if (lane == 31) bsum[blockIdx.x] = wi;
    }
    __syncthreads();
    int64_t run = s_w[warp] + inc - local;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        if (base + j < n) loc[base + j] = run;
        run += v[j];
    }
}

// start[s] = top[b / TP_SCAN_B] + loc2[b] + loc1[s], b = s / TP_SCAN_B.
__global__ void __launch_bounds__(256) k_mm_materialize(const uint32_t *loc1, const int64_t *loc2, const int64_t *top,
                                                        int64_t n, int64_t *start)
{
    for (int64_t s = blockIdx.x * 256ll + threadIdx.x; s < n; s += static_cast<int64_t>(gridDim.x) * 256) {
        const int64_t b = s / TP_SCAN_B;
        start[s] = top[b / TP_SCAN_B] + loc2[b] + loc1[s];
    }
}

unsigned grid_of(qe_ctx *ctx, int64_t n)
{
    int64_t g = qe_ceil_div(n, 256);
    const int64_t cap = static_cast<int64_t>(ctx->num_sms) * 8;
    if (g > cap) g = cap;
    return static_cast<unsigned>(g < 1 ? 1 : g);
}

// Exclusive scan of n uint32 counts into int64 starts (three levels: counts
// in blocks of TP_SCAN_B, block totals in blocks of TP_SCAN_B, at most 4096
// of those); *total (device) receives the sum.
qe_status mm_scan(qe_ctx *ctx, const uint32_t *cnt, int64_t n, int64_t *start, int64_t *total, cudaStream_t s)
{
    const int64_t nb1 = qe_ceil_div(n, TP_SCAN_B), nb2 = qe_ceil_div(nb1, TP_SCAN_B);
    if (nb2 > 4096) return qe_fail(ctx, QE_ERR_INVALID_ARG, "multimap: too many keys");
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t b_loc1 = up(static_cast<size_t>(n) * 4), b_bs1 = up(static_cast<size_t>(nb1) * 8),
                 b_loc2 = up(static_cast<size_t>(nb1) * 8), b_bs2 = up(static_cast<size_t>(nb2 + 1) * 8);
    void *scratch = nullptr;
    qe_status st = qe_alloc(ctx, &scratch, b_loc1 + b_bs1 + b_loc2 + b_bs2, s);
    if (st != QE_OK) return st;
    unsigned char *p = static_cast<unsigned char *>(scratch);
    uint32_t *loc1 = reinterpret_cast<uint32_t *>(p);
    int64_t *bs1 = reinterpret_cast<int64_t *>(p + b_loc1);
    int64_t *loc2 = reinterpret_cast<int64_t *>(p + b_loc1 + b_bs1);
    int64_t *bs2 = reinterpret_cast<int64_t *>(p + b_loc1 + b_bs1 + b_loc2);
    k_tp_scan_local<<<static_cast<unsigned>(nb1), 1024, 0, s>>>(cnt, loc1, n, bs1);
    QE_LAUNCHED(ctx);
    k_mm_scan_local_i64<<<static_cast<unsigned>(nb2), 1024, 0, s>>>(bs1, loc2, nb1, bs2);
    QE_LAUNCHED(ctx);
    k_tp_scan_top<<<1, 1024, 0, s>>>(bs2, static_cast<int>(nb2), total, INT64_MAX, ctx->dstat);
    QE_LAUNCHED(ctx);
    k_mm_materialize<<<grid_of(ctx, n), 256, 0, s>>>(loc1, loc2, bs2, n, start);
    QE_LAUNCHED(ctx);
    const cudaError_t e = cudaGetLastError();
    qe_free(ctx, scratch, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "multimap scan");
    return QE_OK;
}

// ---------------------------------------------------------------- probe
// Matches of the segment's positions, totalled per segment (one warp each).
// Each position's run word is kept in runs[pos] for the write pass, which
// then reads it in order instead of repeating the random lookups.
__global__ void __launch_bounds__(256) k_mm_probe_count(MmView v, const int32_t *keys, const int32_t *sel, int64_t n,
                                                        int64_t nseg, int64_t *seg_tot, unsigned long long *runs)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * 8;
    for (int64_t seg = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); seg < nseg; seg += warps) {
        int64_t tot = 0;
#pragma unroll
        for (int k = 0; k < MM_ITEMS; k++) {
            const int64_t pos = seg * MM_SEG + k * 32 + lane;
            if (pos < n) {
                const int32_t row = sel ? __ldcs(sel + pos) : static_cast<int32_t>(pos);
                const unsigned long long w = mm_run(v, __ldg(keys + row));
                runs[pos] = w;
                tot += static_cast<uint32_t>(w);
            }
        }
        tot = warp_incl_scan(tot);
        if (lane == 31) seg_tot[seg] = tot;
    }
}

// Each position's run, written at its offset: segment start, then the
// matches of the segment's earlier positions (in position order).  The
// warp writes the runs of its 32 positions together, 32 consecutive outputs
// per step: output j of the step belongs to the first lane whose inclusive
// match count exceeds j (a binary search over the lanes' counts), so every
// store is a coalesced warp store whatever the run lengths.
__global__ void __launch_bounds__(256) k_mm_probe_write(MmView v, const int32_t *sel, int64_t n, int64_t nseg,
                                                        const unsigned long long *runs, const int64_t *loc,
                                                        const int64_t *bsum, int32_t *out_row, int32_t *out_pay,
                                                        int64_t capacity)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * 8;
    for (int64_t seg = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); seg < nseg; seg += warps) {
        int64_t o = bsum[seg / TP_SCAN_B] + loc[seg];
        if (o >= capacity) continue;
#pragma unroll 1
        for (int k = 0; k < MM_ITEMS; k++) {
            const int64_t pos = seg * MM_SEG + k * 32 + lane;
            int32_t row = 0;
            uint32_t c = 0;
            int64_t beg = 0;
            if (pos < n) {
                const unsigned long long w = __ldcs(runs + pos);
                c = static_cast<uint32_t>(w);
                beg = static_cast<int64_t>(w >> 32);
                row = sel ? __ldcs(sel + pos) : static_cast<int32_t>(pos);
            }
            const int64_t inc = warp_incl_scan(static_cast<int64_t>(c));
            const int64_t total = __shfl_sync(QE_FULL_MASK, inc, 31);
            for (int64_t base = 0; base < total; base += 32) {
                const int64_t j = base + lane;
                int owner = 0;   // lanes whose inclusive count is <= j (at most 31 for j < total)
#pragma unroll
                for (int b = 16; b >= 1; b >>= 1)
                    if (__shfl_sync(QE_FULL_MASK, inc, owner + b - 1) <= j) owner += b;
                const int64_t end = __shfl_sync(QE_FULL_MASK, inc, owner);
                const uint32_t cnt = __shfl_sync(QE_FULL_MASK, c, owner);
                const int32_t r = __shfl_sync(QE_FULL_MASK, row, owner);
                const int64_t b0 = __shfl_sync(QE_FULL_MASK, beg, owner);
                if (j < total && o + j < capacity) {
                    __stcs(out_row + o + j, r);
                    __stcs(out_pay + o + j, __ldg(v.vals + b0 + (j - (end - cnt))));
                }
            }
            o += total;
        }
    }
}

__global__ void __launch_bounds__(256) k_mm_fill_u64(unsigned long long *p, int64_t n, unsigned long long v)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) p[i] = v;
}

}  // namespace

extern "C" qe_status qe_join_build_multi(qe_ctx *ctx, const int32_t *keys, const int32_t *payload, int64_t nrows,
                                         const qe_build_opts *opts, qe_hash_table **out, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!out || nrows < 0 || nrows >= (int64_t(1) << 31) || (nrows > 0 && (!keys || !payload)) ||
        !qe_aligned(keys, 4) || !qe_aligned(payload, 4))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "build multi: bad argument");
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qe_build_opts o{};
    if (opts) o = *opts;
    if (o.layout < QE_HT_AUTO || o.layout > QE_HT_OPEN) return qe_fail(ctx, QE_ERR_INVALID_ARG, "build multi: bad layout");
    int32_t kmin = 0, kmax = -1;
    if (nrows > 0) {
        if (o.have_range) {
            kmin = o.key_min;
            kmax = o.key_max;
            if (kmin > kmax) return qe_fail(ctx, QE_ERR_INVALID_ARG, "build multi: empty key range");
        } else {
            int32_t mm[4];
            const qe_status st = join_key_range(ctx, keys, nullptr, nrows, mm, s);
            if (st != QE_OK) return st;
            kmin = mm[0];
            kmax = mm[1];
        }
    }
    const uint64_t range = nrows > 0 ? static_cast<uint64_t>(static_cast<int64_t>(kmax) - kmin + 1) : 1;
    int layout = o.layout;
    if (layout == QE_HT_AUTO)
        layout = (range <= static_cast<uint64_t>(4 * (nrows > 0 ? nrows : 1)) && range < (1ull << 31)) ? QE_HT_DENSE
                                                                                                      : QE_HT_OPEN;
    if (layout == QE_HT_DENSE && range >= (1ull << 31))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "build multi: key range too wide for a dense table");
    uint64_t nslots = range;
    if (layout == QE_HT_OPEN) {
        nslots = 64;
        while (nslots < static_cast<uint64_t>(2 * nrows)) nslots <<= 1;
        if (nslots > (1ull << 32)) return qe_fail(ctx, QE_ERR_INVALID_ARG, "build multi: too many keys");
    }
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t b_start = up(nslots * 8), b_cnt = up(nslots * 4), b_vals = up(static_cast<size_t>(nrows) * 4 + 4),
                 b_open = layout == QE_HT_OPEN ? up(nslots * 8) : 0, b_tot = 256;
    qe_hash_table *ht = new qe_hash_table();
    ht->layout = layout;
    ht->multi = 1;
    ht->key_min = kmin;
    ht->key_max = kmax;
    ht->nkeys = nrows;
    ht->slots = static_cast<int64_t>(nslots);
    ht->bytes = b_start + b_cnt + b_vals + b_open + b_tot;
    qe_status st = qe_alloc(ctx, &ht->mem, ht->bytes, s);
    if (st != QE_OK) {
        delete ht;
        return st;
    }
    unsigned char *p = static_cast<unsigned char *>(ht->mem);
    ht->mstart = reinterpret_cast<int64_t *>(p);
    ht->mcnt = reinterpret_cast<uint32_t *>(p + b_start);
    ht->payload = reinterpret_cast<int32_t *>(p + b_start + b_cnt);
    ht->open = layout == QE_HT_OPEN ? reinterpret_cast<unsigned long long *>(p + b_start + b_cnt + b_vals) : nullptr;
    int64_t *total = reinterpret_cast<int64_t *>(p + b_start + b_cnt + b_vals + b_open);
    const unsigned grid = grid_of(ctx, nrows);
    const uint32_t r32 = static_cast<uint32_t>(range), mask = static_cast<uint32_t>(nslots - 1);
    // rows in region order (dense: by key range; open: by slot) when the
    // table is far larger than L2
    const int log2s = qe_log2_ceil(nslots);
    int lp = region_plan_log2(ctx, ht->bytes, nrows, true);
    lp = lp < log2s ? lp : log2s;
    const int32_t *cols[2] = {keys, payload};
    void *scratch = nullptr;
    st = region_order(ctx, RegionPlan{layout == QE_HT_DENSE ? RP_DENSE : RP_HASH32, lp, log2s - lp, mask, kmin}, cols,
                      2, nrows, &scratch, s);
    if (st != QE_OK) {
        qe_free(ctx, ht->mem, s);
        delete ht;
        return st;
    }
    keys = cols[0];
    payload = cols[1];
    // 1. rows per key (dense slot, or open slot's low half copied out)
    cudaError_t e = cudaMemsetAsync(ht->mcnt, 0, nslots * 4, s);
    if (e == cudaSuccess) {
        ProfScope prof(ctx, "build", s);
        if (layout == QE_HT_DENSE) {
            if (nrows > 0) {
                k_mm_count_dense<<<grid, 256, 0, s>>>(keys, nrows, kmin, r32, ht->mcnt, ctx->dstat);
                QE_LAUNCHED(ctx);
            }
        } else {
            k_mm_fill_u64<<<grid_of(ctx, static_cast<int64_t>(nslots)), 256, 0, s>>>(
                ht->open, static_cast<int64_t>(nslots), HT_EMPTY_SLOT);
            QE_LAUNCHED(ctx);
            if (nrows > 0) {
                k_mm_insert_open<<<grid, 256, 0, s>>>(keys, nrows, ht->open, mask, ctx->dstat);
                QE_LAUNCHED(ctx);
            }
            k_mm_slot_counts<<<grid_of(ctx, static_cast<int64_t>(nslots)), 256, 0, s>>>(
                ht->open, static_cast<int64_t>(nslots), ht->mcnt);
            QE_LAUNCHED(ctx);
        }
        e = cudaGetLastError();
    }
    // 2. runs: start of every key's run; 3. rows into their runs (the counts
    // are rebuilt by the cursors)
    if (e == cudaSuccess) st = mm_scan(ctx, ht->mcnt, static_cast<int64_t>(nslots), ht->mstart, total, s);
    if (e == cudaSuccess && st == QE_OK) e = cudaMemsetAsync(ht->mcnt, 0, nslots * 4, s);
    if (e == cudaSuccess && st == QE_OK && nrows > 0) {
        ProfScope prof(ctx, "build", s);
        if (layout == QE_HT_DENSE)
            k_mm_fill_dense<<<grid, 256, 0, s>>>(keys, payload, nrows, kmin, r32, ht->mstart, ht->mcnt, ht->payload);
        else
            k_mm_fill_open<<<grid, 256, 0, s>>>(keys, payload, nrows, ht->open, mask, ht->mstart, ht->mcnt,
                                                ht->payload);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    // 4. each run as one word (start, length): with no rows the lengths are the zeros set above
    if (e == cudaSuccess && st == QE_OK) {
        k_mm_pack_runs<<<grid_of(ctx, static_cast<int64_t>(nslots)), 256, 0, s>>>(ht->mstart, ht->mcnt,
                                                                                   static_cast<int64_t>(nslots));
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    if (scratch) qe_free(ctx, scratch, s);
    if (e != cudaSuccess || st != QE_OK) {
        qe_free(ctx, ht->mem, s);
        delete ht;
        return e != cudaSuccess ? qe_cuda_fail(ctx, e, "build multi") : st;
    }
    *out = ht;
    return QE_OK;
}

extern "C" qe_status qe_join_probe_multi(qe_ctx *ctx, const qe_hash_table *ht, const int32_t *probe_keys,
                                         const int32_t *sel, int64_t n, int32_t *out_probe_row,
                                         int32_t *out_build_payload, int64_t capacity, int64_t *out_count,
                                         void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!ht || n < 0 || n >= (int64_t(1) << 31) || !out_count || capacity < 0 ||
        (capacity > 0 && (!out_probe_row || !out_build_payload)) || (n > 0 && !probe_keys))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "probe multi: bad argument");
    if (!ht->multi) return qe_fail(ctx, QE_ERR_INVALID_ARG, "probe multi: needs a table from qe_join_build_multi");
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        QE_CUDA(ctx, cudaMemsetAsync(out_count, 0, sizeof(int64_t), s));
        return QE_OK;
    }
    const MmView v = mm_view(ht);
    const int64_t nseg = qe_ceil_div(n, MM_SEG), nb = qe_ceil_div(nseg, TP_SCAN_B);
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t b_seg = up(static_cast<size_t>(nseg) * 8), b_bs = up(static_cast<size_t>(nb) * 8);
    void *scratch = nullptr;
    // segment totals and offsets, block sums, and one run word per position
    qe_status st = qe_alloc(ctx, &scratch, 2 * b_seg + b_bs + static_cast<size_t>(n) * 8, s);
    if (st != QE_OK) return st;
    unsigned char *p = static_cast<unsigned char *>(scratch);
    int64_t *seg_tot = reinterpret_cast<int64_t *>(p);
    int64_t *loc = reinterpret_cast<int64_t *>(p + b_seg);
    int64_t *bsum = reinterpret_cast<int64_t *>(p + 2 * b_seg);
    unsigned long long *runs = reinterpret_cast<unsigned long long *>(p + 2 * b_seg + b_bs);
    int64_t g = qe_ceil_div(nseg, 8);
    if (g > static_cast<int64_t>(ctx->num_sms) * 8) g = static_cast<int64_t>(ctx->num_sms) * 8;
    {
        ProfScope prof(ctx, "probe", s);
        k_mm_probe_count<<<static_cast<unsigned>(g), 256, 0, s>>>(v, probe_keys, sel, n, nseg, seg_tot, runs);
        QE_LAUNCHED(ctx);
        k_mm_scan_local_i64<<<static_cast<unsigned>(nb), 1024, 0, s>>>(seg_tot, loc, nseg, bsum);
        QE_LAUNCHED(ctx);
        k_tp_scan_top<<<1, 1024, 0, s>>>(bsum, static_cast<int>(nb), out_count, capacity, ctx->dstat);
        QE_LAUNCHED(ctx);
        k_mm_probe_write<<<static_cast<unsigned>(g), 256, 0, s>>>(v, sel, n, nseg, runs, loc, bsum, out_probe_row,
                                                                  out_build_payload, capacity);
        QE_LAUNCHED(ctx);
    }
    const cudaError_t e = cudaGetLastError();
    qe_free(ctx, scratch, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "probe multi");
    return QE_OK;
}
