// qe_join.cu -- hash-join build and probe (Sec. 2.2: the local join once
// both inputs are co-located; Sec. 7.2 on large build sides).
//
// Two table layouts, both library-owned:
//   DENSE  direct-mapped on key - key_min (a perfect hash for dense key
//          domains): payload[range] plus an occupancy bitmap used to detect
//          duplicates; when every slot is occupied the probe skips the bitmap.
//          A 20M-key dimension takes 80 MB of payload, which stays resident in
//          the 126 MB L2 while the fact columns stream through it.
//   OPEN   open addressing with linear probing over 8-byte slots
//          (key << 32 | payload), inserted with 64-bit CAS; INT32_MIN marks an
//          empty slot.  Load factor <= 0.5.
#include <climits>

#include "qe_compact.cuh"


HtView ht_view(const qe_hash_table *ht)
{
    HtView v{};
    v.layout = ht->layout;
    v.full = ht->full;
    v.key_min = ht->key_min;
    v.range = ht->layout == QE_HT_DENSE ? static_cast<uint32_t>(ht->slots) : 0;
    v.mask = ht->layout == QE_HT_OPEN ? static_cast<uint32_t>(ht->slots - 1) : 0;
    v.payload = ht->payload;
    v.bitmap = ht->bitmap;
    v.slots = ht->open;
    return v;
}

namespace {

// Min and max of the build keys and of the payloads: mm = {kmin, kmax, pmin,
// pmax}; without payloads (a key set) the payload half stays empty.
__global__ void __launch_bounds__(256) k_minmax(const int32_t *keys, const int32_t *pay, int64_t n, int32_t *mm)
{
    int32_t lo = INT_MAX, hi = INT_MIN, plo = INT_MAX, phi = INT_MIN;
    // four rows per thread and step, their loads in flight together
    constexpr int MR = 4;
    const int64_t step = static_cast<int64_t>(gridDim.x) * 256 * MR;
    for (int64_t i0 = blockIdx.x * 256ll * MR + threadIdx.x; i0 < n; i0 += step) {
        int32_t k[MR], p[MR];
#pragma unroll
        for (int j = 0; j < MR; j++) {
            const int64_t i = i0 + j * 256;
            k[j] = i < n ? __ldcs(keys + i) : INT_MAX;
            p[j] = i < n && pay ? __ldcs(pay + i) : INT_MAX;
        }
#pragma unroll
        for (int j = 0; j < MR; j++) {
            if (i0 + j * 256 >= n) continue;
            lo = min(lo, k[j]);
            hi = max(hi, k[j]);
            plo = min(plo, p[j]);
            phi = pay ? max(phi, p[j]) : phi;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(QE_FULL_MASK, lo, d));
        hi = max(hi, __shfl_xor_sync(QE_FULL_MASK, hi, d));
        plo = min(plo, __shfl_xor_sync(QE_FULL_MASK, plo, d));
        phi = max(phi, __shfl_xor_sync(QE_FULL_MASK, phi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mm, lo);
        atomicMax(mm + 1, hi);
        atomicMin(mm + 2, plo);
        atomicMax(mm + 3, phi);
    }
}

__global__ void k_minmax_init(int32_t *mm)
{
    mm[0] = INT_MAX;
    mm[1] = INT_MIN;
    mm[2] = INT_MAX;
    mm[3] = INT_MIN;
}

// payload == NULL: a key set (repeated keys are not an error).
// BD_ROWS rows per thread and step, so that their bitmap atomics (whose old
// value decides whether the payload is written) are in flight together.
constexpr int BD_ROWS = 4;

__global__ void __launch_bounds__(256) k_build_dense(const int32_t *keys, const int32_t *pay, int64_t n,
                                                     int32_t key_min, uint32_t range, int32_t *payload,
                                                     uint32_t *bitmap, qe_dev_status *st)
{
    const int64_t step = static_cast<int64_t>(gridDim.x) * 256 * BD_ROWS;
    for (int64_t i0 = blockIdx.x * 256ll * BD_ROWS + threadIdx.x; i0 < n; i0 += step) {
        uint32_t sl[BD_ROWS], old[BD_ROWS];
        int32_t v[BD_ROWS];
#pragma unroll
        for (int j = 0; j < BD_ROWS; j++) {
            const int64_t i = i0 + j * 256;
            sl[j] = i < n ? static_cast<uint32_t>(__ldcs(keys + i)) - static_cast<uint32_t>(key_min) : 0xffffffffu;
            v[j] = i < n && payload ? __ldcs(pay + i) : 0;
        }
#pragma unroll
        for (int j = 0; j < BD_ROWS; j++) {
            old[j] = 0;
            if (sl[j] < range) old[j] = atomicOr(bitmap + (sl[j] >> 5), 1u << (sl[j] & 31));
        }
#pragma unroll
        for (int j = 0; j < BD_ROWS; j++) {
            if (i0 + j * 256 >= n) continue;
            if (sl[j] >= range) {
                dev_report(st, QE_ERR_INVALID_ARG, 0);
                continue;
            }
            if (!payload) continue;
            if ((old[j] >> (sl[j] & 31)) & 1u) {
                dev_report(st, QE_ERR_DUPLICATE_KEY, 0);
                continue;
            }
            payload[sl[j]] = v[j];
        }
    }
}

__global__ void __launch_bounds__(256) k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) p[i] = v;
}

// pay == NULL: a key set (payload word 0, repeated keys are not an error).
__global__ void __launch_bounds__(256) k_build_open(const int32_t *keys, const int32_t *pay, int64_t n,
                                                    unsigned long long *slots, uint32_t mask, qe_dev_status *st)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) {
        const int32_t k = __ldcs(keys + i);
        if (k == HT_EMPTY_KEY) {
            dev_report(st, QE_ERR_RESERVED_KEY, 0);
            continue;
        }
        const unsigned long long w = (static_cast<unsigned long long>(static_cast<uint32_t>(k)) << 32) |
                                     (pay ? static_cast<uint32_t>(__ldcs(pay + i)) : 0u);
        uint32_t h = dev_fmix32(static_cast<uint32_t>(k)) & mask;
        bool done = false;
        for (uint32_t probes = 0; probes <= mask && !done; probes++) {
            unsigned long long old = atomicCAS(slots + h, HT_EMPTY_SLOT, w);
            if (old == HT_EMPTY_SLOT) {
                done = true;
            } else if (static_cast<int32_t>(old >> 32) == k) {
                if (pay) dev_report(st, QE_ERR_DUPLICATE_KEY, 0);
                done = true;
            } else {
                h = (h + 1) & mask;
            }
        }
        if (!done) dev_report(st, QE_ERR_CAPACITY, n);
    }
}

unsigned grid_for(qe_ctx *ctx, int64_t n)
{
    int64_t g = qe_ceil_div(n, 256);
    int64_t cap = static_cast<int64_t>(ctx->num_sms) * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return static_cast<unsigned>(g);
}

// Probe as a stable compaction: position i probes row sel[i] (or i).
constexpr int PROBE_ITEMS = 8;
constexpr int64_t PROBE_TWO_PASS_ROWS = int64_t(1) << 22;   // from here on: the two-pass compaction

struct ProbeOp {
    HtView ht;
    const int32_t *keys;
    const int32_t *sel;
    int32_t *out_row;
    int32_t *out_pay;

    struct Slot {
        int32_t row[PROBE_ITEMS];
        int32_t pay[PROBE_ITEMS];
    };
    // the probe rows (selection vector entries), loaded a tile ahead
    struct Pre {
        int32_t row[PROBE_ITEMS];
    };

    template <int ITEMS>
    __device__ __forceinline__ void load(int64_t pos0, const bool (&in)[ITEMS], Pre &p) const
    {
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            int64_t i = pos0 + 32 * k;
            p.row[k] = in[k] ? (sel ? __ldcs(sel + i) : static_cast<int32_t>(i)) : 0;
        }
    }

    template <int ITEMS>
    __device__ __forceinline__ void eval(int64_t, bool (&ok)[ITEMS], const Pre &pre, Slot &s) const
    {
        int32_t key[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            s.row[k] = pre.row[k];
            key[k] = ok[k] ? __ldg(keys + s.row[k]) : 0;
        }
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            int32_t p = 0;
            if (ok[k]) ok[k] = ht_lookup(ht, key[k], p);
            s.pay[k] = p;
        }
    }

    __device__ __forceinline__ void emit(int64_t o, int64_t, int k, const Slot &s) const
    {
        __stcs(out_row + o, s.row[k]);
        __stcs(out_pay + o, s.pay[k]);
    }
    // two-pass probe: the payload word a survivor keeps between the passes,
    // and a survivor restored from its row and that word
    static constexpr bool kPay = true;
    __device__ __forceinline__ int32_t word(int k, const Slot &s) const { return s.pay[k]; }
    template <int ITEMS>
    __device__ __forceinline__ void restore(const Pre &pre, const int32_t (&w)[ITEMS], Slot &s) const
    {
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            s.row[k] = pre.row[k];
            s.pay[k] = w[k];
        }
    }
};

// Semi- / anti-join as a stable compaction: position i keeps row sel[i] (or
// i) when its key's membership differs from `anti`.
struct SemiOp {
    HtView ht;
    const int32_t *keys;
    const int32_t *sel;
    int32_t *out_row;
    int32_t anti;

    struct Slot {
        int32_t row[PROBE_ITEMS];
    };
    struct Pre {
        int32_t row[PROBE_ITEMS];
    };

    template <int ITEMS>
    __device__ __forceinline__ void load(int64_t pos0, const bool (&in)[ITEMS], Pre &p) const
    {
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            int64_t i = pos0 + 32 * k;
            p.row[k] = in[k] ? (sel ? __ldcs(sel + i) : static_cast<int32_t>(i)) : 0;
        }
    }

    template <int ITEMS>
    __device__ __forceinline__ void eval(int64_t, bool (&ok)[ITEMS], const Pre &pre, Slot &s) const
    {
        int32_t key[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            s.row[k] = pre.row[k];
            key[k] = ok[k] ? __ldg(keys + s.row[k]) : 0;
        }
#pragma unroll
        for (int k = 0; k < ITEMS; k++)
            if (ok[k]) ok[k] = ht_contains(ht, key[k]) != static_cast<bool>(anti);
    }

    __device__ __forceinline__ void emit(int64_t o, int64_t, int k, const Slot &s) const
    {
        __stcs(out_row + o, s.row[k]);
    }
    // two-pass: survivors keep no payload; a survivor is its row
    static constexpr bool kPay = false;
    __device__ __forceinline__ int32_t word(int, const Slot &) const { return 0; }
    template <int ITEMS>
    __device__ __forceinline__ void restore(const Pre &pre, const int32_t (&)[ITEMS], Slot &s) const
    {
#pragma unroll
        for (int k = 0; k < ITEMS; k++) s.row[k] = pre.row[k];
    }
};

// ---------------------------------------------------------------- pair keys
// A pair of int32 key columns packed as (uint32)hi << 32 | (uint32)lo; the
// packed (INT32_MIN, INT32_MIN) is the empty slot (HT_EMPTY_SLOT).  Open
// addressing over 16-byte slots {packed key, payload, unused}: a probe that
// finds its key has the payload in the same DRAM sector.
__device__ __forceinline__ unsigned long long pair_key(int32_t hi, int32_t lo)
{
    return (static_cast<unsigned long long>(static_cast<uint32_t>(hi)) << 32) | static_cast<uint32_t>(lo);
}

__global__ void __launch_bounds__(256) k_build_pair(const int32_t *khi, const int32_t *klo, const int32_t *pay,
                                                    int64_t n, unsigned long long *slots, uint32_t mask,
                                                    qe_dev_status *st)
{
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) {
        const unsigned long long k = pair_key(__ldcs(khi + i), __ldcs(klo + i));
        if (k == HT_EMPTY_SLOT) {
            dev_report(st, QE_ERR_RESERVED_KEY, 0);
            continue;
        }
        uint32_t h = static_cast<uint32_t>(dev_fmix64(k)) & mask;
        bool done = false;
        for (uint32_t probes = 0; probes <= mask && !done; probes++) {
            const unsigned long long old = atomicCAS(slots + 2 * static_cast<uint64_t>(h), HT_EMPTY_SLOT, k);
            if (old == HT_EMPTY_SLOT) {
                reinterpret_cast<int32_t *>(slots + 2 * static_cast<uint64_t>(h) + 1)[0] = __ldcs(pay + i);
                done = true;
            } else if (old == k) {
                dev_report(st, QE_ERR_DUPLICATE_KEY, 0);
                done = true;
            } else {
                h = (h + 1) & mask;
            }
        }
        if (!done) dev_report(st, QE_ERR_CAPACITY, n);
    }
}

struct PairView {
    const unsigned long long *slots;   // 2 words per slot: key, payload (low half)
    uint32_t mask;
};

__device__ __forceinline__ bool pair_lookup(const PairView &v, unsigned long long k, int32_t &pay)
{
    uint32_t h = static_cast<uint32_t>(dev_fmix64(k)) & v.mask;
    for (uint32_t probes = 0; probes <= v.mask; probes++) {
        const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2 *>(v.slots) + h);
        if (w.x == k) {
            pay = static_cast<int32_t>(static_cast<uint32_t>(w.y));
            return true;
        }
        if (w.x == HT_EMPTY_SLOT) return false;
        h = (h + 1) & v.mask;
    }
    return false;
}

// Pair-key probe as a stable compaction: position i probes row sel[i] (or i).
struct PairProbeOp {
    PairView ht;
    const int32_t *khi, *klo;
    const int32_t *sel;
    int32_t *out_row;
    int32_t *out_pay;

    struct Slot {
        int32_t row[PROBE_ITEMS];
        int32_t pay[PROBE_ITEMS];
    };
    struct Pre {
        int32_t row[PROBE_ITEMS];
    };

    template <int ITEMS>
    __device__ __forceinline__ void load(int64_t pos0, const bool (&in)[ITEMS], Pre &p) const
    {
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            int64_t i = pos0 + 32 * k;
            p.row[k] = in[k] ? (sel ? __ldcs(sel + i) : static_cast<int32_t>(i)) : 0;
        }
    }

    template <int ITEMS>
    __device__ __forceinline__ void eval(int64_t, bool (&ok)[ITEMS], const Pre &pre, Slot &s) const
    {
        unsigned long long key[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            s.row[k] = pre.row[k];
            key[k] = ok[k] ? pair_key(__ldg(khi + s.row[k]), __ldg(klo + s.row[k])) : 0;
        }
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            int32_t p = 0;
            if (ok[k]) ok[k] = key[k] != HT_EMPTY_SLOT && pair_lookup(ht, key[k], p);
            s.pay[k] = p;
        }
    }

    __device__ __forceinline__ void emit(int64_t o, int64_t, int k, const Slot &s) const
    {
        __stcs(out_row + o, s.row[k]);
        __stcs(out_pay + o, s.pay[k]);
    }
    // two-pass probe: the payload word a survivor keeps between the passes,
    // and a survivor restored from its row and that word
    static constexpr bool kPay = true;
    __device__ __forceinline__ int32_t word(int k, const Slot &s) const { return s.pay[k]; }
    template <int ITEMS>
    __device__ __forceinline__ void restore(const Pre &pre, const int32_t (&w)[ITEMS], Slot &s) const
    {
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            s.row[k] = pre.row[k];
            s.pay[k] = w[k];
        }
    }
};

}  // namespace

qe_status join_key_range(qe_ctx *ctx, const int32_t *keys, const int32_t *pay, int64_t nrows, int32_t host[4],
                         cudaStream_t s)
{
    void *mm = nullptr;
    qe_status st = qe_alloc(ctx, &mm, 16, s);
    if (st != QE_OK) return st;
    k_minmax_init<<<1, 1, 0, s>>>(static_cast<int32_t *>(mm));
    QE_LAUNCHED(ctx);
    k_minmax<<<grid_for(ctx, nrows), 256, 0, s>>>(keys, pay, nrows, static_cast<int32_t *>(mm));
    QE_LAUNCHED(ctx);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, mm, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    qe_free(ctx, mm, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "build: key range");
    return QE_OK;
}

qe_status join_build_impl(qe_ctx *ctx, const int32_t *keys, const int32_t *payload, int64_t nrows,
                          const qe_build_opts *opts, bool key_set, qe_hash_table **out, cudaStream_t s)
{
    if (key_set) payload = nullptr;   // the build kernels read no payloads for a key set
    qe_build_opts o{};
    if (opts) o = *opts;
    if (o.layout < QE_HT_AUTO || o.layout > QE_HT_OPEN) return qe_fail(ctx, QE_ERR_INVALID_ARG, "build: bad layout");
    int32_t kmin = 0, kmax = -1;
    int32_t have_pay = 0, pay_min = 0, pay_max = -1;
    if (nrows > 0) {
        if (o.have_range) {
            kmin = o.key_min;
            kmax = o.key_max;
            if (kmin > kmax) return qe_fail(ctx, QE_ERR_INVALID_ARG, "build: empty key range");
        } else {
            int32_t host[4];
            const qe_status st = join_key_range(ctx, keys, payload, nrows, host, s);
            if (st != QE_OK) return st;
            kmin = host[0];
            kmax = host[1];
            have_pay = key_set ? 0 : 1;
            pay_min = host[2];
            pay_max = host[3];
        }
    }
    const uint64_t range = nrows > 0 ? static_cast<uint64_t>(static_cast<int64_t>(kmax) - kmin + 1) : 1;
    int layout = o.layout;
    if (layout == QE_HT_AUTO)
        layout = (range <= static_cast<uint64_t>(4 * (nrows > 0 ? nrows : 1)) && range < (1ull << 31)) ? QE_HT_DENSE
                                                                                                      : QE_HT_OPEN;
    if (layout == QE_HT_DENSE && range >= (1ull << 31))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "build: key range too wide for a dense table");
    qe_hash_table *ht = new qe_hash_table();
    ht->layout = layout;
    ht->key_min = kmin;
    ht->key_max = kmax;
    ht->have_pay = have_pay;
    ht->pay_min = pay_min;
    ht->pay_max = pay_max;
    ht->nkeys = nrows;
    ht->set = key_set ? 1 : 0;
    qe_status st;
    if (layout == QE_HT_DENSE) {
        ht->slots = static_cast<int64_t>(range);
        const size_t pay_bytes = key_set ? 0 : ((range * 4 + 255) / 256) * 256;
        const size_t bm_bytes = ((range + 31) / 32) * 4;
        ht->bytes = pay_bytes + bm_bytes;
        st = qe_alloc(ctx, &ht->mem, ht->bytes, s);
        if (st != QE_OK) {
            delete ht;
            return st;
        }
        ht->payload = key_set ? nullptr : static_cast<int32_t *>(ht->mem);
        ht->bitmap = reinterpret_cast<uint32_t *>(static_cast<char *>(ht->mem) + pay_bytes);
        // a key set may repeat keys, so its row count says nothing about occupancy
        ht->full = !key_set && static_cast<uint64_t>(nrows) == range ? 1 : 0;
        cudaError_t e = cudaMemsetAsync(ht->bitmap, 0, bm_bytes, s);
        if (e == cudaSuccess && nrows > 0) {
            ProfScope prof(ctx, "build", s);
            k_build_dense<<<grid_for(ctx, nrows), 256, 0, s>>>(keys, payload, nrows, kmin,
                                                               static_cast<uint32_t>(range), ht->payload,
                                                               ht->bitmap, ctx->dstat);
            QE_LAUNCHED(ctx);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            qe_free(ctx, ht->mem, s);
            delete ht;
            return qe_cuda_fail(ctx, e, "build: dense");
        }
    } else {
        uint64_t slots = 64;
        while (slots < static_cast<uint64_t>(2 * nrows)) slots <<= 1;
        if (slots > (1ull << 32)) return qe_fail(ctx, QE_ERR_INVALID_ARG, "build: too many keys");
        ht->slots = static_cast<int64_t>(slots);
        ht->bytes = slots * 8;
        st = qe_alloc(ctx, &ht->mem, ht->bytes, s);
        if (st != QE_OK) {
            delete ht;
            return st;
        }
        ht->open = static_cast<unsigned long long *>(ht->mem);
        // rows in region order when the table is far larger than L2, only
        // when tuned so: on GB300 it measured slower for this table (20M /
        // 50M keys: 0.78 -> 0.86 ms and 2.08 -> 2.50 ms)
        const int log2s = qe_log2_ceil(slots);
        int lp = region_plan_log2(ctx, ht->bytes, nrows, false);
        lp = lp < log2s - 4 ? lp : (log2s > 5 ? log2s - 4 : 0);   // regions of >= 16 slots
        const RegionPlan plan{RP_HASH32, lp, log2s - lp, static_cast<uint32_t>(slots - 1), 0};
        const int32_t *cols[2] = {keys, payload};
        void *scratch = nullptr;
        const uint32_t *counts = nullptr;
        st = region_order(ctx, plan, cols, payload ? 2 : 1, nrows, &scratch, s, &counts);
        if (st == QE_OK && scratch)
            st = region_fill_insert(ctx, false, cols, payload != nullptr, nrows, ht->open, slots, plan, counts, s);
        if (st != QE_OK) {
            if (scratch) qe_free(ctx, scratch, s);
            qe_free(ctx, ht->mem, s);
            delete ht;
            return st;
        }
        cudaError_t e = cudaSuccess;
        if (!scratch) {
            k_fill_u64<<<grid_for(ctx, static_cast<int64_t>(slots)), 256, 0, s>>>(
                ht->open, static_cast<int64_t>(slots), HT_EMPTY_SLOT);
            QE_LAUNCHED(ctx);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && nrows > 0 && !scratch) {
            ProfScope prof(ctx, "build", s);
            k_build_open<<<grid_for(ctx, nrows), 256, 0, s>>>(cols[0], payload ? cols[1] : nullptr, nrows, ht->open,
                                                              static_cast<uint32_t>(slots - 1), ctx->dstat);
            QE_LAUNCHED(ctx);
            e = cudaGetLastError();
        }
        if (scratch) qe_free(ctx, scratch, s);
        if (e != cudaSuccess) {
            qe_free(ctx, ht->mem, s);
            delete ht;
            return qe_cuda_fail(ctx, e, "build: open");
        }
    }
    *out = ht;
    return QE_OK;
}

extern "C" qe_status qe_join_build(qe_ctx *ctx, const int32_t *keys, const int32_t *payload, int64_t nrows,
                                   const qe_build_opts *opts, qe_hash_table **out, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!out || nrows < 0 || nrows >= (int64_t(1) << 31) || (nrows > 0 && (!keys || !payload)) ||
        !qe_aligned(keys, 4) || !qe_aligned(payload, 4))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "build: bad argument");
    cudaSetDevice(ctx->device);
    return join_build_impl(ctx, keys, payload, nrows, opts, false, out, static_cast<cudaStream_t>(stream));
}

extern "C" qe_status qe_join_build_pair(qe_ctx *ctx, const int32_t *key_hi, const int32_t *key_lo,
                                        const int32_t *payload, int64_t nrows, qe_hash_table **out, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!out || nrows < 0 || nrows >= (int64_t(1) << 31) || (nrows > 0 && (!key_hi || !key_lo || !payload)) ||
        !qe_aligned(key_hi, 4) || !qe_aligned(key_lo, 4) || !qe_aligned(payload, 4))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "build pair: bad argument");
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t slots = 64;
    while (slots < static_cast<uint64_t>(2 * nrows)) slots <<= 1;
    qe_hash_table *ht = new qe_hash_table();
    ht->layout = QE_HT_OPEN;
    ht->pair = 1;
    ht->nkeys = nrows;
    ht->slots = static_cast<int64_t>(slots);
    ht->bytes = slots * 16;
    qe_status st = qe_alloc(ctx, &ht->mem, ht->bytes, s);
    if (st != QE_OK) {
        delete ht;
        return st;
    }
    ht->open = static_cast<unsigned long long *>(ht->mem);
    // rows in region order when the table is far larger than L2 (on by
    // default: 80M pairs into a 4 GB table, 6.5 -> 5.1 ms on GB300)
    const int log2s = qe_log2_ceil(slots);
    int lp = region_plan_log2(ctx, ht->bytes, nrows, true);
    lp = lp < log2s - 4 ? lp : (log2s > 5 ? log2s - 4 : 0);   // regions of >= 16 slots
    const RegionPlan plan{RP_PAIR64, lp, log2s - lp, static_cast<uint32_t>(slots - 1), 0};
    const int32_t *cols[3] = {key_hi, key_lo, payload};
    void *scratch = nullptr;
    const uint32_t *counts = nullptr;
    st = region_order(ctx, plan, cols, 3, nrows, &scratch, s, &counts);
    if (st == QE_OK && scratch) st = region_fill_insert(ctx, true, cols, true, nrows, ht->open, slots, plan, counts, s);
    if (st != QE_OK) {
        if (scratch) qe_free(ctx, scratch, s);
        qe_free(ctx, ht->mem, s);
        delete ht;
        return st;
    }
    cudaError_t e = cudaSuccess;
    if (!scratch) {
        // every word to the empty marker: the key words mark empty slots, the
        // payload words are written before any probe reads them
        const int64_t words = static_cast<int64_t>(2 * slots);
        k_fill_u64<<<grid_for(ctx, words), 256, 0, s>>>(ht->open, words, HT_EMPTY_SLOT);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && nrows > 0 && !scratch) {
        ProfScope prof(ctx, "build", s);
        k_build_pair<<<grid_for(ctx, nrows), 256, 0, s>>>(cols[0], cols[1], cols[2], nrows, ht->open,
                                                          static_cast<uint32_t>(slots - 1), ctx->dstat);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    if (scratch) qe_free(ctx, scratch, s);
    if (e != cudaSuccess) {
        qe_free(ctx, ht->mem, s);
        delete ht;
        return qe_cuda_fail(ctx, e, "build pair");
    }
    *out = ht;
    return QE_OK;
}

extern "C" qe_status qe_join_probe_pair(qe_ctx *ctx, const qe_hash_table *ht, const int32_t *probe_hi,
                                        const int32_t *probe_lo, const int32_t *sel, int64_t n, int32_t *out_probe_row,
                                        int32_t *out_build_payload, int64_t capacity, int64_t *out_count, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!ht || n < 0 || n >= (int64_t(1) << 31) || !out_count || capacity < 0 ||
        (capacity > 0 && (!out_probe_row || !out_build_payload)) || (n > 0 && (!probe_hi || !probe_lo)))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "probe pair: bad argument");
    if (!ht->pair) return qe_fail(ctx, QE_ERR_INVALID_ARG, "probe pair: needs a table from qe_join_build_pair");
    cudaSetDevice(ctx->device);
    PairProbeOp op{};
    op.ht.slots = ht->open;
    op.ht.mask = static_cast<uint32_t>(ht->slots - 1);
    op.khi = probe_hi;
    op.klo = probe_lo;
    op.sel = sel;
    op.out_row = out_probe_row;
    op.out_pay = out_build_payload;
    if (n >= PROBE_TWO_PASS_ROWS)
        return launch_two_pass<PROBE_ITEMS>(ctx, "probe", n, capacity, out_count, op, static_cast<cudaStream_t>(stream));
    return launch_compact<PROBE_ITEMS>(ctx, "probe", n, capacity, out_count, op, static_cast<cudaStream_t>(stream));
}

extern "C" qe_status qe_join_build_set(qe_ctx *ctx, const int32_t *keys, int64_t nrows, const qe_build_opts *opts,
                                       qe_hash_table **out, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!out || nrows < 0 || nrows >= (int64_t(1) << 31) || (nrows > 0 && !keys) || !qe_aligned(keys, 4))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "build set: bad argument");
    cudaSetDevice(ctx->device);
    return join_build_impl(ctx, keys, nullptr, nrows, opts, true, out, static_cast<cudaStream_t>(stream));
}

extern "C" qe_status qe_join_semi(qe_ctx *ctx, const qe_hash_table *ht, const int32_t *probe_keys,
                                  const int32_t *sel, int64_t n, int anti, int32_t *out_rows, int64_t capacity,
                                  int64_t *out_count, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!ht || n < 0 || n >= (int64_t(1) << 31) || !out_count || capacity < 0 || (capacity > 0 && !out_rows) ||
        (n > 0 && !probe_keys) || (anti != 0 && anti != 1))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "semi-join: bad argument");
    if (ht->multi || ht->pair)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "semi-join: takes a key set or a unique-key table");
    cudaSetDevice(ctx->device);
    SemiOp op{};
    op.ht = ht_view(ht);
    op.keys = probe_keys;
    op.sel = sel;
    op.out_row = out_rows;
    op.anti = anti;
    const char *name = anti ? "anti_join" : "semi_join";
    if (n >= PROBE_TWO_PASS_ROWS)
        return launch_two_pass<PROBE_ITEMS>(ctx, name, n, capacity, out_count, op, static_cast<cudaStream_t>(stream));
    return launch_compact<PROBE_ITEMS>(ctx, name, n, capacity, out_count, op, static_cast<cudaStream_t>(stream));
}

extern "C" qe_status qe_join_probe(qe_ctx *ctx, const qe_hash_table *ht, const int32_t *probe_keys,
                                   const int32_t *sel, int64_t n, int32_t *out_probe_row, int32_t *out_build_payload,
                                   int64_t capacity, int64_t *out_count, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    if (!ht || n < 0 || n >= (int64_t(1) << 31) || !out_count || capacity < 0 ||
        (capacity > 0 && (!out_probe_row || !out_build_payload)) || (n > 0 && !probe_keys))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "probe: bad argument");
    if (ht->set) return qe_fail(ctx, QE_ERR_INVALID_ARG, "probe: a key set has no payloads (use qe_join_semi)");
    if (ht->multi) return qe_fail(ctx, QE_ERR_INVALID_ARG, "probe: a multimap needs qe_join_probe_multi");
    if (ht->pair) return qe_fail(ctx, QE_ERR_INVALID_ARG, "probe: a pair-key table needs qe_join_probe_pair");
    cudaSetDevice(ctx->device);
    ProbeOp op{};
    op.ht = ht_view(ht);
    op.keys = probe_keys;
    op.sel = sel;
    op.out_row = out_probe_row;
    op.out_pay = out_build_payload;
    if (n >= PROBE_TWO_PASS_ROWS)
        return launch_two_pass<PROBE_ITEMS>(ctx, "probe", n, capacity, out_count, op, static_cast<cudaStream_t>(stream));
    return launch_compact<PROBE_ITEMS>(ctx, "probe", n, capacity, out_count, op, static_cast<cudaStream_t>(stream));
}

extern "C" qe_status qe_join_info(const qe_hash_table *ht, qe_ht_info *info)
{
    if (!ht || !info) return QE_ERR_INVALID_ARG;
    info->layout = ht->layout;
    info->full = ht->full;
    info->nkeys = ht->nkeys;
    info->slots = ht->slots;
    info->bytes = static_cast<int64_t>(ht->bytes);
    info->key_min = ht->key_min;
    info->key_max = ht->key_max;
    info->have_payload_range = ht->have_pay;
    info->payload_min = ht->pay_min;
    info->payload_max = ht->pay_max;
    info->key_set = ht->pair ? 3 : ht->multi ? 2 : ht->set;
    return QE_OK;
}

extern "C" qe_status qe_join_destroy(qe_ctx *ctx, qe_hash_table *ht, void *stream)
{
    if (!ctx || !ht) return QE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    qe_free(ctx, ht->mem, static_cast<cudaStream_t>(stream));
    delete ht;
    return QE_OK;
}
