// qe_internal.cuh -- shared host and device pieces of libqe (sm_103a).
//
// Host: the context (allocation under an HBM budget, the device-side error
// word, launch geometry).  Device: status reporting, the partition hash, the
// join-table hash, warp scans, the decoupled look-back used by the stable
// compaction kernels, and the hash group-table primitives.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "qe.h"

// ------------------------------------------------------------------ host

struct qe_dev_status {
    int32_t code;        // first qe_status recorded by a kernel (0 = none)
    int32_t pad;
    int64_t required;    // size the failing output needed (max over reports)
};

struct qe_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;              // 0 = unlimited
    size_t in_use = 0;
    int fail_after = 0;             // fault injection: n-th allocation fails
    int64_t spin_limit = 1 << 22;   // bounded device waits (iterations)
    size_t smem_optin = 0;          // max dynamic shared memory per block
    qe_dev_status *dstat = nullptr; // device
    qe_dev_status *hstat = nullptr; // pinned host mirror
    std::string last_error;
    std::mutex mu;
    std::unordered_map<void *, size_t> live;
    std::atomic<int64_t> launches{0};
    int tune_star_items = 0;        // 0: default
    int tune_force_generic = 0;
    int tune_part_general = 0;      // partition: skip the write-combining scatter
    int tune_part_span = 0;         // two-pass partition: first-pass ranges per second-pass item (0 = 8)
    int tune_gb_partition = 0;      // large HBM group tables: 0 auto, 1 never partition, 2 always
    int tune_gb_part_log2p = 0;     // parts of the partitioned group-by (log2; 0 = planned)
    int tune_gb_part_log2q = -1;    // sub-parts per part (log2; -1 = planned)
    int tune_gb_fold2 = 0;          // partitioned fold: two 512-thread blocks per SM
    int tune_l2_hint = 0;           // star pipeline: L2 policies on fact loads and payload lookups
    int tune_join_partition = 0;    // join builds into large tables: 0 auto, 1 never region-order, 2 always
    int tune_join_part_log2 = 0;    // regions of a region-ordered build (log2; 0 = planned)
    bool profiling = false;
    std::mutex prof_mu;
    std::map<std::string, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> prof;
};

// Count one kernel launch of the context.
#define QE_LAUNCHED(ctx) ((ctx)->launches.fetch_add(1, std::memory_order_relaxed))

// Brackets the launches inside its scope with profiling events when the
// context has profiling enabled.
struct ProfScope {
    qe_ctx *ctx;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    const char *name;
    ProfScope(qe_ctx *c, const char *n, cudaStream_t st) : ctx(c), s(st), name(n)
    {
        if (!ctx->profiling) return;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            cudaGetLastError();
            a = b = nullptr;
            return;
        }
        cudaEventRecord(a, s);
    }
    ~ProfScope()
    {
        if (!a) return;
        cudaEventRecord(b, s);
        std::lock_guard<std::mutex> g(ctx->prof_mu);
        ctx->prof[name].push_back({a, b});
    }
};

qe_status qe_fail(qe_ctx *ctx, qe_status st, const std::string &msg);
qe_status qe_cuda_fail(qe_ctx *ctx, cudaError_t e, const char *where);
qe_status qe_alloc(qe_ctx *ctx, void **p, size_t bytes, cudaStream_t s);
void qe_free(qe_ctx *ctx, void *p, cudaStream_t s);

// Region-ordered build input (qe_join_part.cu).  The region of a row is the
// top log2p bits of its slot: fmix32(key) & mask (RP_HASH32, the open
// table), (uint32)fmix64(hi << 32 | lo) & mask (RP_PAIR64, the pair-key
// table), or key - kmin (RP_DENSE, a dense table, clamped to the last
// region); region = slot >> shift.
enum : int { RP_HASH32 = 0, RP_PAIR64 = 1, RP_DENSE = 2 };
struct RegionPlan {
    int kind;
    int log2p;        // 1 .. 8
    int shift;
    uint32_t mask;
    int32_t kmin;
};
// log2 of the regions for a build of nrows into a table of table_bytes, or 0
// for a build in input order (the knobs "join_partition", "join_part_log2").
// With the knob at 0 (automatic) only builds with by_default set are
// reordered: the multimap build gains (80M rows: 6.2 -> 3.0 ms), the
// open-addressing and pair-key builds measured slower reordered.
int region_plan_log2(const qe_ctx *ctx, uint64_t table_bytes, int64_t nrows, bool by_default);
// Rows of ncols int32 columns (column 0 the key; columns 0 and 1 the key pair
// of RP_PAIR64) reordered region by region into *scratch, allocated here
// from the context (the caller frees it with qe_free once the build kernels
// are enqueued); on return cols[c] points at the reordered column c.  The
// order inside a region is unspecified.  plan.log2p == 0: nothing is done,
// *scratch = NULL.
qe_status region_order(qe_ctx *ctx, const RegionPlan &plan, const int32_t **cols, int ncols, int64_t n,
                       void **scratch, cudaStream_t s, const uint32_t **counts = nullptr);
// Fills and builds an open-addressing table of nslots slots (8-byte {key,
// payload} words, or pair = 16-byte {packed key pair, payload} slots) from
// rows that region_order reordered with `plan` (counts: its rows per
// region); plan.shift >= 4.  Replaces the fill and the insert kernel of a
// build in input order; reports the same errors.
qe_status region_fill_insert(qe_ctx *ctx, bool pair, const int32_t *const *cols, bool has_pay, int64_t n,
                             unsigned long long *slots, uint64_t nslots, const RegionPlan &plan, const uint32_t *counts,
                             cudaStream_t s);

#define QE_CUDA(ctx, call)                                        \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return qe_cuda_fail(ctx, e_, #call); \
    } while (0)

#define QE_CHECK_LAUNCH(ctx) QE_CUDA(ctx, cudaGetLastError())

static inline int64_t qe_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int qe_log2_ceil(uint64_t x)
{
    int l = 0;
    while ((uint64_t(1) << l) < x) l++;
    return l;
}
static inline bool qe_aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
static inline bool qe_valid_type(int t) { return t == QE_I8 || t == QE_I32 || t == QE_I64; }

// ------------------------------------------------------------------ device

#define QE_FULL_MASK 0xffffffffu

__device__ __forceinline__ void dev_report(qe_dev_status *st, int code, int64_t required)
{
    atomicCAS(&st->code, 0, code);
    if (required > 0)
        atomicMax(reinterpret_cast<unsigned long long *>(&st->required),
                  static_cast<unsigned long long>(required));
}

// Bounds check of the checked build (QE_CHECKED): true when `cond` holds;
// otherwise records QE_ERR_DEVICE_CHECK with `val` and returns false, so the
// caller skips the access.  Always true in the plain build.
#ifdef QE_CHECKED
#define QE_DCHECK(st, cond, val) \
    ((cond) ? true : (dev_report((st), QE_ERR_DEVICE_CHECK, static_cast<int64_t>(val) + 1), false))
#else
#define QE_DCHECK(st, cond, val) true
#endif

// MurmurHash3 64-bit finalizer (A. Appleby, public domain), the partition
// function: destination = top log2(F) bits.
__device__ __forceinline__ uint64_t dev_fmix64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

// MurmurHash3 32-bit finalizer: slot hash of the open-addressing join table.
__device__ __forceinline__ uint32_t dev_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Partition id: hash mode (top bits of fmix64) or radix mode (key bits).
__device__ __forceinline__ uint32_t dev_part_id(int64_t key, int log2f, int mode, int shift)
{
    if (log2f == 0) return 0;
    uint64_t k = static_cast<uint64_t>(key);
    if (mode == QE_PART_HASH) {
        // The destination is the top log2f (<= 12) bits of fmix64(k).  They
        // lie in the high word, which fmix64's last step k ^= k >> 33 leaves
        // unchanged, so it is skipped.
        k ^= k >> 33;
        k *= 0xff51afd7ed558ccdULL;
        k ^= k >> 33;
        k *= 0xc4ceb9fe1a85ec53ULL;
        return static_cast<uint32_t>(k >> 32) >> (32 - log2f);
    }
    return static_cast<uint32_t>((k >> shift) & ((uint64_t(1) << log2f) - 1));
}

// L2 eviction policies (createpolicy) and loads that carry one.  The fused
// pipeline streams its fact columns once (evict first) while the dimension's
// payload array is looked up at random for the whole pass (evict last), so
// the lookups keep hitting L2 instead of being pushed out by the stream.
__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ int32_t ld_hint_i32(const int32_t *a, uint64_t pol)
{
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ int32_t ld_hint_s8(const signed char *a, uint64_t pol)
{
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s8 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ long long ld_hint_i64(const long long *a, uint64_t pol)
{
    long long v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol));
    return v;
}

// Random lookup that allocates in L1 and carries an L2 policy.
__device__ __forceinline__ int32_t ld_lookup_i32(const int32_t *a, uint64_t pol)
{
    int32_t v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}

// Read element i of a column as int64 (sign-extended).
__device__ __forceinline__ int64_t dev_col(const void *p, int type, int64_t i)
{
    if (type == QE_I32) return static_cast<int64_t>(__ldg(static_cast<const int32_t *>(p) + i));
    if (type == QE_I64) return __ldg(static_cast<const long long *>(p) + i);
    return static_cast<int64_t>(__ldg(static_cast<const signed char *>(p) + i));
}

// Streaming read (evict-first): fact columns are read once per pass.
__device__ __forceinline__ int64_t dev_col_stream(const void *p, int type, int64_t i)
{
    if (type == QE_I32) return static_cast<int64_t>(__ldcs(static_cast<const int32_t *>(p) + i));
    if (type == QE_I64) return __ldcs(static_cast<const long long *>(p) + i);
    return static_cast<int64_t>(__ldcs(reinterpret_cast<const signed char *>(p) + i));
}

__device__ __forceinline__ bool dev_cmp(int64_t x, int op, int64_t lo, int64_t hi)
{
    switch (op) {
    case QE_LT: return x < lo;
    case QE_LE: return x <= lo;
    case QE_GT: return x > lo;
    case QE_GE: return x >= lo;
    case QE_EQ: return x == lo;
    case QE_NE: return x != lo;
    default: return lo <= x && x <= hi;
    }
}

// A comparison as a closed range [a, b], possibly negated: x satisfies
// (lo, op, hi) iff (a <= x <= b) != neg.  Returns false when [a, b] is empty.
__host__ __device__ inline bool qe_pred_range(int op, int64_t lo, int64_t hi, int64_t &a, int64_t &b, bool &neg)
{
    a = INT64_MIN;
    b = INT64_MAX;
    neg = false;
    switch (op) {
    case QE_LT:
        if (lo == INT64_MIN) return false;
        b = lo - 1;
        return true;
    case QE_LE: b = lo; return true;
    case QE_GT:
        if (lo == INT64_MAX) return false;
        a = lo + 1;
        return true;
    case QE_GE: a = lo; return true;
    case QE_EQ: a = b = lo; return true;
    case QE_NE: a = b = lo; neg = true; return true;
    default: a = lo; b = hi; return lo <= hi;
    }
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(QE_FULL_MASK, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(QE_FULL_MASK, v, d);
    return v;
}

// ---------------------------------------------- decoupled look-back scan
// Single-pass prefix over tiles (Merrill & Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", 2016).  A status word holds a
// 2-bit flag (0 = not ready, 1 = tile aggregate, 2 = inclusive prefix) and a
// 62-bit count.  Tiles are claimed in order from an atomic counter, so every
// tile a claimant waits on is already running; each wait is still bounded
// and reports QE_ERR_TIMEOUT instead of spinning forever.

#define LB_AGG (1ull << 62)
#define LB_PRE (2ull << 62)
#define LB_VAL ((1ull << 62) - 1)

__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Called by one full warp.  Publishes `agg` for `tile`, returns the exclusive
// prefix of the tile (identical in all lanes) and publishes the inclusive one.
__device__ __forceinline__ int64_t lb_exclusive(unsigned long long *state, int64_t tile, int64_t agg,
                                                qe_dev_status *st, int64_t spin_limit)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) lb_store(state, LB_PRE | static_cast<unsigned long long>(agg));
        return 0;
    }
    if (lane == 0) lb_store(state + tile, LB_AGG | static_cast<unsigned long long>(agg));
    int64_t excl = 0, pred = tile - 1, spins = 0;
    while (true) {
        // a window of 32 predecessors, nearest in lane 0: sum back to the
        // nearest one that published its inclusive prefix; only the tiles up
        // to it must have published something
        int64_t t = pred - lane;
        unsigned long long w = t >= 0 ? lb_load(state + t) : LB_PRE;
        unsigned flag = static_cast<unsigned>(w >> 62);
        const unsigned pm = __ballot_sync(QE_FULL_MASK, flag == 2);
        const unsigned nr = __ballot_sync(QE_FULL_MASK, flag == 0);
        const int stop = pm ? __ffs(pm) - 1 : 31;
        const unsigned need = stop == 31 ? QE_FULL_MASK : ((2u << stop) - 1u);
        if (nr & need) {
            if (++spins > spin_limit) {
                if (lane == 0) dev_report(st, QE_ERR_TIMEOUT, 0);
                break;
            }
            __nanosleep(32);
            continue;
        }
        int64_t v = lane <= stop ? static_cast<int64_t>(w & LB_VAL) : 0;
        excl += warp_sum(v);
        if (pm) break;
        pred -= 32;
    }
    if (lane == 0) lb_store(state + tile, LB_PRE | static_cast<unsigned long long>(excl + agg));
    return excl;
}

// ---------------------------------------------- join table view
struct HtView {
    int32_t layout;          // QE_HT_DENSE / QE_HT_OPEN
    int32_t full;            // dense: every slot occupied (no bitmap check)
    int32_t key_min;
    uint32_t range;          // dense: key_max - key_min + 1
    uint32_t mask;           // open: slots - 1
    const int32_t *payload;  // dense payload [range]
    const uint32_t *bitmap;  // dense occupancy [ceil(range/32)]
    const unsigned long long *slots;  // open: key << 32 | payload
    int32_t coherent;        // built by the same kernel: read through L2 only
    int32_t pad;
};

// Read a join-table word: the read-only path for tables built before the
// kernel, L2-only (coherent) loads for tables built earlier in the same
// kernel by other blocks.
template <typename T>
__device__ __forceinline__ T ht_ld(const HtView &h, const T *p)
{
    return h.coherent ? __ldcg(p) : __ldg(p);
}

#define HT_EMPTY_KEY (static_cast<int32_t>(0x80000000u))
#define HT_EMPTY_SLOT 0x8000000080000000ull

__device__ __forceinline__ bool ht_lookup(const HtView &h, int32_t key, int32_t &pay)
{
    if (h.layout == QE_HT_DENSE) {
        uint32_t s = static_cast<uint32_t>(key) - static_cast<uint32_t>(h.key_min);
        if (s >= h.range) return false;
        int32_t p = ht_ld(h, h.payload + s);
        if (!h.full && !((ht_ld(h, h.bitmap + (s >> 5)) >> (s & 31)) & 1u)) return false;
        pay = p;
        return true;
    }
    uint32_t i = dev_fmix32(static_cast<uint32_t>(key)) & h.mask;
    for (uint32_t probes = 0; probes <= h.mask; probes++) {
        unsigned long long w = ht_ld(h, h.slots + i);
        int32_t k = static_cast<int32_t>(w >> 32);
        if (k == key) {
            pay = static_cast<int32_t>(w & 0xffffffffu);
            return true;
        }
        if (k == HT_EMPTY_KEY) return false;
        i = (i + 1) & h.mask;
    }
    return false;
}

// Membership only: the payload is not read (a key set has none).
__device__ __forceinline__ bool ht_contains(const HtView &h, int32_t key)
{
    if (h.layout == QE_HT_DENSE) {
        uint32_t s = static_cast<uint32_t>(key) - static_cast<uint32_t>(h.key_min);
        if (s >= h.range) return false;
        return h.full || ((ht_ld(h, h.bitmap + (s >> 5)) >> (s & 31)) & 1u);
    }
    uint32_t i = dev_fmix32(static_cast<uint32_t>(key)) & h.mask;
    for (uint32_t probes = 0; probes <= h.mask; probes++) {
        const int32_t k = static_cast<int32_t>(ht_ld(h, h.slots + i) >> 32);
        if (k == key) return true;
        if (k == HT_EMPTY_KEY) return false;
        i = (i + 1) & h.mask;
    }
    return false;
}

// ---------------------------------------------- group tables
// Keys are stored as key ^ INT64_MIN so that an all-zero slot is empty
// (INT64_MIN itself is reserved).  Aggregates are stored so that zero is
// each one's identity and every update is an unsigned atomic:
//   SUM   : two's-complement sum (atomicAdd)
//   COUNT : atomicAdd 1
//   MIN   : ~(v ^ SIGN), combined with atomicMax
//   MAX   :  (v ^ SIGN), combined with atomicMax
#define GB_SIGN 0x8000000000000000ull

struct AggOps {
    int n;
    int op[QE_MAX_AGGS];
};

__device__ __forceinline__ unsigned long long agg_encode(int op, int64_t v)
{
    unsigned long long u = static_cast<unsigned long long>(v);
    if (op == QE_SUM) return u;
    if (op == QE_COUNT) return 1ull;
    if (op == QE_MIN) return ~(u ^ GB_SIGN);
    return u ^ GB_SIGN;
}

__device__ __forceinline__ int64_t agg_decode(int op, unsigned long long s)
{
    if (op == QE_MIN) return static_cast<int64_t>(~s ^ GB_SIGN);
    if (op == QE_MAX) return static_cast<int64_t>(s ^ GB_SIGN);
    return static_cast<int64_t>(s);
}

// Fold an encoded contribution into an aggregate cell (shared or global).
// Fold one encoded value into an HBM aggregate cell.  The MAX-kind check
// reads L2 (where the atomics land) without the ordering of a volatile
// load, so independent rows' reads can overlap; a stale value can only
// cause a redundant atomic, since cells only grow.
__device__ __forceinline__ void agg_fold(unsigned long long *cell, int op, unsigned long long e)
{
    if (op == QE_SUM || op == QE_COUNT) {
        if (e) atomicAdd(cell, e);
    } else {
        if (__ldcg(cell) < e) atomicMax(cell, e);
    }
}

__device__ __forceinline__ uint32_t gb_hash(unsigned long long kx) { return static_cast<uint32_t>(dev_fmix64(kx)); }

// Global (HBM) group table: `slots` entries of (1 + naggs) words.
struct GTable {
    unsigned long long *words;
    uint64_t mask;                    // slots - 1
    int stride;                       // 1 + naggs
    int64_t capacity;                 // caller's group capacity
    qe_dev_status *st;
};

// Longest probe chain before the table counts as overfull.  With at least
// twice as many slots as the caller's capacity the load stays at or below
// one half while the groups fit, where linear-probing chains stay short.
#define GT_MAX_PROBE 4096

// Returns the slot index of key kx (inserting it), or -1 when no slot turns
// up within GT_MAX_PROBE probes (more groups than the capacity filled the
// table; QE_ERR_CAPACITY recorded).  Groups are counted, and a count above
// the capacity reported, when the table is compacted, so inserts share no
// counter.  Slot keys only change from 0 to their key, so a stale read
// (plain L2 loads, no volatile ordering) is either 0 (the CAS then returns
// the key) or the final key.
__device__ __forceinline__ int64_t gt_find_insert(const GTable &g, unsigned long long kx)
{
    uint64_t i = gb_hash(kx) & g.mask;
    const uint64_t limit = g.mask < GT_MAX_PROBE ? g.mask : GT_MAX_PROBE;
    for (uint64_t probes = 0; probes <= limit; probes++) {
        unsigned long long *cell = g.words + i * g.stride;
        const unsigned long long cur = __ldcg(cell);
        if (cur == kx) return static_cast<int64_t>(i);
        if (cur == 0) {
            const unsigned long long old = atomicCAS(cell, 0ull, kx);
            if (old == 0 || old == kx) return static_cast<int64_t>(i);
        }
        i = (i + 1) & g.mask;
    }
    dev_report(g.st, QE_ERR_CAPACITY, g.capacity + 1);
    return -1;
}

// Shared-memory group table: keys[S] then aggs[a][S] (S a power of two).
// Returns the slot of kx or -1 when max_probe slots were tried (spill).
__device__ __forceinline__ int st_find_insert(unsigned long long *keys, uint32_t mask, unsigned long long kx,
                                              int max_probe)
{
    uint32_t i = gb_hash(kx) & mask;
    for (int p = 0; p < max_probe; p++) {
        unsigned long long cur = reinterpret_cast<volatile unsigned long long *>(keys)[i];
        if (cur == kx) return static_cast<int>(i);
        if (cur == 0) {
            unsigned long long old = atomicCAS(keys + i, 0ull, kx);
            if (old == 0 || old == kx) return static_cast<int>(i);
        }
        i = (i + 1) & mask;
    }
    return -1;
}

// Fold one row (encoded contributions e[a]) into the global table.
__device__ __forceinline__ void gt_fold_row(const GTable &g, const AggOps &ops, unsigned long long kx,
                                            const unsigned long long *e)
{
    int64_t s = gt_find_insert(g, kx);
    if (s < 0) return;
    unsigned long long *cell = g.words + s * g.stride + 1;
    _Pragma("unroll") for (int a = 0; a < QE_MAX_AGGS; a++) if (a < ops.n) agg_fold(cell + a, ops.op[a], e[a]);
}

// Zero a shared-memory table of S slots (keys then naggs aggregate rows).
__device__ __forceinline__ void st_zero(unsigned long long *sm, int S, int naggs)
{
    for (int i = threadIdx.x; i < S * (1 + naggs); i += blockDim.x) sm[i] = 0;
}

// Fold one row into the shared-memory table, spilling to the global table
// when the key is not placed within max_probe slots.
__device__ __forceinline__ void st_fold_row(unsigned long long *sm, int S, const AggOps &ops, const GTable &g,
                                            unsigned long long kx, const unsigned long long *e, int max_probe)
{
    if (S) {
        int slot = st_find_insert(sm, static_cast<uint32_t>(S - 1), kx, max_probe);
        if (slot >= 0) {
            _Pragma("unroll") for (int a = 0; a < QE_MAX_AGGS; a++) if (a < ops.n) agg_fold(sm + (a + 1) * S + slot, ops.op[a], e[a]);
            return;
        }
    }
    gt_fold_row(g, ops, kx, e);
}

// Merge a block's shared-memory table into the global table (after the
// block's last update and a __syncthreads()).
__device__ __forceinline__ void st_flush(unsigned long long *sm, int S, const AggOps &ops, const GTable &g)
{
    for (int slot = threadIdx.x; slot < S; slot += blockDim.x) {
        unsigned long long kx = sm[slot];
        if (!kx) continue;
        unsigned long long e[QE_MAX_AGGS];
        _Pragma("unroll") for (int a = 0; a < QE_MAX_AGGS; a++) if (a < ops.n) e[a] = sm[(a + 1) * S + slot];
        gt_fold_row(g, ops, kx, e);
    }
}

// ------------------------------------------------------------ dense group layout
// When the two parts of the group key have known, small ranges, the group
// table is a direct array (a perfect hash): slot = (hi - hi_min) * lo_span +
// (lo - lo_min).  Each slot holds the aggregate words plus, when no COUNT is
// asked for, one hidden row count that marks occupied slots.
struct DenseKey {
    int32_t on;
    int32_t has_hi;
    int64_t hi_min, lo_min;
    uint64_t hi_span, lo_span;
    uint64_t nslots;
    int32_t occ;       // word that counts rows (a COUNT aggregate or the hidden word)
    int32_t stride;    // words per slot
    int32_t hidden;    // the occ word is hidden (no COUNT aggregate)
    int32_t pad;
};

__device__ __forceinline__ int64_t dense_index(const DenseKey &d, int64_t hi, int64_t lo)
{
    const uint64_t l = static_cast<uint64_t>(lo - d.lo_min);
    if (l >= d.lo_span) return -1;
    uint64_t h = 0;
    if (d.has_hi) {
        h = static_cast<uint64_t>(hi - d.hi_min);
        if (h >= d.hi_span) return -1;
    }
    return static_cast<int64_t>(h * d.lo_span + l);
}

__device__ __forceinline__ int64_t dense_key(const DenseKey &d, uint64_t idx)
{
    const int64_t lo = d.lo_min + static_cast<int64_t>(idx % d.lo_span);
    if (!d.has_hi) return lo;
    const int64_t hi = d.hi_min + static_cast<int64_t>(idx / d.lo_span);
    return static_cast<int64_t>((static_cast<uint64_t>(hi) << 32) | static_cast<uint32_t>(lo));
}

// Host: a dense layout for the key parts' ranges, or on = 0 when the ranges
// are too wide (more than max_slots slots, or a 64-bit low part that the key
// packing would truncate).
static inline DenseKey dense_plan(bool has_hi, int64_t hi_min, int64_t hi_max, int64_t lo_min, int64_t lo_max,
                                  const AggOps &ops, uint64_t max_slots)
{
    DenseKey d{};
    if (lo_max < lo_min || (has_hi && hi_max < hi_min)) return d;
    const uint64_t ls = static_cast<uint64_t>(lo_max - lo_min) + 1;
    const uint64_t hs = has_hi ? static_cast<uint64_t>(hi_max - hi_min) + 1 : 1;
    if (ls == 0 || hs == 0 || ls > max_slots || hs > max_slots || ls * hs > max_slots) return d;
    if (has_hi && ls > (1ull << 32)) return d;
    d.on = 1;
    d.has_hi = has_hi;
    d.hi_min = has_hi ? hi_min : 0;
    d.lo_min = lo_min;
    d.hi_span = hs;
    d.lo_span = ls;
    d.nslots = ls * hs;
    d.occ = -1;
    for (int a = 0; a < ops.n; a++)
        if (ops.op[a] == QE_COUNT) d.occ = a;
    d.hidden = d.occ < 0;
    if (d.hidden) d.occ = ops.n;
    d.stride = ops.n + (d.hidden ? 1 : 0);
    return d;
}

// Host helpers shared by group-by and pipeline.
struct GroupTableHost {
    unsigned long long *words = nullptr;  // device
    uint64_t slots = 0;
    int stride = 0;
    size_t bytes = 0;
};

qe_status gt_create(qe_ctx *ctx, int64_t capacity, int naggs, GroupTableHost &t, cudaStream_t s);
// Compact the table into `out` (keys + decoded aggregates + ngroups).
qe_status gt_finalize(qe_ctx *ctx, const GroupTableHost &t, const AggOps &ops, const qe_groups_out *out,
                      cudaStream_t s);
// Same, first emitting the occupied slots of a global dense table
// (AoS, d.stride words per slot).
qe_status gt_finalize_dense(qe_ctx *ctx, const GroupTableHost &t, const AggOps &ops, const DenseKey &d,
                            const unsigned long long *dense, const qe_groups_out *out, cudaStream_t s);
// Checks the output arrays of a group-by with aggregates `ops`, including
// the derived averages (each over a SUM, with a COUNT among the aggregates).
qe_status gt_check_out(qe_ctx *ctx, const qe_groups_out *out, const AggOps &ops);
int agg_count_index(const AggOps &ops);

// Derived averages of one output group (Sec. 2.3 lists average among the
// final aggregation kinds): for each aggregate a with out.avg[a] set,
// avg = (double)SUM / (double)COUNT from the exact int64 values; value(a)
// returns aggregate a of the group, cnt is the COUNT aggregate's index.
template <class F>
__device__ __forceinline__ void write_avgs(const qe_groups_out &out, int64_t pos, int naggs, int cnt, F value)
{
    double c = 0.0;
    bool have_c = false;
    for (int a = 0; a < naggs; a++) {
        if (!out.avg[a]) continue;
        if (!have_c) {
            c = static_cast<double>(value(cnt));
            have_c = true;
        }
        out.avg[a][pos] = static_cast<double>(value(a)) / c;
    }
}

// Smem group-table sizing: slots for `groups` at <= 75% load, 0 when the
// table would not fit `smem_budget` bytes.
static inline int st_slots_for(int64_t groups, int naggs, size_t smem_budget)
{
    uint64_t want = static_cast<uint64_t>(groups) * 4 / 3 + 1;
    uint64_t s = 64;
    while (s < want) s <<= 1;
    if (s * 8 * (1 + naggs) > smem_budget) return 0;
    return static_cast<int>(s);
}

// Largest power-of-two slot count whose table fits `smem_budget` bytes.
static inline int st_slots_max(int naggs, size_t smem_budget)
{
    uint64_t s = 64;
    if (s * 8 * (1 + naggs) > smem_budget) return 0;
    while ((s * 2) * 8 * (1 + naggs) <= smem_budget) s <<= 1;
    return static_cast<int>(s);
}

// Library-owned join table (qe_join.cu builds it).
struct qe_hash_table {
    int32_t layout = QE_HT_DENSE;
    int32_t full = 0;
    int32_t key_min = 0, key_max = -1;
    int32_t have_pay = 0, pay_min = 0, pay_max = -1;
    int64_t nkeys = 0;
    int64_t slots = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    int32_t *payload = nullptr;       // NULL for a key set
    uint32_t *bitmap = nullptr;
    unsigned long long *open = nullptr;
    int32_t set = 0;                  // key set: membership only, keys may repeat
    int32_t multi = 0;                // multimap (qe_join_build_multi): payload = the runs of values
    int32_t pair = 0;                 // pair keys (qe_join_build_pair): open = packed keys, payload per slot
    int64_t *mstart = nullptr;        // multimap: each key's run (per dense slot / open slot), start << 32 | length
    uint32_t *mcnt = nullptr;         // multimap: rows of each key
};

HtView ht_view(const qe_hash_table *ht);
// Min and max of nrows build keys (and of the payloads when pay is not
// NULL) into mm = {kmin, kmax, pmin, pmax}; synchronizes the stream.
qe_status join_key_range(qe_ctx *ctx, const int32_t *keys, const int32_t *pay, int64_t nrows, int32_t mm[4],
                         cudaStream_t s);
// key_set: membership only (repeated keys allowed, payload ignored and not stored).
qe_status join_build_impl(qe_ctx *ctx, const int32_t *keys, const int32_t *payload, int64_t nrows,
                          const qe_build_opts *opts, bool key_set, qe_hash_table **out, cudaStream_t s);
