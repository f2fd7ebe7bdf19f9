// qe_join_part.cu -- region-ordered join builds (Sec. 7.2: a hash table with
// hundreds of millions of keys is too large to build efficiently; Sec. 2.2:
// one partitioning function applied to the rows before the local join).
//
// Inserting rows in their input order into a table far larger than L2 puts
// every insert at a random slot: a DRAM read-modify-write of one sector on a
// random page.  Here the build rows are first partitioned into P regions by
// the top bits of the slot they hash to (a dense table: by the top bits of
// key - key_min), and the unchanged insert kernels then run over the rows in
// region order.  Their grid-stride loops keep the blocks in flight within a
// window of a few hundred thousand consecutive rows, so they insert into one
// or two regions of tens of MB at a time: those stay in L2, the table's
// pages are visited in order, and every sector of the table leaves the chip
// once.  The order of rows inside a region is not kept; the builds that use
// it do not depend on insertion order for their result (an open-addressing
// table finds the same key set in any order, and the order inside a
// multimap's run is unspecified).
//
// Two kernels and a memset:
//   k_rp_count    rows per region (shared-memory histogram per block, one
//                 global add per block and region);
//   k_rp_scatter  tiles of 4,096 rows: rank each row in its region by a
//                 shared-memory atomic, claim the tile's run of every region
//                 with one global add, stage the tile in region order in
//                 shared memory and write it out run by run.
#include "qe_internal.cuh"

namespace {

constexpr int RT = 512;                 // scatter threads per block
constexpr int R_ITEMS = 8;              // rows per thread and tile
constexpr int R_TILE = RT * R_ITEMS;    // 4,096 rows
constexpr int R_MAXP = 256;
constexpr int R_MAXC = 3;
constexpr int CT = 1024;                // count threads per block
constexpr int C_ITEMS = 4;

struct RegionArgs {
    int kind, shift;
    uint32_t mask, last;    // last = regions - 1
    int32_t kmin;
    int p, ncols;
    int64_t n;
    const int32_t *in[R_MAXC];
    int32_t *out[R_MAXC];
    uint32_t *cnt;          // [p] rows per region
    uint32_t *used;         // [p] rows placed so far
    qe_dev_status *st;
};

__device__ __forceinline__ uint32_t rp_region(const RegionArgs &A, int32_t k0, int32_t k1)
{
    if (A.kind == RP_DENSE) {
        // keys outside the range go to the last region; the insert kernel reports them
        const uint32_t d = static_cast<uint32_t>(k0) - static_cast<uint32_t>(A.kmin);
        return min(d >> A.shift, A.last);
    }
    uint32_t slot;
    if (A.kind == RP_PAIR64) {
        const unsigned long long k = (static_cast<unsigned long long>(static_cast<uint32_t>(k0)) << 32) |
                                     static_cast<uint32_t>(k1);
        slot = static_cast<uint32_t>(dev_fmix64(k)) & A.mask;
    } else {
        slot = dev_fmix32(static_cast<uint32_t>(k0)) & A.mask;
    }
    return slot >> A.shift;
}

__global__ void __launch_bounds__(CT) k_rp_count(RegionArgs A)
{
    __shared__ uint32_t h[R_MAXP];
    for (int i = threadIdx.x; i < A.p; i += CT) h[i] = 0;
    __syncthreads();
    const bool two = A.kind == RP_PAIR64;
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * CT * C_ITEMS; b < A.n;
         b += static_cast<int64_t>(gridDim.x) * CT * C_ITEMS) {
        int32_t k0[C_ITEMS], k1[C_ITEMS];
#pragma unroll
        for (int j = 0; j < C_ITEMS; j++) {
            const int64_t i = b + j * CT + threadIdx.x;
            k0[j] = i < A.n ? __ldcs(A.in[0] + i) : 0;
            k1[j] = two && i < A.n ? __ldcs(A.in[1] + i) : 0;
        }
#pragma unroll
        for (int j = 0; j < C_ITEMS; j++)
            if (b + j * CT + threadIdx.x < A.n) atomicAdd(&h[rp_region(A, k0[j], k1[j])], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < A.p; i += CT)
        if (h[i]) atomicAdd(A.cnt + i, h[i]);
}

// Exclusive scan of v[0..p) in place by the first warps of the block (p <=
// 256 = 8 warps x 32); returns nothing, every thread must call it.
__device__ __forceinline__ void rp_scan(uint32_t *v, uint32_t *wsum, int p)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = 0;
    if (threadIdx.x < R_MAXP) {
        x = threadIdx.x < p ? v[threadIdx.x] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(QE_FULL_MASK, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) wsum[w] = x;
    }
    __syncthreads();
    if (threadIdx.x < R_MAXP && threadIdx.x < p) {
        uint32_t off = 0;
        for (int i = 0; i < w; i++) off += wsum[i];
        v[threadIdx.x] = off + x - v[threadIdx.x];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(RT, 2) k_rp_scatter(RegionArgs A)
{
    extern __shared__ __align__(16) int32_t sm[];
    int32_t *s_col = sm;                                             // [ncols][R_TILE]
    uint8_t *s_reg = reinterpret_cast<uint8_t *>(sm + R_MAXC * R_TILE);   // [R_TILE]
    __shared__ uint32_t s_excl[R_MAXP], s_hist[R_MAXP], s_base[R_MAXP], s_wsum[R_MAXP / 32];

    // every region's start in the output: exclusive scan of the counts
    for (int i = threadIdx.x; i < R_MAXP; i += RT) s_excl[i] = i < A.p ? A.cnt[i] : 0;
    __syncthreads();
    rp_scan(s_excl, s_wsum, A.p);

    const bool two = A.kind == RP_PAIR64;
    const int64_t ntiles = (A.n + R_TILE - 1) / R_TILE;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * R_TILE;
        const int rows = static_cast<int>(min(static_cast<int64_t>(R_TILE), A.n - base));
        for (int i = threadIdx.x; i < R_MAXP; i += RT) s_hist[i] = 0;
        int32_t v[R_MAXC][R_ITEMS];
#pragma unroll
        for (int j = 0; j < R_ITEMS; j++) {
            const int r = j * RT + threadIdx.x;
#pragma unroll
            for (int c = 0; c < R_MAXC; c++)
                v[c][j] = c < A.ncols && r < rows ? __ldcs(A.in[c] + base + r) : 0;
        }
        __syncthreads();
        uint32_t reg[R_ITEMS], rk[R_ITEMS];
#pragma unroll
        for (int j = 0; j < R_ITEMS; j++) {
            reg[j] = rp_region(A, v[0][j], two ? v[1][j] : 0);
            rk[j] = j * RT + static_cast<int>(threadIdx.x) < rows ? atomicAdd(&s_hist[reg[j]], 1u) : 0;
        }
        __syncthreads();
        // claim this tile's run of every region; then the runs' starts inside the tile
        for (int i = threadIdx.x; i < A.p; i += RT)
            s_base[i] = s_hist[i] ? s_excl[i] + atomicAdd(A.used + i, s_hist[i]) : 0;
        __syncthreads();
        rp_scan(s_hist, s_wsum, A.p);
#pragma unroll
        for (int j = 0; j < R_ITEMS; j++) {
            if (j * RT + static_cast<int>(threadIdx.x) >= rows) continue;
            const uint32_t pos = s_hist[reg[j]] + rk[j];
            if (!QE_DCHECK(A.st, pos < static_cast<uint32_t>(R_TILE), pos)) continue;
#pragma unroll
            for (int c = 0; c < R_MAXC; c++)
                if (c < A.ncols) s_col[c * R_TILE + pos] = v[c][j];
            s_reg[pos] = static_cast<uint8_t>(reg[j]);
        }
        __syncthreads();
        for (int pos = threadIdx.x; pos < rows; pos += RT) {
            const uint32_t r = s_reg[pos];
            const int64_t o = static_cast<int64_t>(s_base[r]) + (pos - static_cast<int64_t>(s_hist[r]));
            if (!QE_DCHECK(A.st, o >= 0 && o < A.n, o)) continue;
#pragma unroll
            for (int c = 0; c < R_MAXC; c++)
                if (c < A.ncols) A.out[c][o] = s_col[c * R_TILE + pos];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ fill + insert
// An open-addressing table built from region-ordered rows in one kernel that
// also fills it: work items are taken in the order F0 .. F(L-1), then
// F(L), I0, F(L+1), I1, ..., I(p-1), where F(r) writes the empty marker over
// region r (items of 128 KB) and I(r) inserts region r's rows (items of
// 2,048 rows); the fills lead the inserts by L regions, L chosen so that the
// items between a fill and the inserts waiting on it outnumber the blocks.
// An insert item first waits (bounded) until regions r and r+1 are filled,
// since a probe may run on past the end of its region.  A region is thus
// written shortly before its inserts, its lines are still in L2 when the
// CASes arrive, and the table goes to DRAM once, when its lines leave L2:
// no DRAM read of the table at all.  A probe that would leave regions r and
// r+1 (never seen at load factor <= 0.5; possible for adversarial keys)
// stops there and its row goes to an overflow list, inserted by a second
// kernel into the complete table.
constexpr int FT = 512;
constexpr int FI_ROWS = 4;
constexpr int FI_ITEM = FT * FI_ROWS;                   // rows per insert item (2,048)
constexpr int64_t FILL_WORDS = int64_t(FT) * 16 * 2;    // 64-bit words per fill item (128 KB)

struct FillInsertArgs {
    const int32_t *c0, *c1, *c2;   // open: key, payload (NULL: a key set); pair: hi, lo, payload
    int pair;
    int64_t n;
    unsigned long long *slots;
    uint32_t mask;                 // slots - 1
    int shift, p;                  // region of slot h = h >> shift; p regions
    int64_t region_words;          // 64-bit words per region
    int fills;                     // fill items per region
    int lead;                      // L: regions the fills run ahead of the inserts
    const uint32_t *cnt;           // [p] rows per region, in region order
    uint32_t *ctl;                 // [0] item ticket, [1] overflow rows, [2 + r] fill items done in region r
    uint32_t *ovf;                 // [ovf_cap] ordered row indices for the overflow kernel
    uint32_t ovf_cap;
    int64_t spin_limit;
    qe_dev_status *st;
};

__device__ __forceinline__ unsigned long long fi_key(const FillInsertArgs &A, int64_t i)
{
    if (A.pair)
        return (static_cast<unsigned long long>(static_cast<uint32_t>(__ldcs(A.c0 + i))) << 32) |
               static_cast<uint32_t>(__ldcs(A.c1 + i));
    return static_cast<uint32_t>(__ldcs(A.c0 + i));
}

__device__ __forceinline__ uint32_t fi_home(const FillInsertArgs &A, unsigned long long k)
{
    return (A.pair ? static_cast<uint32_t>(dev_fmix64(k)) : dev_fmix32(static_cast<uint32_t>(k))) & A.mask;
}

// The word a CAS claims for key k: the packed pair, or key << 32 | payload.
__device__ __forceinline__ unsigned long long *fi_slot(const FillInsertArgs &A, uint32_t h)
{
    return A.slots + (A.pair ? 2 * static_cast<uint64_t>(h) : h);
}

__device__ __forceinline__ bool fi_same_key(const FillInsertArgs &A, unsigned long long old, unsigned long long k)
{
    return A.pair ? old == k : static_cast<uint32_t>(old >> 32) == static_cast<uint32_t>(k);
}

__global__ void __launch_bounds__(FT, 2) k_region_fill_insert(FillInsertArgs A)
{
    __shared__ uint32_t s_seg[2 * R_MAXP + 1];   // first ticket of every segment
    __shared__ uint16_t s_what[2 * R_MAXP];      // segment: region | 0x8000 for a fill
    __shared__ uint32_t s_row[R_MAXP + 1];       // first ordered row of every region
    __shared__ uint32_t s_item, s_g, s_abort;
    const bool has_pay = A.pair || A.c1 != nullptr;
    for (int r = threadIdx.x; r < A.p; r += FT) s_row[r + 1] = A.cnt[r];
    __syncthreads();
    if (threadIdx.x == 0) {
        s_row[0] = 0;
        for (int r = 0; r < A.p; r++) s_row[r + 1] += s_row[r];
        uint32_t acc = 0;
        int g = 0;
        auto push = [&](int r, bool fill) {
            s_seg[g] = acc;
            s_what[g++] = static_cast<uint16_t>(r | (fill ? 0x8000 : 0));
            acc += fill ? static_cast<uint32_t>(A.fills)
                        : static_cast<uint32_t>((s_row[r + 1] - s_row[r] + FI_ITEM - 1) / FI_ITEM);
        };
        for (int r = 0; r < A.lead && r < A.p; r++) push(r, true);
        for (int r = 0; r < A.p; r++) {
            if (r + A.lead < A.p) push(r + A.lead, true);
            push(r, false);
        }
        s_seg[g] = acc;
        s_abort = 0;
    }
    __syncthreads();
    const uint32_t total = s_seg[2 * A.p];
    // thread 0 claims the next item while the block works on the current one;
    // an item only waits on items with smaller tickets, so the smallest
    // unfinished ticket is always some block's current item and progresses
    uint32_t next = threadIdx.x == 0 ? atomicAdd(A.ctl, 1u) : 0;
    while (true) {
        if (threadIdx.x == 0) {
            const uint32_t it = next;
            int lo = 0, hi = 2 * A.p;                     // s_seg[lo] <= it < s_seg[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_seg[mid] <= it) lo = mid;
                else hi = mid;
            }
            s_item = it;
            s_g = static_cast<uint32_t>(lo);
            if (it < total) next = atomicAdd(A.ctl, 1u);
        }
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= total) break;
        const int g = static_cast<int>(s_g);
        const uint32_t local = it - s_seg[g];
        const bool fill = (s_what[g] & 0x8000) != 0;
        const int r = s_what[g] & 0x7fff;
        if (fill) {
            const int64_t w0 = r * A.region_words + static_cast<int64_t>(local) * FILL_WORDS;
            const int64_t w1 = min(w0 + FILL_WORDS, (r + 1) * A.region_words);
            const uint4 e = make_uint4(0x80000000u, 0x80000000u, 0x80000000u, 0x80000000u);   // HT_EMPTY_SLOT
            for (int64_t w = w0 + 2 * threadIdx.x; w < w1; w += 2 * FT)
                *reinterpret_cast<uint4 *>(A.slots + w) = e;
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(A.ctl + 2 + r, 1u);
            }
            continue;
        }
        const int rn = r + 1 < A.p ? r + 1 : 0;
        if (threadIdx.x == 0) {
            int64_t spins = 0;
            while (*reinterpret_cast<volatile uint32_t *>(A.ctl + 2 + r) < static_cast<uint32_t>(A.fills) ||
                   *reinterpret_cast<volatile uint32_t *>(A.ctl + 2 + rn) < static_cast<uint32_t>(A.fills)) {
                if (++spins > A.spin_limit) {
                    dev_report(A.st, QE_ERR_TIMEOUT, 0);
                    s_abort = 1;
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
        }
        __syncthreads();
        if (s_abort) break;
        const int64_t ib = s_row[r] + static_cast<int64_t>(local) * FI_ITEM;
        const int64_t re = min(ib + FI_ITEM, static_cast<int64_t>(s_row[r + 1]));
        {
            const int64_t rb = ib;
            unsigned long long k[FI_ROWS], w[FI_ROWS], old[FI_ROWS];
            uint32_t h[FI_ROWS];
            int32_t pay[FI_ROWS];
            bool ok[FI_ROWS];
#pragma unroll
            for (int j = 0; j < FI_ROWS; j++) {
                const int64_t i = rb + j * FT + threadIdx.x;
                ok[j] = i < re;
                k[j] = ok[j] ? fi_key(A, i) : 0;
                pay[j] = ok[j] && has_pay ? __ldcs((A.pair ? A.c2 : A.c1) + i) : 0;
            }
#pragma unroll
            for (int j = 0; j < FI_ROWS; j++) {
                const bool reserved = A.pair ? k[j] == HT_EMPTY_SLOT : static_cast<int32_t>(k[j]) == HT_EMPTY_KEY;
                if (ok[j] && reserved) {
                    dev_report(A.st, QE_ERR_RESERVED_KEY, 0);
                    ok[j] = false;
                }
                w[j] = A.pair ? k[j] : (k[j] << 32) | static_cast<uint32_t>(pay[j]);
                h[j] = fi_home(A, k[j]);
                old[j] = ok[j] ? atomicCAS(fi_slot(A, h[j]), HT_EMPTY_SLOT, w[j]) : HT_EMPTY_SLOT;
            }
#pragma unroll
            for (int j = 0; j < FI_ROWS; j++) {
                if (!ok[j]) continue;
                for (uint32_t probes = 0;; probes++) {
                    if (old[j] == HT_EMPTY_SLOT) {
                        if (A.pair) reinterpret_cast<int32_t *>(fi_slot(A, h[j]) + 1)[0] = pay[j];
                        break;
                    }
                    if (fi_same_key(A, old[j], k[j])) {
                        if (has_pay) dev_report(A.st, QE_ERR_DUPLICATE_KEY, 0);
                        break;
                    }
                    if (probes >= A.mask) {
                        dev_report(A.st, QE_ERR_CAPACITY, A.n);
                        break;
                    }
                    h[j] = (h[j] + 1) & A.mask;
                    const int hr = static_cast<int>(h[j] >> A.shift);
                    if (hr != r && hr != rn) {
                        // the probe left the two filled regions: finish it after this kernel
                        const uint32_t o = atomicAdd(A.ctl + 1, 1u);
                        if (o < A.ovf_cap) A.ovf[o] = static_cast<uint32_t>(rb + j * FT + threadIdx.x);
                        else dev_report(A.st, QE_ERR_CAPACITY, A.n);
                        break;
                    }
                    old[j] = atomicCAS(fi_slot(A, h[j]), HT_EMPTY_SLOT, w[j]);
                }
            }
        }
        __syncthreads();
    }
}

// The overflow rows of k_region_fill_insert, into the complete table.
__global__ void __launch_bounds__(256) k_region_overflow(FillInsertArgs A)
{
    const uint32_t m = min(*reinterpret_cast<volatile uint32_t *>(A.ctl + 1), A.ovf_cap);
    const bool has_pay = A.pair || A.c1 != nullptr;
    for (uint32_t t = blockIdx.x * 256u + threadIdx.x; t < m; t += gridDim.x * 256u) {
        const int64_t i = A.ovf[t];
        const unsigned long long k = fi_key(A, i);
        const int32_t pay = has_pay ? __ldcs((A.pair ? A.c2 : A.c1) + i) : 0;
        const unsigned long long w = A.pair ? k : (k << 32) | static_cast<uint32_t>(pay);
        uint32_t h = fi_home(A, k);
        bool done = false;
        for (uint32_t probes = 0; probes <= A.mask && !done; probes++) {
            const unsigned long long old = atomicCAS(fi_slot(A, h), HT_EMPTY_SLOT, w);
            if (old == HT_EMPTY_SLOT) {
                if (A.pair) reinterpret_cast<int32_t *>(fi_slot(A, h) + 1)[0] = pay;
                done = true;
            } else if (fi_same_key(A, old, k)) {
                if (has_pay) dev_report(A.st, QE_ERR_DUPLICATE_KEY, 0);
                done = true;
            } else {
                h = (h + 1) & A.mask;
            }
        }
        if (!done) dev_report(A.st, QE_ERR_CAPACITY, A.n);
    }
}

}  // namespace

int region_plan_log2(const qe_ctx *ctx, uint64_t table_bytes, int64_t nrows, bool by_default)
{
    if (ctx->tune_join_partition == 1 || nrows <= 0) return 0;
    if (ctx->tune_join_partition == 0 &&
        (!by_default || table_bytes < (uint64_t(256) << 20) || nrows < (int64_t(1) << 22)))
        return 0;
    if (ctx->tune_join_part_log2 > 0) return ctx->tune_join_part_log2;
    // regions of about 32 MB, at least 2
    int l = qe_log2_ceil(qe_ceil_div(static_cast<int64_t>(table_bytes), int64_t(32) << 20));
    return l < 1 ? 1 : (l > 8 ? 8 : l);
}

qe_status region_order(qe_ctx *ctx, const RegionPlan &plan, const int32_t **cols, int ncols, int64_t n,
                       void **scratch, cudaStream_t s, const uint32_t **counts)
{
    *scratch = nullptr;
    if (counts) *counts = nullptr;
    if (plan.log2p == 0 || n <= 0) return QE_OK;
    if (plan.log2p < 1 || plan.log2p > 8 || plan.shift < 0 || plan.shift > 31 || ncols < 1 || ncols > R_MAXC ||
        (plan.kind == RP_PAIR64 && ncols < 2))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "region partition: bad plan");
    const size_t col_bytes = ((static_cast<size_t>(n) * 4 + 255) / 256) * 256;
    // the columns, then the counters
    qe_status st = qe_alloc(ctx, scratch, ncols * col_bytes + 2 * R_MAXP * sizeof(uint32_t), s);
    if (st != QE_OK) return st;
    RegionArgs A{};
    A.kind = plan.kind;
    A.shift = plan.shift;
    A.mask = plan.mask;
    A.kmin = plan.kmin;
    A.p = 1 << plan.log2p;
    A.last = static_cast<uint32_t>(A.p - 1);
    A.ncols = ncols;
    A.n = n;
    A.st = ctx->dstat;
    char *base = static_cast<char *>(*scratch);
    for (int c = 0; c < ncols; c++) {
        A.in[c] = cols[c];
        A.out[c] = reinterpret_cast<int32_t *>(base + c * col_bytes);
    }
    A.cnt = reinterpret_cast<uint32_t *>(base + ncols * col_bytes);
    A.used = A.cnt + R_MAXP;
    const size_t smem = R_MAXC * R_TILE * sizeof(int32_t) + R_TILE;
    cudaError_t e =
        cudaFuncSetAttribute(k_rp_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaMemsetAsync(A.cnt, 0, 2 * R_MAXP * sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        ProfScope prof(ctx, "build_partition", s);
        const int64_t cg = qe_ceil_div(n, int64_t(CT) * C_ITEMS);
        k_rp_count<<<static_cast<unsigned>(cg < ctx->num_sms * 2 ? cg : ctx->num_sms * 2), CT, 0, s>>>(A);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            const int64_t tiles = qe_ceil_div(n, R_TILE);
            const int64_t g = tiles < ctx->num_sms * 2 ? tiles : ctx->num_sms * 2;
            k_rp_scatter<<<static_cast<unsigned>(g), RT, smem, s>>>(A);
            QE_LAUNCHED(ctx);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        qe_free(ctx, *scratch, s);
        *scratch = nullptr;
        return qe_cuda_fail(ctx, e, "region partition");
    }
    for (int c = 0; c < ncols; c++) cols[c] = A.out[c];
    if (counts) *counts = A.cnt;
    return QE_OK;
}

qe_status region_fill_insert(qe_ctx *ctx, bool pair, const int32_t *const *cols, bool has_pay, int64_t n,
                             unsigned long long *slots, uint64_t nslots, const RegionPlan &plan, const uint32_t *counts,
                             cudaStream_t s)
{
    const int p = 1 << plan.log2p;
    if (plan.log2p < 1 || plan.log2p > 8 || plan.shift < 4 || (uint64_t(p) << plan.shift) != nslots)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "region build: bad plan");
    FillInsertArgs A{};
    A.c0 = cols[0];
    A.c1 = pair || has_pay ? cols[1] : nullptr;
    A.c2 = pair ? cols[2] : nullptr;
    A.pair = pair ? 1 : 0;
    A.n = n;
    A.slots = slots;
    A.mask = static_cast<uint32_t>(nslots - 1);
    A.shift = plan.shift;
    A.p = p;
    A.region_words = (int64_t(1) << plan.shift) * (pair ? 2 : 1);
    A.fills = static_cast<int>(qe_ceil_div(A.region_words, FILL_WORDS));
    // lead: the items of L regions cover twice the tickets the blocks hold
    // (each holds its current item and the next); the L + 1 regions in
    // flight stay within about 80 MB of L2 where the region size allows
    const int grid = ctx->num_sms * 2;
    const int64_t per_region = A.fills + qe_ceil_div(qe_ceil_div(n, p), FI_ITEM);
    const int64_t region_bytes = A.region_words * 8;
    int64_t lead = qe_ceil_div(int64_t(4) * grid, per_region);
    const int64_t lead_l2 = (int64_t(80) << 20) / region_bytes - 1;
    if (lead > lead_l2) lead = lead_l2;
    if (lead > p - 1) lead = p - 1;
    A.lead = static_cast<int>(lead < 1 ? 1 : lead);
    A.cnt = counts;
    A.ovf_cap = static_cast<uint32_t>(n / 8 > 4096 ? n / 8 : 4096);
    A.spin_limit = ctx->spin_limit;
    A.st = ctx->dstat;
    void *mem = nullptr;
    const size_t ctl_bytes = ((2 + R_MAXP) * sizeof(uint32_t) + 255) / 256 * 256;
    qe_status st = qe_alloc(ctx, &mem, ctl_bytes + A.ovf_cap * sizeof(uint32_t), s);
    if (st != QE_OK) return st;
    A.ctl = static_cast<uint32_t *>(mem);
    A.ovf = reinterpret_cast<uint32_t *>(static_cast<char *>(mem) + ctl_bytes);
    cudaError_t e = cudaMemsetAsync(A.ctl, 0, ctl_bytes, s);
    if (e == cudaSuccess) {
        ProfScope prof(ctx, "build", s);
        k_region_fill_insert<<<grid, FT, 0, s>>>(A);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            k_region_overflow<<<ctx->num_sms, 256, 0, s>>>(A);
            QE_LAUNCHED(ctx);
            e = cudaGetLastError();
        }
    }
    qe_free(ctx, mem, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "region build");
    return QE_OK;
}
