// qe_compact.cuh -- single-pass stable stream compaction.
//
// A tile is 256 threads x ITEMS rows.  Warp w of a tile owns 32*ITEMS
// consecutive positions; item k of lane l is position w*32*ITEMS + k*32 + l,
// so every column read is one 128-byte (int32) or 256-byte (int64) coalesced
// warp access and the natural row order is (warp, item, lane).  Survivors of
// item k are ranked inside the warp with one ballot, warps are ranked with a
// shared-memory scan, and tiles with a block-wide decoupled look-back; each survivor
// is written once at its final position.  Tiles are claimed from an atomic
// counter by a persistent grid.
#pragma once

#include "qe_internal.cuh"

struct CompactCommon {
    int64_t n;                      // positions
    int64_t ntiles;
    int64_t capacity;               // output capacity
    int64_t *out_count;             // device
    unsigned long long *tile_state; // [ntiles], zeroed
    unsigned long long *tile_counter;
    qe_dev_status *st;
    int64_t spin_limit;
};

// Op must provide:
//   struct Pre;                                       per-thread loads of a tile
//   struct Slot;                                      per-thread item data
//   __device__ void load(int64_t pos0, const bool (&in)[ITEMS], Pre &p) const;
//        the tile's independent loads (in[k]: position in range);
//   __device__ void eval(int64_t pos0, bool (&ok)[ITEMS], const Pre &p, Slot &s) const;
//        pos0 = this lane's first position (item k is pos0 + 32k); ok[k]
//        arrives true for in-range positions; eval clears non-survivors.
//   __device__ void emit(int64_t out_pos, int64_t pos, int k, const Slot &s) const;
//
// Tiles are not prefetched across claims: a claimed tile that waits behind
// its block's current one would hold up the look-back of every later tile.
// Loads in flight come from resident blocks instead (registers per thread
// kept low so that many blocks fit).
// Decoupled look-back by the whole block (Merrill & Garland's single-pass
// scan): tile `tile` publishes its aggregate, then its 256 threads read 256
// predecessors per round, nearest first, and sum back to the nearest one
// that has published its inclusive prefix (all tiles up to it must have
// published at least their aggregate).  With hundreds of tiles in flight the
// nearest inclusive prefix is often a few hundred tiles back, which one
// warp would reach only after many dependent rounds.  Returns the exclusive
// prefix to every thread.  Bounded: after spin_limit empty rounds it records
// QE_ERR_TIMEOUT and returns what it has.
__device__ __forceinline__ int64_t lb_exclusive_block(unsigned long long *state, int64_t tile, int64_t agg,
                                                      qe_dev_status *st, int64_t spin_limit, int *s_min,
                                                      long long *s_sum)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) lb_store(state + tile, LB_AGG | static_cast<unsigned long long>(agg));
    int64_t excl = 0, pred = tile - 1, spins = 0;
    while (true) {
        if (threadIdx.x == 0) *s_min = 256;
        if (threadIdx.x < 8) s_sum[threadIdx.x] = 0;
        __syncthreads();
        const int64_t t = pred - threadIdx.x;
        const unsigned long long w = t >= 0 ? lb_load(state + t) : LB_PRE;
        const unsigned flag = static_cast<unsigned>(w >> 62);
        const unsigned pm = __ballot_sync(QE_FULL_MASK, flag == 2);
        if (lane == 0 && pm) atomicMin(s_min, warp * 32 + __ffs(pm) - 1);
        __syncthreads();
        const int stop = *s_min;                  // nearest inclusive prefix, 256 if none
        const bool mine = static_cast<int>(threadIdx.x) <= stop;
        if (__syncthreads_or(mine && flag == 0)) {
            if (++spins > spin_limit) {
                if (threadIdx.x == 0) dev_report(st, QE_ERR_TIMEOUT, 0);
                break;
            }
            __nanosleep(32);
            continue;
        }
        const int64_t v = warp_sum(mine ? static_cast<int64_t>(w & LB_VAL) : 0);
        if (lane == 0) s_sum[warp] = v;
        __syncthreads();
        int64_t round = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) round += s_sum[i];
        excl += round;
        if (stop < 256) break;
        pred -= 256;
        __syncthreads();                          // s_sum / s_min are reused
    }
    if (threadIdx.x == 0) lb_store(state + tile, LB_PRE | static_cast<unsigned long long>(excl + agg));
    return excl;
}

template <int ITEMS, class Op>
__global__ void __launch_bounds__(256) k_compact(CompactCommon C, Op op)
{
    constexpr int TILE = 256 * ITEMS;
    __shared__ long long s_tile;
    __shared__ int s_wofs[8];
    __shared__ int s_min;
    __shared__ long long s_sum[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    while (true) {
        if (threadIdx.x == 0) s_tile = static_cast<long long>(atomicAdd(C.tile_counter, 1ull));
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= C.ntiles) break;
        const int64_t pos0 = tile * TILE + warp * 32 * ITEMS + lane;
        bool ok[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) ok[k] = pos0 + 32 * k < C.n;
        typename Op::Pre pre;
        op.load(pos0, ok, pre);
        typename Op::Slot slot;
        op.eval(pos0, ok, pre, slot);
        unsigned mask[ITEMS];
        int wtotal = 0;
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            mask[k] = __ballot_sync(QE_FULL_MASK, ok[k]);
            wtotal += __popc(mask[k]);
        }
        if (lane == 0) s_wofs[warp] = wtotal;
        __syncthreads();
        int woff = 0, tot = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int x = s_wofs[i];
            woff += i < warp ? x : 0;
            tot += x;
        }
        const int64_t excl = lb_exclusive_block(C.tile_state, tile, tot, C.st, C.spin_limit, &s_min, s_sum);
        if (threadIdx.x == 0 && tile == C.ntiles - 1) {
            const int64_t total = excl + tot;
            *C.out_count = total;
            if (total > C.capacity) dev_report(C.st, QE_ERR_CAPACITY, total);
        }
        int64_t pos = excl + woff;
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            if (ok[k]) {
                int64_t o = pos + __popc(mask[k] & lt);
                if (o < C.capacity) op.emit(o, pos0 + 32 * k, k, slot);
            }
            pos += __popc(mask[k]);
        }
        __syncthreads();
    }
}

// Host: allocate + zero the tile state, launch a persistent grid, free.
template <int ITEMS, class Op>
qe_status launch_compact(qe_ctx *ctx, const char *name, int64_t n, int64_t capacity, int64_t *out_count,
                         const Op &op, cudaStream_t s)
{
    constexpr int TILE = 256 * ITEMS;
    if (n == 0) {
        QE_CUDA(ctx, cudaMemsetAsync(out_count, 0, sizeof(int64_t), s));
        return QE_OK;
    }
    CompactCommon C;
    C.n = n;
    C.ntiles = qe_ceil_div(n, TILE);
    C.capacity = capacity;
    C.out_count = out_count;
    C.st = ctx->dstat;
    C.spin_limit = ctx->spin_limit;
    void *scratch = nullptr;
    size_t bytes = (static_cast<size_t>(C.ntiles) + 1) * sizeof(unsigned long long);
    qe_status st = qe_alloc(ctx, &scratch, bytes, s);
    if (st != QE_OK) return st;
    C.tile_counter = static_cast<unsigned long long *>(scratch);
    C.tile_state = C.tile_counter + 1;
    cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, s);
    if (e != cudaSuccess) {
        qe_free(ctx, scratch, s);
        return qe_cuda_fail(ctx, e, "cudaMemsetAsync(tile state)");
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_compact<ITEMS, Op>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(ctx->num_sms) * per_sm;
    if (grid > C.ntiles) grid = C.ntiles;
    {
        ProfScope prof(ctx, name, s);
        k_compact<ITEMS, Op><<<static_cast<unsigned>(grid), 256, 0, s>>>(C, op);
        QE_LAUNCHED(ctx);
    }
    e = cudaGetLastError();
    qe_free(ctx, scratch, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "k_compact launch");
    return QE_OK;
}

// ---------------------------------------------------------------------------
// Two-pass stable compaction for large inputs, with no dependency between
// blocks (so as many tiles are in flight as occupancy allows; the price is a
// second pass over the selection rows and the survivors kept by the first).  A warp segment is 32 lanes x ITEMS rows in
// the tile order above (item k of lane l is position seg*32*ITEMS + 32k + l).
// Pass 1 counts each segment's survivors and keeps what pass 2 needs: the
// survivor ballot of every item and, for ops with a payload (Op::kPay), each
// survivor's payload word; a two-level scan turns the counts into offsets
// (blocks of TP_SCAN_B counts, then at most 4 * 1024 block totals); pass 2
// reads the selection rows again, restores the survivors from the kept
// ballots and words (no second key gather or table lookup) and writes them
// item by item at the segment's offset.
constexpr int TP_SCAN_B = 4096;

template <int ITEMS, class Op>
__global__ void __launch_bounds__(256) k_tp_count(Op op, int64_t n, int64_t nseg, uint32_t *cnt, uint32_t *masks,
                                                 int32_t *words)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * 8;
    for (int64_t seg = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); seg < nseg; seg += warps) {
        const int64_t pos0 = seg * 32 * ITEMS + lane;
        bool ok[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) ok[k] = pos0 + 32 * k < n;
        typename Op::Pre pre;
        typename Op::Slot slot;
        op.load(pos0, ok, pre);
        op.eval(pos0, ok, pre, slot);
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const unsigned m = __ballot_sync(QE_FULL_MASK, ok[k]);
            c += __popc(m);
            if (lane == 0) masks[seg * ITEMS + k] = m;
            if constexpr (Op::kPay) {
                if (ok[k]) words[pos0 + 32 * k] = op.word(k, slot);
            }
        }
        if (lane == 0) cnt[seg] = c;
    }
}

// Each block of 1024 threads scans TP_SCAN_B counts into local offsets and
// writes its total.
static __global__ void __launch_bounds__(1024) k_tp_scan_local(const uint32_t *cnt, uint32_t *loc, int64_t nseg,
                                                        int64_t *bsum)
{
    __shared__ uint32_t s_w[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * TP_SCAN_B + 4 * t;
    uint32_t v[4], local = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        v[j] = base + j < nseg ? cnt[base + j] : 0u;
        local += v[j];
    }
    const uint32_t inc = warp_incl_scan(local);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = s_w[lane];
        const uint32_t wi = warp_incl_scan(w);
        s_w[lane] = wi - w;
        if (lane == 31) bsum[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = s_w[warp] + inc - local;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        if (base + j < nseg) loc[base + j] = run;
        run += v[j];
    }
}

// One block: exclusive scan of at most 4096 block totals in place, the total
// into out_count, capacity check.
static __global__ void __launch_bounds__(1024) k_tp_scan_top(int64_t *bsum, int nblk, int64_t *out_count, int64_t capacity,
                                                      qe_dev_status *st)
{
    __shared__ int64_t s_w[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int64_t v[4], local = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        v[j] = 4 * t + j < nblk ? bsum[4 * t + j] : 0;
        local += v[j];
    }
    const int64_t inc = warp_incl_scan(local);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int64_t w = s_w[lane];
        const int64_t wi = warp_incl_scan(w);
        s_w[lane] = wi - w;
    }
    __syncthreads();
    int64_t run = s_w[warp] + inc - local;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        if (4 * t + j < nblk) bsum[4 * t + j] = run;
        run += v[j];
    }
    if (t == 1023) {
        *out_count = run;
        if (run > capacity) dev_report(st, QE_ERR_CAPACITY, run);
    }
}

template <int ITEMS, class Op>
__global__ void __launch_bounds__(256) k_tp_write(Op op, int64_t n, int64_t nseg, const uint32_t *loc,
                                                 const int64_t *bsum, int64_t capacity, const uint32_t *masks,
                                                 const int32_t *words)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * 8;
    for (int64_t seg = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5); seg < nseg; seg += warps) {
        const int64_t pos0 = seg * 32 * ITEMS + lane;
        bool ok[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) ok[k] = pos0 + 32 * k < n;
        typename Op::Pre pre;
        typename Op::Slot slot;
        op.load(pos0, ok, pre);
        int32_t w[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            ok[k] = (masks[seg * ITEMS + k] >> lane) & 1u;
            w[k] = 0;
            if constexpr (Op::kPay) w[k] = ok[k] ? words[pos0 + 32 * k] : 0;
        }
        op.restore(pre, w, slot);
        int64_t pos = bsum[seg / TP_SCAN_B] + loc[seg];
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            const unsigned m = __ballot_sync(QE_FULL_MASK, ok[k]);
            if (ok[k]) {
                const int64_t o = pos + __popc(m & lt);
                if (o < capacity) op.emit(o, pos0 + 32 * k, k, slot);
            }
            pos += __popc(m);
        }
    }
}

// Host: scratch, the two passes and the scan.  nseg must not exceed
// 4 * 1024 * TP_SCAN_B.
template <int ITEMS, class Op>
qe_status launch_two_pass(qe_ctx *ctx, const char *name, int64_t n, int64_t capacity, int64_t *out_count,
                          const Op &op, cudaStream_t s)
{
    const int64_t nseg = qe_ceil_div(n, static_cast<int64_t>(32) * ITEMS);
    const int64_t nblk = qe_ceil_div(nseg, TP_SCAN_B);
    if (nblk > 4 * 1024) return qe_fail(ctx, QE_ERR_INVALID_ARG, std::string(name) + ": too many rows");
    void *scratch = nullptr;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t cnt_bytes = up(static_cast<size_t>(nseg) * 4), bs_bytes = up(static_cast<size_t>(nblk) * 8),
                 mask_bytes = up(static_cast<size_t>(nseg) * ITEMS * 4),
                 word_bytes = Op::kPay ? static_cast<size_t>(nseg) * ITEMS * 32 * 4 : 0;
    // counts, offsets, block sums, survivor ballots (4 bytes per 32 positions), payload words (4 per position)
    qe_status st = qe_alloc(ctx, &scratch, 2 * cnt_bytes + bs_bytes + mask_bytes + word_bytes, s);
    if (st != QE_OK) return st;
    char *p = static_cast<char *>(scratch);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(p);
    uint32_t *loc = reinterpret_cast<uint32_t *>(p + cnt_bytes);
    int64_t *bsum = reinterpret_cast<int64_t *>(p + 2 * cnt_bytes);
    uint32_t *masks = reinterpret_cast<uint32_t *>(p + 2 * cnt_bytes + bs_bytes);
    int32_t *words = Op::kPay ? reinterpret_cast<int32_t *>(p + 2 * cnt_bytes + bs_bytes + mask_bytes) : nullptr;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tp_write<ITEMS, Op>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = static_cast<int64_t>(ctx->num_sms) * per_sm;
    if (grid > qe_ceil_div(nseg, 8)) grid = qe_ceil_div(nseg, 8);
    cudaError_t e;
    {
        ProfScope prof(ctx, name, s);
        k_tp_count<ITEMS, Op><<<static_cast<unsigned>(grid), 256, 0, s>>>(op, n, nseg, cnt, masks, words);
        QE_LAUNCHED(ctx);
        k_tp_scan_local<<<static_cast<unsigned>(nblk), 1024, 0, s>>>(cnt, loc, nseg, bsum);
        QE_LAUNCHED(ctx);
        k_tp_scan_top<<<1, 1024, 0, s>>>(bsum, static_cast<int>(nblk), out_count, capacity, ctx->dstat);
        QE_LAUNCHED(ctx);
        k_tp_write<ITEMS, Op><<<static_cast<unsigned>(grid), 256, 0, s>>>(op, n, nseg, loc, bsum, capacity, masks,
                                                                          words);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    qe_free(ctx, scratch, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "two-pass compaction launch");
    return QE_OK;
}
