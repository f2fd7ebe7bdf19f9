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
