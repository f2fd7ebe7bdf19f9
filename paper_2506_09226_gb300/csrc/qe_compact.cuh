// qe_compact.cuh -- single-pass stable stream compaction.
//
// A tile is 256 threads x ITEMS rows.  Warp w of a tile owns 32*ITEMS
// consecutive positions; item k of lane l is position w*32*ITEMS + k*32 + l,
// so every column read is one 128-byte (int32) or 256-byte (int64) coalesced
// warp access and the natural row order is (warp, item, lane).  Survivors of
// item k are ranked inside the warp with one ballot, warps are ranked with a
// shared-memory scan, and tiles with the decoupled look-back; each survivor
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
//   struct Slot;                                      per-thread item data
//   __device__ void eval(int64_t pos0, bool (&ok)[ITEMS], Slot &s) const;
//        pos0 = this lane's first position (item k is pos0 + 32k); ok[k]
//        arrives true for in-range positions; eval clears non-survivors.
//   __device__ void emit(int64_t out_pos, int64_t pos, int k, const Slot &s) const;
template <int ITEMS, class Op>
__global__ void __launch_bounds__(256) k_compact(CompactCommon C, Op op)
{
    constexpr int TILE = 256 * ITEMS;
    __shared__ long long s_tile;
    __shared__ int s_wofs[8];
    __shared__ long long s_excl;
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
        typename Op::Slot slot;
        op.eval(pos0, ok, slot);
        unsigned mask[ITEMS];
        int wtotal = 0;
#pragma unroll
        for (int k = 0; k < ITEMS; k++) {
            mask[k] = __ballot_sync(QE_FULL_MASK, ok[k]);
            wtotal += __popc(mask[k]);
        }
        if (lane == 0) s_wofs[warp] = wtotal;
        __syncthreads();
        if (warp == 0) {
            int v = lane < 8 ? s_wofs[lane] : 0;
            int inc = warp_incl_scan(v);
            int tot = __shfl_sync(QE_FULL_MASK, inc, 7);
            int64_t excl = lb_exclusive(C.tile_state, tile, tot, C.st, C.spin_limit);
            if (lane < 8) s_wofs[lane] = inc - v;
            if (lane == 0) {
                s_excl = excl;
                if (tile == C.ntiles - 1) {
                    int64_t total = excl + tot;
                    *C.out_count = total;
                    if (total > C.capacity) dev_report(C.st, QE_ERR_CAPACITY, total);
                }
            }
        }
        __syncthreads();
        int64_t pos = s_excl + s_wofs[warp];
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
