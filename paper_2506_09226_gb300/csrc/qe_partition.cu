// qe_partition.cu -- stable radix / hash partition with per-destination
// offsets (Sec. 2.2, Fig. 1; Sec. 2.3: one contiguous run per destination in
// each column, located by a start offset).
//
// Three steps over G blocks, block b owning the contiguous input rows
// [b*R, (b+1)*R):
//   1. k_part_hist     per-block histogram of destinations (shared-memory
//                      atomics), written as hist[b][p];
//   2. k_part_colscan / k_part_basescan
//                      off[b][p] = sum over earlier blocks of hist[.][p] and
//                      base[p] = sum over earlier destinations of all rows, so
//                      block b's rows for p start at base[p] + off[b][p];
//   3. k_part_scatter  block b walks its rows in chunks of CHUNK in order.  The
//                      next chunk's keys (and an int64 payload) are copied into
//                      shared memory with bulk TMA copies while the current one
//                      is processed (double buffer, mbarrier completion).  A
//                      chunk is ranked stably by destination in shared memory
//                      (one or two LSD digit passes; within a warp equal digits
//                      are ranked with __match_any_sync, warps and digits with a
//                      block scan); rows are then written in destination order
//                      through the inverse permutation, so consecutive lanes
//                      store consecutive rows of one destination.  Each block
//                      keeps a running output offset per destination, so rows
//                      keep their input order.
#include "qe_pipe_core.cuh"

namespace {

constexpr int PT = 1024;           // scatter threads per block (32 warps), one block per SM
constexpr int NW = PT / 32;
constexpr int P_ITEMS = 4;         // rows per thread per chunk
constexpr int CHUNK = PT * P_ITEMS;
constexpr int HT = 1024;           // histogram threads per block
constexpr int H_ITEMS = 8;
constexpr int H_SPLIT = 4;         // histogram blocks per scatter block
constexpr int MAX_PAY = QE_MAX_COLS - 1;

struct PartArgs {
    const int64_t *keys;
    int64_t n;
    int64_t rows_per_block;   // R
    int log2f, mode, shift;
    int npay;
    const void *pay[MAX_PAY];
    int32_t pay_type[MAX_PAY];
    int64_t *out_keys;
    void *out_pay[MAX_PAY];
    uint32_t *hist;           // [G][F], zeroed
    int64_t *off;             // [G][F]
    const int64_t *base;      // [F + 1] (= out_offsets)
    int tma;                  // keys (and the int64 payload) are 16-byte aligned
    int64_t spin_limit;
    qe_dev_status *st;
};

// Histogram of destinations; H_SPLIT blocks share each scatter block's range
// and add their counts into hist[b][p].
__global__ void __launch_bounds__(HT) k_part_hist(PartArgs A)
{
    extern __shared__ uint32_t s_hist[];
    const int F = 1 << A.log2f;
    for (int p = threadIdx.x; p < F; p += HT) s_hist[p] = 0;
    __syncthreads();
    const int b = blockIdx.x / H_SPLIT, k = blockIdx.x % H_SPLIT;
    const int64_t blo = static_cast<int64_t>(b) * A.rows_per_block;
    const int64_t bhi = min(A.n, blo + A.rows_per_block);
    const int64_t sub = (A.rows_per_block + H_SPLIT - 1) / H_SPLIT;
    const int64_t lo = blo + k * sub;
    const int64_t hi = min(bhi, lo + sub);
    for (int64_t c = lo; c < hi; c += static_cast<int64_t>(HT) * H_ITEMS) {
        int64_t key[H_ITEMS];
#pragma unroll
        for (int i = 0; i < H_ITEMS; i++) {
            const int64_t r = c + i * HT + threadIdx.x;
            key[i] = r < hi ? __ldcs(reinterpret_cast<const long long *>(A.keys) + r) : 0;
        }
#pragma unroll
        for (int i = 0; i < H_ITEMS; i++) {
            const int64_t r = c + i * HT + threadIdx.x;
            if (r < hi) atomicAdd(&s_hist[dev_part_id(key[i], A.log2f, A.mode, A.shift)], 1u);
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < F; p += HT) {
        const uint32_t c = s_hist[p];
        if (c) atomicAdd(A.hist + static_cast<int64_t>(b) * F + p, c);
    }
}

// One thread per destination p: prefix of hist[.][p] over blocks.
__global__ void k_part_colscan(const uint32_t *hist, int64_t *off, int64_t *tot, int G, int F)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= F) return;
    int64_t run = 0;
    for (int b = 0; b < G; b++) {
        int64_t idx = static_cast<int64_t>(b) * F + p;
        uint32_t h = hist[idx];
        off[idx] = run;
        run += h;
    }
    tot[p] = run;
}

// One block: exclusive scan of the per-destination totals (F <= 4096).
__global__ void __launch_bounds__(1024) k_part_basescan(const int64_t *tot, int64_t *out_offsets, int F, int64_t n)
{
    __shared__ int64_t s_w[32];
    const int per = (F + 1023) / 1024;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int64_t v[4] = {0, 0, 0, 0};
    int64_t local = 0;
    for (int j = 0; j < per; j++) {
        int p = t * per + j;
        v[j] = p < F ? tot[p] : 0;
        local += v[j];
    }
    int64_t inc = warp_incl_scan(local);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = s_w[lane];
        int64_t wi = warp_incl_scan(w);
        s_w[lane] = wi - w;
    }
    __syncthreads();
    int64_t run = s_w[warp] + inc - local;
    for (int j = 0; j < per; j++) {
        int p = t * per + j;
        if (p < F) out_offsets[p] = run;
        run += v[j];
    }
    if (t == 0) out_offsets[F] = n;
}

// Digit counters: cnt[d * CSTRIDE + w] (uint32) for digit d and warp w.  The
// odd stride puts different digits of one warp in different banks.
constexpr int CSTRIDE = NW + 1;

// Block-wide exclusive scan, in place, of the counters in digit-major order
// (d, then w) over ndig digits.  Totals are at most CHUNK.
__device__ __forceinline__ void block_excl_scan_cnt(uint32_t *cnt, int ndig, int *s_w)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int N = ndig * NW;
    const int per = (N + PT - 1) / PT;
    uint32_t local = 0;
    for (int j = 0; j < per; j++) {
        const int i = t * per + j;
        if (i < N) local += cnt[(i / NW) * CSTRIDE + (i % NW)];
    }
    const uint32_t inc = warp_incl_scan(local);
    if (lane == 31) s_w[warp] = static_cast<int>(inc);
    __syncthreads();
    if (warp == 0) {
        const int w = lane < NW ? s_w[lane] : 0;
        const int wi = warp_incl_scan(w);
        if (lane < NW) s_w[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = static_cast<uint32_t>(s_w[warp]) + inc - local;
    for (int j = 0; j < per; j++) {
        const int i = t * per + j;
        if (i < N) {
            uint32_t *c = cnt + (i / NW) * CSTRIDE + (i % NW);
            const uint32_t v = *c;
            *c = run;
            run += v;
        }
    }
    __syncthreads();
}

// Stable rank of the chunk's m packed words (destination << 12 | source row)
// by the digit (destination >> shift) & (2^bits - 1): in[s] moves to out[rank].
// Items are warp-striped: warp w owns positions [w*32*P_ITEMS, (w+1)*32*P_ITEMS),
// so the natural order is (warp, item, lane).
__device__ __forceinline__ void rank_pass(const uint32_t *in, uint32_t *out, int m, int shift, int bits, uint32_t *cnt,
                                          int *s_w)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    const int ndig = 1 << bits;
    const unsigned dmask = ndig - 1;
    for (int i = threadIdx.x; i < ndig * CSTRIDE; i += PT) cnt[i] = 0;
    __syncthreads();
    uint32_t wv[P_ITEMS], r[P_ITEMS];
#pragma unroll
    for (int k = 0; k < P_ITEMS; k++) {
        const int s2 = warp * 32 * P_ITEMS + k * 32 + lane;
        const bool valid = s2 < m;
        wv[k] = valid ? in[s2] : 0;
        const unsigned d = valid ? ((wv[k] >> (12 + shift)) & dmask) : 0xffffu;
        const unsigned peers = __match_any_sync(QE_FULL_MASK, d);
        uint32_t basec = 0;
        if (valid) basec = cnt[d * CSTRIDE + warp];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[d * CSTRIDE + warp] = basec + __popc(peers);
        __syncwarp();
        r[k] = basec + __popc(peers & lt);
    }
    __syncthreads();
    block_excl_scan_cnt(cnt, ndig, s_w);
#pragma unroll
    for (int k = 0; k < P_ITEMS; k++) {
        const int s2 = warp * 32 * P_ITEMS + k * 32 + lane;
        if (s2 < m) {
            const unsigned d = (wv[k] >> (12 + shift)) & dmask;
            out[cnt[d * CSTRIDE + warp] + r[k]] = wv[k];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void copy_elem(void *dst, const void *src, int type, int64_t d, int64_t s)
{
    if (type == QE_I64)
        static_cast<long long *>(dst)[d] = __ldg(static_cast<const long long *>(src) + s);
    else if (type == QE_I32)
        static_cast<int32_t *>(dst)[d] = __ldg(static_cast<const int32_t *>(src) + s);
    else
        static_cast<signed char *>(dst)[d] = __ldg(static_cast<const signed char *>(src) + s);
}

// FAST: exactly one int64 payload column, staged in shared memory with the
// keys.  Otherwise payload columns are gathered by chunk-local source row.
template <bool FAST>
__global__ void __launch_bounds__(PT, 1) k_part_scatter(PartArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ int s_w[NW];
    __shared__ int s_abort;
    const int F = 1 << A.log2f;
    // layout: bufK[2][CHUNK] i64 | bufP[2][CHUNK] i64 (FAST) | run[F] i64 |
    //         wA, wB [CHUNK] u32 (destination << 12 | source row) | start[F] u16 |
    //         cnt[64 * CSTRIDE] u32
    int64_t *bufK = reinterpret_cast<int64_t *>(smem);
    int64_t *bufP = bufK + 2 * CHUNK;
    int64_t *run = FAST ? bufP + 2 * CHUNK : bufP;
    uint32_t *wA = reinterpret_cast<uint32_t *>(run + F);
    uint32_t *wB = wA + CHUNK;
    uint32_t *cnt = wB + CHUNK;
    uint16_t *start = reinterpret_cast<uint16_t *>(cnt + 64 * CSTRIDE);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    const int64_t lo = static_cast<int64_t>(b) * A.rows_per_block;
    const int64_t hi = min(A.n, lo + A.rows_per_block);
    const int64_t nch = (hi - lo + CHUNK - 1) / CHUNK;
    for (int p = threadIdx.x; p < F; p += PT) run[p] = A.base[p] + A.off[static_cast<int64_t>(b) * F + p];
    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_fence_init();
    }
    const int passes = A.log2f == 0 ? 0 : (A.log2f <= 6 ? 1 : 2);
    const int bits1 = passes == 2 ? (A.log2f + 1) / 2 : A.log2f;
    const int bits2 = A.log2f - bits1;
    __syncthreads();
    const uint64_t pol = l2_evict_first_policy();

    // chunk c: rows [lo + c*CHUNK, ...) into buffer c & 1
    auto issue = [&](int64_t c) {
        const int64_t r0 = lo + c * CHUNK;
        const int m = static_cast<int>(hi - r0 < CHUNK ? hi - r0 : CHUNK);
        const int mc = A.tma ? (m & ~1) : 0;      // 16-byte multiple
        unsigned long long *bar = &s_bar[c & 1];
        const uint32_t bytes = static_cast<uint32_t>(mc) * 8u * (FAST ? 2u : 1u);
        if (bytes) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, bytes);
            tma_load_1d(bufK + (c & 1) * CHUNK, A.keys + r0, mc * 8u, bar, pol);
            if (FAST) tma_load_1d(bufP + (c & 1) * CHUNK, static_cast<const long long *>(A.pay[0]) + r0, mc * 8u, bar, pol);
        } else {
            mbar_arrive(bar);
        }
    };
    if (threadIdx.x == 0 && nch > 0) issue(0);

    for (int64_t c = 0; c < nch; c++) {
        if (threadIdx.x == 0 && c + 1 < nch) issue(c + 1);
        const int64_t r0 = lo + c * CHUNK;
        const int m = static_cast<int>(hi - r0 < CHUNK ? hi - r0 : CHUNK);
        const int mc = A.tma ? (m & ~1) : 0;
        int64_t *keys = bufK + (c & 1) * CHUNK;
        int64_t *pays = bufP + (c & 1) * CHUNK;
        if (!mbar_wait(&s_bar[c & 1], static_cast<uint32_t>((c >> 1) & 1), A.spin_limit)) {
            if (threadIdx.x == 0) dev_report(A.st, QE_ERR_TIMEOUT, 0);
            s_abort = 1;
        }
        // rows the bulk copy did not cover (unaligned columns, odd tail)
        for (int s2 = mc + threadIdx.x; s2 < m; s2 += PT) {
            keys[s2] = A.keys[r0 + s2];
            if (FAST) pays[s2] = static_cast<const long long *>(A.pay[0])[r0 + s2];
        }
        __syncthreads();
        if (s_abort) break;
#pragma unroll
        for (int k = 0; k < P_ITEMS; k++) {
            const int s2 = warp * 32 * P_ITEMS + k * 32 + lane;
            if (s2 < m) wA[s2] = (dev_part_id(keys[s2], A.log2f, A.mode, A.shift) << 12) | static_cast<uint32_t>(s2);
        }
        __syncthreads();
        const uint32_t *sorted = wA;
        if (passes >= 1) {
            rank_pass(wA, wB, m, 0, bits1, cnt, s_w);
            sorted = wB;
        }
        if (passes == 2) {
            rank_pass(wB, wA, m, bits1, bits2, cnt, s_w);
            sorted = wA;
        }
        // run starts (positions where the destination changes)
        for (int t = threadIdx.x; t < m; t += PT) {
            const uint32_t p = sorted[t] >> 12;
            if (t == 0 || (sorted[t - 1] >> 12) != p) start[p] = static_cast<uint16_t>(t);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += PT) {
            const uint32_t w = sorted[t];
            const uint32_t p = w >> 12;
            const int src = static_cast<int>(w & 0xfffu);
            const int64_t d = run[p] + (t - start[p]);
            __stcs(reinterpret_cast<long long *>(A.out_keys) + d, keys[src]);
            if (FAST) {
                __stcs(static_cast<long long *>(A.out_pay[0]) + d, pays[src]);
            } else {
                for (int j = 0; j < A.npay; j++) copy_elem(A.out_pay[j], A.pay[j], A.pay_type[j], d, r0 + src);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += PT) {
            const uint32_t p = sorted[t] >> 12;
            if (t == m - 1 || (sorted[t + 1] >> 12) != p) run[p] += t - start[p] + 1;
        }
        __syncthreads();
    }
    if (s_abort && threadIdx.x == 0) {
        // let copies still in flight land before the block exits (bounded)
        mbar_wait(&s_bar[0], 0, A.spin_limit);
        mbar_wait(&s_bar[1], 0, A.spin_limit);
    }
}

size_t scatter_smem(int log2f, bool fast)
{
    const size_t F = size_t(1) << log2f;
    return 2 * CHUNK * 8 * (fast ? 2 : 1) + F * 8 + 2 * CHUNK * 4 + 64 * CSTRIDE * 4 + F * 2;
}

}  // namespace

extern "C" qe_status qe_partition(qe_ctx *ctx, const int64_t *keys, const qe_col *payload, int npayload,
                                  int64_t nrows, int log2_fanout, int mode, int shift, int64_t *out_keys,
                                  void *const *out_payload, int64_t *out_offsets, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nrows < 0 || log2_fanout < 0 || log2_fanout > 12 || (mode != QE_PART_HASH && mode != QE_PART_RADIX) ||
        shift < 0 || shift > 63 || npayload < 0 || npayload > MAX_PAY || !out_offsets)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "partition: bad argument");
    if (nrows > 0 && (!keys || !out_keys || !qe_aligned(keys, 8) || !qe_aligned(out_keys, 8)))
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "partition: bad key column");
    PartArgs A{};
    A.keys = keys;
    A.n = nrows;
    A.log2f = log2_fanout;
    A.mode = mode;
    A.shift = shift;
    A.npay = npayload;
    A.out_keys = out_keys;
    for (int j = 0; j < npayload; j++) {
        const qe_col &c = payload[j];
        if (!qe_valid_type(c.type) || c.gather || (nrows > 0 && (!c.data || !out_payload || !out_payload[j])) ||
            !qe_aligned(c.data, c.type) || !qe_aligned(out_payload[j], c.type))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "partition: bad payload column");
        A.pay[j] = c.data;
        A.pay_type[j] = c.type;
        A.out_pay[j] = out_payload[j];
    }
    const int F = 1 << log2_fanout;
    cudaSetDevice(ctx->device);
    if (nrows == 0) {
        QE_CUDA(ctx, cudaMemsetAsync(out_offsets, 0, (F + 1) * sizeof(int64_t), s));
        return QE_OK;
    }
    const bool fast = npayload == 1 && A.pay_type[0] == QE_I64 && qe_aligned(A.pay[0], 8);
    const size_t smem = scatter_smem(log2_fanout, fast);
    if (smem > ctx->smem_optin) return qe_fail(ctx, QE_ERR_INVALID_ARG, "partition: fan-out too large");
    auto kscatter = fast ? k_part_scatter<true> : k_part_scatter<false>;
    QE_CUDA(ctx, cudaFuncSetAttribute(kscatter, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    QE_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kscatter, PT, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t G = static_cast<int64_t>(ctx->num_sms) * per_sm;
    int64_t need = qe_ceil_div(nrows, CHUNK);
    if (G > need) G = need;
    // whole chunks per block, so every chunk but the last starts 32 KB-aligned
    A.rows_per_block = qe_ceil_div(qe_ceil_div(nrows, G), CHUNK) * CHUNK;
    G = qe_ceil_div(nrows, A.rows_per_block);
    A.tma = qe_aligned(keys, 16) && (!fast || qe_aligned(A.pay[0], 16));
    A.spin_limit = ctx->spin_limit;
    A.st = ctx->dstat;

    void *scratch = nullptr;
    const size_t hist_bytes = static_cast<size_t>(G) * F * sizeof(uint32_t);
    const size_t off_bytes = static_cast<size_t>(G) * F * sizeof(int64_t);
    const size_t tot_bytes = static_cast<size_t>(F) * sizeof(int64_t);
    qe_status st = qe_alloc(ctx, &scratch, hist_bytes + off_bytes + tot_bytes + 64, s);
    if (st != QE_OK) return st;
    unsigned char *sp = static_cast<unsigned char *>(scratch);
    A.off = reinterpret_cast<int64_t *>(sp);
    int64_t *tot = reinterpret_cast<int64_t *>(sp + off_bytes);
    A.hist = reinterpret_cast<uint32_t *>(sp + off_bytes + tot_bytes);
    A.base = out_offsets;

    cudaError_t e = cudaMemsetAsync(A.hist, 0, hist_bytes, s);
    if (e == cudaSuccess) {
        ProfScope prof(ctx, "part_hist", s);
        k_part_hist<<<static_cast<unsigned>(G * H_SPLIT), HT, F * sizeof(uint32_t), s>>>(A);
        QE_LAUNCHED(ctx);
    }
    if ((e = cudaGetLastError()) == cudaSuccess) {
        k_part_colscan<<<(F + 255) / 256, 256, 0, s>>>(A.hist, A.off, tot, static_cast<int>(G), F);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_part_basescan<<<1, 1024, 0, s>>>(tot, out_offsets, F, nrows);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ProfScope prof(ctx, "part_scatter", s);
        kscatter<<<static_cast<unsigned>(G), PT, smem, s>>>(A);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    qe_free(ctx, scratch, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "partition launch");
    return QE_OK;
}
