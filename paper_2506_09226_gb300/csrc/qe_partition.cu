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
//   3. k_part_scatter  block b walks its rows in chunks of CHUNK in order.  A
//                      chunk is ranked stably by destination in shared memory
//                      (one or two LSD digit passes; within a warp equal digits
//                      are ranked with __match_any_sync, warps and digits with a
//                      block scan), staged in destination order, and written
//                      out so that consecutive lanes store consecutive rows of
//                      one destination.  Each block keeps a running output
//                      offset per destination, so rows keep their input order.
#include "qe_internal.cuh"

namespace {

constexpr int PT = 512;            // threads per block (16 warps)
constexpr int NW = PT / 32;
constexpr int P_ITEMS = 8;         // rows per thread per chunk
constexpr int CHUNK = PT * P_ITEMS;
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
    uint32_t *hist;           // [G][F]
    int64_t *off;             // [G][F]
    const int64_t *base;      // [F + 1] (= out_offsets)
};

__global__ void __launch_bounds__(PT) k_part_hist(PartArgs A)
{
    extern __shared__ uint32_t s_hist[];
    const int F = 1 << A.log2f;
    for (int p = threadIdx.x; p < F; p += PT) s_hist[p] = 0;
    __syncthreads();
    const int64_t lo = static_cast<int64_t>(blockIdx.x) * A.rows_per_block;
    const int64_t hi = min(A.n, lo + A.rows_per_block);
    for (int64_t c = lo; c < hi; c += CHUNK) {
        int64_t k[P_ITEMS];
#pragma unroll
        for (int i = 0; i < P_ITEMS; i++) {
            int64_t r = c + i * PT + threadIdx.x;
            k[i] = r < hi ? __ldcs(reinterpret_cast<const long long *>(A.keys) + r) : 0;
        }
#pragma unroll
        for (int i = 0; i < P_ITEMS; i++) {
            int64_t r = c + i * PT + threadIdx.x;
            if (r < hi) atomicAdd(&s_hist[dev_part_id(k[i], A.log2f, A.mode, A.shift)], 1u);
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < F; p += PT) A.hist[static_cast<int64_t>(blockIdx.x) * F + p] = s_hist[p];
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

// Block-wide exclusive scan, in place, of cnt[0..N) (uint16 counts, N a
// multiple of PT or smaller than PT), totals <= CHUNK.
__device__ __forceinline__ void block_excl_scan_u16(uint16_t *cnt, int N, int *s_w)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (N + PT - 1) / PT;
    int local = 0;
    for (int j = 0; j < per; j++) {
        int i = t * per + j;
        if (i < N) local += cnt[i];
    }
    int inc = warp_incl_scan(local);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NW ? s_w[lane] : 0;
        int wi = warp_incl_scan(w);
        if (lane < NW) s_w[lane] = wi - w;
    }
    __syncthreads();
    int run = s_w[warp] + inc - local;
    for (int j = 0; j < per; j++) {
        int i = t * per + j;
        if (i < N) {
            int c = cnt[i];
            cnt[i] = static_cast<uint16_t>(run);
            run += c;
        }
    }
    __syncthreads();
}

// Stable rank of chunk positions s < m by digit (pid_in[s] >> shift) & mask.
// Writes newpos[s] (rank) and pid_out[rank] = pid_in[s].  Items are
// warp-striped: warp w owns positions [w*32*P_ITEMS, (w+1)*32*P_ITEMS).
__device__ __forceinline__ void rank_pass(const uint16_t *pid_in, int m, int shift, int bits, uint16_t *cnt,
                                          uint16_t *newpos, uint16_t *pid_out, int *s_w)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    const int ndig = 1 << bits;
    const unsigned dmask = ndig - 1;
    for (int i = threadIdx.x; i < ndig * NW; i += PT) cnt[i] = 0;
    __syncthreads();
    uint16_t r[P_ITEMS];
    uint16_t dg[P_ITEMS];
#pragma unroll
    for (int k = 0; k < P_ITEMS; k++) {
        const int s = warp * 32 * P_ITEMS + k * 32 + lane;
        const bool valid = s < m;
        const unsigned d = valid ? ((pid_in[s] >> shift) & dmask) : 0xffffu;
        const unsigned peers = __match_any_sync(QE_FULL_MASK, d);
        int basec = 0;
        if (valid) basec = cnt[d * NW + warp];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[d * NW + warp] = static_cast<uint16_t>(basec + __popc(peers));
        __syncwarp();
        r[k] = static_cast<uint16_t>(basec + __popc(peers & lt));
        dg[k] = static_cast<uint16_t>(d);
    }
    __syncthreads();
    block_excl_scan_u16(cnt, ndig * NW, s_w);
#pragma unroll
    for (int k = 0; k < P_ITEMS; k++) {
        const int s = warp * 32 * P_ITEMS + k * 32 + lane;
        if (s < m) {
            int t = cnt[dg[k] * NW + warp] + r[k];
            newpos[s] = static_cast<uint16_t>(t);
            pid_out[t] = pid_in[s];
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
__global__ void __launch_bounds__(PT) k_part_scatter(PartArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int F = 1 << A.log2f;
    // layout: run[F] i64 | skey[CHUNK] i64 | spay[CHUNK] i64 (FAST) or
    //         srow[CHUNK] u16 (generic) | start[F] u16 |
    //         pidA, pidB, pos1, pos2 [CHUNK] u16 | cnt[256*NW] u16
    int64_t *run = reinterpret_cast<int64_t *>(smem);
    int64_t *skey = run + F;
    int64_t *spay = skey + CHUNK;
    uint16_t *srow = reinterpret_cast<uint16_t *>(spay);
    uint16_t *start = reinterpret_cast<uint16_t *>(spay + CHUNK);
    uint16_t *pidA = start + F;
    uint16_t *pidB = pidA + CHUNK;
    uint16_t *pos1 = pidB + CHUNK;
    uint16_t *pos2 = pos1 + CHUNK;
    uint16_t *cnt = pos2 + CHUNK;
    __shared__ int s_w[NW];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    for (int p = threadIdx.x; p < F; p += PT) run[p] = A.base[p] + A.off[static_cast<int64_t>(b) * F + p];
    // digit plan: one pass for F <= 256, else two passes of ceil(log2f / 2) bits
    const int passes = A.log2f == 0 ? 0 : (A.log2f <= 8 ? 1 : 2);
    const int bits1 = passes == 2 ? (A.log2f + 1) / 2 : A.log2f;
    const int bits2 = A.log2f - bits1;
    __syncthreads();

    const int64_t lo = static_cast<int64_t>(b) * A.rows_per_block;
    const int64_t hi = min(A.n, lo + A.rows_per_block);
    for (int64_t c = lo; c < hi; c += CHUNK) {
        const int m = static_cast<int>(hi - c < CHUNK ? hi - c : CHUNK);
        int64_t key[P_ITEMS], pay[P_ITEMS];
#pragma unroll
        for (int k = 0; k < P_ITEMS; k++) {
            const int s = warp * 32 * P_ITEMS + k * 32 + lane;
            key[k] = s < m ? __ldcs(reinterpret_cast<const long long *>(A.keys) + c + s) : 0;
            if (FAST) pay[k] = s < m ? __ldcs(static_cast<const long long *>(A.pay[0]) + c + s) : 0;
        }
#pragma unroll
        for (int k = 0; k < P_ITEMS; k++) {
            const int s = warp * 32 * P_ITEMS + k * 32 + lane;
            if (s < m) pidA[s] = static_cast<uint16_t>(dev_part_id(key[k], A.log2f, A.mode, A.shift));
        }
        __syncthreads();
        const uint16_t *pidS = pidA;
        if (passes >= 1) {
            rank_pass(pidA, m, 0, bits1, cnt, pos1, pidB, s_w);
            pidS = pidB;
        }
        if (passes == 2) {
            rank_pass(pidB, m, bits1, bits2, cnt, pos2, pidA, s_w);
            pidS = pidA;
        }
        // stage rows in destination order (generic path: the source row)
#pragma unroll
        for (int k = 0; k < P_ITEMS; k++) {
            const int s = warp * 32 * P_ITEMS + k * 32 + lane;
            if (s < m) {
                int t = s;
                if (passes >= 1) t = pos1[t];
                if (passes == 2) t = pos2[t];
                skey[t] = key[k];
                if (FAST) spay[t] = pay[k];
                else srow[t] = static_cast<uint16_t>(s);
            }
        }
        __syncthreads();
        // run starts (positions where the destination changes)
        for (int s = threadIdx.x; s < m; s += PT) {
            uint16_t p = pidS[s];
            if (s == 0 || pidS[s - 1] != p) start[p] = static_cast<uint16_t>(s);
        }
        __syncthreads();
        for (int s = threadIdx.x; s < m; s += PT) {
            const uint16_t p = pidS[s];
            const int64_t d = run[p] + (s - start[p]);
            __stcs(reinterpret_cast<long long *>(A.out_keys) + d, skey[s]);
            if (FAST) {
                __stcs(static_cast<long long *>(A.out_pay[0]) + d, spay[s]);
            } else {
                const int64_t src = c + srow[s];
                for (int j = 0; j < A.npay; j++) copy_elem(A.out_pay[j], A.pay[j], A.pay_type[j], d, src);
            }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < m; s += PT) {
            const uint16_t p = pidS[s];
            if (s == m - 1 || pidS[s + 1] != p) run[p] += s - start[p] + 1;
        }
        __syncthreads();
    }
}

size_t scatter_smem(int log2f, bool fast)
{
    const size_t F = size_t(1) << log2f;
    (void)fast;
    return F * 8 + CHUNK * 8 + CHUNK * 8 + F * 2 + 4 * CHUNK * 2 + 256 * NW * 2;
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
    A.rows_per_block = qe_ceil_div(nrows, G);
    G = qe_ceil_div(nrows, A.rows_per_block);

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

    cudaError_t e = cudaSuccess;
    {
        ProfScope prof(ctx, "part_hist", s);
        k_part_hist<<<static_cast<unsigned>(G), PT, F * sizeof(uint32_t), s>>>(A);
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
