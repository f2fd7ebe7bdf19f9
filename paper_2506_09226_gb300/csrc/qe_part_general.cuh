// qe_part_general.cuh -- the general scatter of qe_partition, included once per
// block size: the including namespace defines PT (threads per block) and
// EVICT_LAST (the L2 policy of the output stores).
// No include guard: each inclusion instantiates the kernel in its own namespace.

constexpr int NW = PT / 32;
constexpr int P_ITEMS = 4;               // rows per thread per chunk
constexpr int CHUNK = PT * P_ITEMS;      // a chunk position fits the low 12 bits of a ranking word
static_assert(CHUNK <= 4096, "chunk positions must fit 12 bits");


__device__ __forceinline__ uint64_t l2_evict_last_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Output store of the general scatter.  With EVICT_LAST (set by the
// including namespace) the short per-destination runs are kept in L2 until
// the neighbouring rows of the same sector arrive; measured on GB300 this
// helps the 512-thread shape at the largest fan-outs and hurts the
// 1024-thread one.
__device__ __forceinline__ void out_store(long long *p, long long v, uint64_t pol)
{
    if (EVICT_LAST)
        asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
    else
        *p = v;
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

// Block-wide exclusive scan of a[0..N) (uint32) into out[0..N).
__device__ __forceinline__ void block_excl_scan_u32(const uint32_t *a, uint32_t *out, int N, int *s_w)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (N + PT - 1) / PT;
    uint32_t local = 0;
    for (int j = 0; j < per; j++) {
        const int i = t * per + j;
        if (i < N) local += a[i];
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
            out[i] = run;
            run += a[i];
        }
    }
}

// Stable rank of the chunk's packed words (destination << 12 | position),
// held by the threads in registers (warp-striped positions: warp w owns
// [w*32*P_ITEMS, (w+1)*32*P_ITEMS), natural order (warp, item, lane)), by the
// digit (destination >> shift) & (2^bits - 1): word moves to out[rank].
// Within a warp equal digits are ranked with __match_any_sync; warps and
// digits with a block scan of the counters.
__device__ __forceinline__ void rank_words(const uint32_t (&wv)[P_ITEMS], const bool (&valid)[P_ITEMS],
                                           uint32_t *out, int shift, int bits, uint32_t *cnt, int *s_w)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    const int ndig = 1 << bits;
    const unsigned dmask = ndig - 1;
    for (int i = threadIdx.x; i < ndig * CSTRIDE; i += PT) cnt[i] = 0;
    __syncthreads();
    uint32_t r[P_ITEMS];
#pragma unroll
    for (int k = 0; k < P_ITEMS; k++) {
        const unsigned d = valid[k] ? ((wv[k] >> (12 + shift)) & dmask) : 0xffffu;
        const unsigned peers = __match_any_sync(QE_FULL_MASK, d);
        uint32_t basec = 0;
        if (valid[k]) basec = cnt[d * CSTRIDE + warp];
        __syncwarp();
        if (valid[k] && lane == __ffs(peers) - 1) cnt[d * CSTRIDE + warp] = basec + __popc(peers);
        __syncwarp();
        r[k] = basec + __popc(peers & lt);
    }
    __syncthreads();
    block_excl_scan_cnt(cnt, ndig, s_w);
#pragma unroll
    for (int k = 0; k < P_ITEMS; k++)
        if (valid[k]) out[cnt[((wv[k] >> (12 + shift)) & dmask) * CSTRIDE + warp] + r[k]] = wv[k];
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
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ int s_w[NW];
    __shared__ int s_abort;
    const int F = 1 << A.log2f;
    // layout: bufK[2][CHUNK] i64 | bufP[2][CHUNK] i64 (FAST) | run[F] i64 |
    //         wA, wB [CHUNK] u32 | hist[F], start[F] u32 | cnt[64 * CSTRIDE] u32
    int64_t *bufK = reinterpret_cast<int64_t *>(smem);
    int64_t *bufP = bufK + 2 * CHUNK;
    int64_t *run = FAST ? bufP + 2 * CHUNK : bufP;
    uint32_t *wA = reinterpret_cast<uint32_t *>(run + F);
    uint32_t *wB = wA + CHUNK;
    uint32_t *hist = wB + CHUNK;
    uint32_t *start = hist + F;
    uint32_t *cnt = start + F;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x;
    const int64_t lo = static_cast<int64_t>(b) * A.rows_per_block;
    const int64_t hi = min(A.n, lo + A.rows_per_block);
    const int64_t nch = (hi - lo + CHUNK - 1) / CHUNK;
    for (int p = threadIdx.x; p < F; p += PT) {
        run[p] = A.base[p] + A.off[static_cast<int64_t>(b) * F + p];
        hist[p] = 0;
    }
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
    const uint64_t wpol = l2_evict_last_policy();

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
        // destinations, chunk histogram and the first ranking pass, in registers
        uint32_t wv[P_ITEMS];
        bool valid[P_ITEMS];
#pragma unroll
        for (int k = 0; k < P_ITEMS; k++) {
            const int s2 = warp * 32 * P_ITEMS + k * 32 + lane;
            valid[k] = s2 < m;
            const uint32_t p = valid[k] ? dev_part_id(keys[s2], A.log2f, A.mode, A.shift) : 0;
            wv[k] = (p << 12) | static_cast<uint32_t>(s2);
            if (valid[k]) atomicAdd(hist + p, 1u);
        }
        if (passes == 0) {
#pragma unroll
            for (int k = 0; k < P_ITEMS; k++)
                if (valid[k]) wA[wv[k] & 0xfffu] = wv[k];
            __syncthreads();
        } else if (passes == 1) {
            rank_words(wv, valid, wA, 0, bits1, cnt, s_w);
        } else {
            rank_words(wv, valid, wB, 0, bits1, cnt, s_w);
#pragma unroll
            for (int k = 0; k < P_ITEMS; k++) {
                const int s2 = warp * 32 * P_ITEMS + k * 32 + lane;
                wv[k] = valid[k] ? wB[s2] : 0;
            }
            rank_words(wv, valid, wA, bits1, bits2, cnt, s_w);
        }
        // start of each destination's run in the sorted chunk; bias the
        // running output offsets so that row t of the chunk goes to run[p] + t
        block_excl_scan_u32(hist, start, F, s_w);
        __syncthreads();
        for (int p = threadIdx.x; p < F; p += PT) run[p] -= start[p];
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += PT) {
            const uint32_t w = wA[t];
            const int src = static_cast<int>(w & 0xfffu);
            const int64_t d = run[w >> 12] + t;
            if (!QE_DCHECK(A.st, d >= 0 && d < A.n, d)) continue;
            out_store(reinterpret_cast<long long *>(A.out_keys) + d, keys[src], wpol);
            if (FAST) {
                out_store(static_cast<long long *>(A.out_pay[0]) + d, pays[src], wpol);
            } else {
                for (int j = 0; j < A.npay; j++) copy_elem(A.out_pay[j], A.pay[j], A.pay_type[j], d, r0 + src);
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < F; p += PT) {
            run[p] += start[p] + hist[p];
            hist[p] = 0;
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
    return 2 * CHUNK * 8 * (fast ? 2 : 1) + F * 8 + 2 * CHUNK * 4 + 2 * F * 4 + 64 * CSTRIDE * 4;
}

