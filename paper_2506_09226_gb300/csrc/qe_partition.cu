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
//   3. scatter        block b walks its rows in chunks, in order, ranks each
//                      chunk stably by destination in shared memory and writes
//                      the rows in destination order, keeping a running output
//                      offset per destination so rows keep their input order.
//                      Two kernels:
//                      k_part_scatter_sf (one int64 payload or none, at most
//                        64 digits a launch: F <= 64 in one pass, F = 128 ..
//                        4096 in two passes): each chunk's successor fetched
//                        into L2 and loaded into registers while the chunk is
//                        processed, one-pass ranking with ballots and
//                        per-warp counts, and write-combining of 32-byte
//                        sectors (see below);
//                      k_part_scatter (qe_part_general.cuh; any payloads, any
//                        fan-out): bulk-copy (TMA) double-buffered chunks and
//                        a one- or two-digit LSD ranking.
#include "qe_internal.cuh"
#include "qe_tma.cuh"

namespace {

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
    // Write-combining scatter only: which digit of the destination it sorts
    // by, and where its work items and their output offsets come from.
    int dshift;               // digit = (destination >> dshift) & dmask
    uint32_t dmask;
    int omode;                // WC_SINGLE, WC_PASS1 or WC_PASS2
    int sub_bits;             // two passes: bits of the second-pass digit
    int64_t nitems;           // work items (WC_SINGLE / WC_PASS1: one per block range)
    int g1;                   // two passes: first-pass block ranges
    int span;                 // two passes: first-pass ranges per second-pass item
    const int64_t *t1;        // two passes: [g1][F1] first-pass start of (range, digit)
    const uint32_t *h1;       // two passes: [g1][F1] rows of (range, digit)
};

// Work items of the write-combining scatter.
enum : int {
    WC_SINGLE = 0,  // one pass: item b = input range b, digit = destination
    WC_PASS1 = 1,   // first of two passes: item b = input range b, digit = the
                    // destination's high bits, output = scratch at t1[b][digit]
    WC_PASS2 = 2,   // second pass: item (q, b) = the scratch rows of input
                    // range b with high bits q, digit = the low bits
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

// One thread per destination p: prefix of hist[.][p] over blocks, sixteen
// blocks' counts loaded at a time so that their loads overlap.
__global__ void k_part_colscan(const uint32_t *hist, int64_t *off, int64_t *tot, int G, int F)
{
    constexpr int B = 16;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= F) return;
    int64_t run = 0;
    for (int b0 = 0; b0 < G; b0 += B) {
        uint32_t h[B];
#pragma unroll
        for (int j = 0; j < B; j++) h[j] = b0 + j < G ? hist[static_cast<int64_t>(b0 + j) * F + p] : 0u;
#pragma unroll
        for (int j = 0; j < B; j++) {
            if (b0 + j < G) off[static_cast<int64_t>(b0 + j) * F + p] = run;
            run += h[j];
        }
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

// ---------------------------------------------------------------------------
// Write-combining scatter (k_part_scatter_sf below): int64 keys with no
// payload or one int64 payload.  A block walks its rows in chunks of T * IT.
//
// Ranking is one pass: each warp counts destinations (equal destinations
// within a warp found with bit-wise ballots, in lane order), the counts are
// scanned over warps per destination and then over destinations, and every
// row moves to its stable sorted position in shared memory.
//
// A DRAM sector is 32 bytes (four 8-byte rows).  With F destinations a chunk
// adds only CHUNK/F rows to each, so writing every chunk's rows at once would
// leave most sectors half written and complete them a chunk later, after L2
// may have evicted them (a read-modify-write in DRAM).  Instead the rows of a
// destination's last, incomplete sector stay in shared memory ("pending", at
// most three) until a later chunk fills the sector; only whole sectors are
// written, except the first and last sector of the block's range, which it
// shares with the neighbouring blocks.
// Fan-outs up to 2^WC_MAX_LOG2F take one pass; above, two passes of at most
// 64 digits.  At 600M pairs, fan-out 128 / 256 took 6.89 / 7.00 ms in two
// passes against 7.35 / 7.87 ms in one pass of a 512-thread kernel for up to
// 256 digits (since removed); fan-out 64 takes 5.57 ms in one pass against
// 6.78 ms in two.
constexpr int WC_MAX_LOG2F = 6;

// Rows r0 + (warp-striped positions) into registers, key in .x and payload
// in .y, so that a row moves to shared memory as one 16-byte element.
template <bool PAY, int IT>
__device__ __forceinline__ void wc_load(const PartArgs &A, int64_t r0, int64_t hi, longlong2 (&kv)[IT])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const int64_t r = r0 + warp * 32 * IT + i * 32 + lane;
        kv[i].x = r < hi ? __ldcs(reinterpret_cast<const long long *>(A.keys) + r) : 0;
        kv[i].y = PAY && r < hi ? __ldcs(static_cast<const long long *>(A.pay[0]) + r) : 0;
    }
}

// Rows [r0, min(r0 + CH, hi)) of the keys and of the int64 payloads fetched
// into L2 (a hint: every address lies inside those rows).  Half the threads
// take the keys' 128-byte lines, half the payloads'.  The small fan-out
// scatter fetches the next chunk at the start of every step and loads it
// into registers halfway through, so that load hits L2.  Measured at 600M
// pairs, fan-out 1024 (whole call, 256 x 8 rows a chunk): 8.74 ms with two
// blocks per SM loading the next chunk into a second register set and no
// fetch; 8.13 ms with the fetch of the chunk after that (8.29 ms three chunks
// ahead); 7.99 ms with three blocks per SM, one register set, each chunk
// loaded at its step's start after a fetch one step ahead; 7.69 ms with the
// load moved halfway (kept); 9.18 ms for the same without the fetch.
template <bool PAY, int T, int CH>
__device__ __forceinline__ void part_prefetch_l2(const PartArgs &A, int64_t r0, int64_t hi)
{
    if (r0 >= hi) return;
    const int64_t nbytes = ((r0 + CH < hi ? r0 + CH : hi) - r0) * 8;
    constexpr int H = PAY ? T / 2 : T;
    const int t = static_cast<int>(threadIdx.x);
    const char *col = (t < H ? reinterpret_cast<const char *>(A.keys) : static_cast<const char *>(A.pay[0])) + r0 * 8;
    for (int64_t o = static_cast<int64_t>(t < H ? t : t - H) * 128; o < nbytes; o += H * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(col + o));
}

// ---------------------------------------------------------------------------
// Small fan-out scatter: at most 64 digits per launch (fan-out <= 64 in one
// pass, and both passes of fan-out 128 .. 4096), with the work per row cut
// down:
//   * a chunk whose rows all lie inside the item is loaded and ranked
//     without per-row bounds tests (FULL); a step fetches the next chunk
//     into L2 first and loads it into the one register set as soon as its
//     own rows are in shared memory, so the loads overlap the write-out;
//   * digit state lives in registers: lane d of every warp keeps the q of
//     digit d's next row (r, the same in every warp), so the digits' sorted
//     starts and the write-out need no shared-memory tables;
//   * every digit's run in the sorted chunk starts on the parity of its r
//     (one row of padding per digit at most), so the rows of whole sectors
//     move from shared memory to DRAM as 16-byte pairs of rows;
//   * the sorted chunk holds its keys, then its payloads, and is
//     double-buffered: two barriers per chunk.
// Each digit is written by one warp (digits p == warp mod NWARP): first the
// rows of every owned digit's partial sectors in one round, a lane per row
// (rows completing the digit's pending sector, rows before the item's first
// sector boundary, and rows of the last incomplete sector, which stay in
// shared memory until a later chunk or the end of the item completes them),
// then the whole sectors: with up to 32 digits one bulk store of keys and
// one of payloads per digit, else two rows per lane.
template <bool PAY, int BITS, int T, int IT>
struct SfLayout {
    static constexpr int NWARP = T / 32, CH = T * IT, NCL = BITS > 5 ? 2 : 1, FMAX = 32 * NCL;
    static constexpr int SROW = CH + FMAX;                      // rows of one sorted buffer (with padding)
    static constexpr int ES = PAY ? 16 : 8;                     // bytes per row: key, payload
    static_assert(SROW % 2 == 0, "16-byte pairs of rows");
    static constexpr size_t sb = 0;                             // [2] x (SROW keys, SROW payloads)
    static constexpr size_t pend = sb + 2 * SROW * ES;          // FMAX * 4 keys, FMAX * 4 payloads
    static constexpr size_t ob = pend + FMAX * 4 * ES;          // [FMAX] key address of q = 0
    static constexpr size_t cnt = ob + FMAX * 8;                // [NWARP][FMAX] rows per warp and digit
    static constexpr size_t total = cnt + NWARP * FMAX * 4;
};

// Rows r0 + (warp-striped positions) of a chunk inside the item: no tests.
template <bool PAY, int IT>
__device__ __forceinline__ void sf_load_full(const PartArgs &A, int64_t r0, longlong2 (&kv)[IT])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long *k = reinterpret_cast<const long long *>(A.keys) + r0 + warp * 32 * IT + lane;
    const long long *v = static_cast<const long long *>(A.pay[0]) + r0 + warp * 32 * IT + lane;
#pragma unroll
    for (int i = 0; i < IT; i++) {
        kv[i].x = __ldcs(k + i * 32);
        kv[i].y = PAY ? __ldcs(v + i * 32) : 0;
    }
}

// Digit and stable rank (among the warp's earlier rows of the chunk with
// that digit) of every row; cl[k] counts the warp's rows of digit
// lane + 32 k.  Lane e forms the mask of lanes whose row has digit e (AND of
// the digit bits' ballots or their complements); a row reads its peers and
// its base count from lane (digit & 31).  Invalid rows get digit ~0u.
template <int BITS, int IT, bool FULL, int NCL>
__device__ __forceinline__ void sf_rank(const PartArgs &A, const longlong2 (&kv)[IT], int vlo, int vhi,
                                        uint32_t (&dg)[IT], uint32_t (&rk)[IT], uint32_t (&cl)[NCL])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    unsigned me0[IT], me1[IT];
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const int row = warp * 32 * IT + i * 32 + lane;
        const bool valid = FULL || (row >= vlo && row < vhi);
        const uint32_t d = valid ? (dev_part_id(kv[i].x, A.log2f, A.mode, A.shift) >> A.dshift) & A.dmask : 0u;
        unsigned me = FULL ? QE_FULL_MASK : __ballot_sync(QE_FULL_MASK, valid);
#pragma unroll
        for (int bit = 0; bit < (BITS < 5 ? BITS : 5); bit++) {
            const unsigned set = __ballot_sync(QE_FULL_MASK, (d >> bit) & 1u);
            me &= ((lane >> bit) & 1) ? set : ~set;
        }
        unsigned me1v = 0;
        if (BITS > 5) {
            const unsigned set5 = __ballot_sync(QE_FULL_MASK, (d >> 5) & 1u);
            me1v = me & set5;
            me &= ~set5;
        }
        me0[i] = me;
        me1[i] = me1v;
        dg[i] = valid ? d : 0xffffffffu;
    }
#pragma unroll
    for (int i = 0; i < IT; i++) {
        const int src = static_cast<int>(dg[i] & 31u);
        unsigned peers = __shfl_sync(QE_FULL_MASK, me0[i], src);
        uint32_t basec = __shfl_sync(QE_FULL_MASK, cl[0], src);
        if (BITS > 5) {
            const unsigned peers1 = __shfl_sync(QE_FULL_MASK, me1[i], src);
            const uint32_t base1 = __shfl_sync(QE_FULL_MASK, cl[NCL - 1], src);
            if (dg[i] >= 32u) {
                peers = peers1;
                basec = base1;
            }
        }
        rk[i] = basec + __popc(peers & lt);
        cl[0] += __popc(me0[i]);
        if (BITS > 5) cl[NCL - 1] += __popc(me1[i]);
    }
}

// Row t of a sorted buffer (N rows) or of the pending slots (N = FMAX * 4)
// as (key, payload): N keys, then N payloads.
template <bool PAY, int N>
__device__ __forceinline__ longlong2 sf_row(const unsigned char *base, int t)
{
    const long long *k = reinterpret_cast<const long long *>(base);
    return make_longlong2(k[t], PAY ? k[N + t] : 0);
}
template <bool PAY, int N>
__device__ __forceinline__ void sf_put(unsigned char *base, int t, longlong2 v)
{
    long long *k = reinterpret_cast<long long *>(base);
    k[t] = v.x;
    if (PAY) k[N + t] = v.y;
}

// Value of a digit's register state (held by lane p & 31 of every warp,
// in slot p >> 5) for the digit p of the calling lane.
template <int NCL, typename V>
__device__ __forceinline__ V sf_get(const V (&v)[NCL], int p)
{
    V x = __shfl_sync(QE_FULL_MASK, v[0], p & 31);
    if (NCL > 1) {
        const V y = __shfl_sync(QE_FULL_MASK, v[NCL - 1], p & 31);
        if (p >= 32) x = y;
    }
    return x;
}

// One chunk: rank, place in sorted buffer `buf`, write out.  rr (q of every
// lane digit's next row) advances by the chunk's rows.  kv then takes the
// rows of the next chunk, at nx (up to hi), as soon as its own rows are in
// shared memory, so those loads overlap the write-out.
template <bool PAY, int BITS, int T, int IT, bool FULL>
__device__ __forceinline__ void sf_chunk(const PartArgs &A, unsigned char *smem, int buf, longlong2 (&kv)[IT],
                                         int vlo, int vhi, int F, int (&rr)[SfLayout<PAY, BITS, T, IT>::NCL],
                                         long long *outK, int64_t dP, bool vecP, int64_t nx, int64_t hi)
{
    using L = SfLayout<PAY, BITS, T, IT>;
    constexpr int NWARP = L::NWARP, NCL = L::NCL, FMAX = L::FMAX, SROW = L::SROW;
    constexpr int NJ = FMAX / NWARP, LPD = 32 / NJ;      // digits per warp, lanes per digit
    // whole sectors as bulk stores for up to 32 digits (at 600M pairs: fan-out
    // 1024 in 8.73 against 8.97 ms); with 64 digits a launch the per-lane
    // copy measured faster (fan-out 64: 5.98 against 6.06 ms)
    constexpr bool SF_BULK = BITS <= 5;
    static_assert(LPD >= 8, "a digit's partial sectors take up to seven lanes");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *sb = smem + L::sb + static_cast<size_t>(buf) * SROW * L::ES;
    unsigned char *pend = smem + L::pend;
    long long *const *ob = reinterpret_cast<long long *const *>(smem + L::ob);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + L::cnt);

    uint32_t dg[IT], rk[IT], cl[NCL];
#pragma unroll
    for (int k = 0; k < NCL; k++) cl[k] = 0;
    sf_rank<BITS, IT, FULL, NCL>(A, kv, vlo, vhi, dg, rk, cl);
    // this buffer's bulk stores of two chunks ago have read it (the previous
    // chunk's, from the other buffer, may still be running); the barrier
    // below orders the wait before anyone writes the buffer
    if (SF_BULK && lane < NJ) tma_store_wait_read<1>();
#pragma unroll
    for (int k = 0; k < NCL; k++)
        if (lane + 32 * k < F) cnt[warp * FMAX + lane + 32 * k] = cl[k];
    __syncthreads();
    // per lane digit: rows of earlier warps (pre) and of the chunk (tot); the
    // digit's run starts at the exclusive scan of (tot + 1) over digits,
    // moved by one row when needed so that its start has the parity of r
    uint32_t pre[NCL], tot[NCL], s0[NCL];
#pragma unroll
    for (int k = 0; k < NCL; k++) {
        pre[k] = 0;
        tot[k] = 0;
        const int d = lane + 32 * k;
        if (d < F) {
#pragma unroll
            for (int w = 0; w < NWARP; w++) {
                const uint32_t x = cnt[w * FMAX + d];
                pre[k] += w < warp ? x : 0u;
                tot[k] += x;
            }
        }
    }
    {
        const uint32_t v0 = lane < F ? tot[0] + 1u : 0u;
        const uint32_t i0 = warp_incl_scan(v0);
        const uint32_t b0 = i0 - v0;
        s0[0] = b0 + ((static_cast<uint32_t>(rr[0]) - b0) & 1u);
        if (NCL > 1) {
            const uint32_t all0 = __shfl_sync(QE_FULL_MASK, i0, 31);
            const uint32_t v1 = lane + 32 < F ? tot[NCL - 1] + 1u : 0u;
            const uint32_t i1 = warp_incl_scan(v1);
            const uint32_t b1 = all0 + i1 - v1;
            s0[NCL - 1] = b1 + ((static_cast<uint32_t>(rr[NCL - 1]) - b1) & 1u);
        }
    }
    // rows to their sorted positions
    {
        const uint32_t o0 = s0[0] + pre[0], o1 = NCL > 1 ? s0[NCL - 1] + pre[NCL - 1] : 0u;
#pragma unroll
        for (int i = 0; i < IT; i++) {
            const int src = static_cast<int>(dg[i] & 31u);
            uint32_t pos = __shfl_sync(QE_FULL_MASK, o0, src);
            if (NCL > 1) {
                const uint32_t pos1 = __shfl_sync(QE_FULL_MASK, o1, src);
                if (dg[i] >= 32u) pos = pos1;
            }
            if (FULL || dg[i] != 0xffffffffu) sf_put<PAY, SROW>(sb, static_cast<int>(pos + rk[i]), kv[i]);
        }
    }
    if (nx + T * IT <= hi) sf_load_full<PAY, IT>(A, nx, kv);
    else if (nx < hi) wc_load<PAY, IT>(A, nx, hi, kv);
    if (SF_BULK) fence_proxy_async_smem();   // the sorted rows, visible to the bulk stores below
    __syncthreads();
    // the rows of every owned digit's partial sectors: lanes LPD j .. LPD j + 6
    // of digit p = warp + NWARP j; roles 0..3 write rows now, roles 4..6 keep
    // rows pending.  All reads come before any write of a pending slot.
    {
        const int j = lane / LPD, role = lane % LPD;
        const int p = warp + NWARP * j;
        const int r = sf_get<NCL>(rr, p);
        const int h = static_cast<int>(sf_get<NCL>(tot, p));
        const int s = static_cast<int>(sf_get<NCL>(s0, p));
        longlong2 v = make_longlong2(0, 0);
        long long *dst = nullptr;
        int slot = -1;
        if (p < F) {
            const int e = r + h;
            const int x = r - s;                       // row q sits at sorted position q - x; x is even
            const int lim = e > 0 ? (e & ~3) : 0;      // rows q < lim are written now
            const int a = r > 0 ? ((r + 3) & ~3) : 0;  // first whole sector of this chunk's rows
            long long *o = ob[p];
            if (role < 4) {
                if (r < 0) {
                    // rows before the item's first sector boundary: their
                    // sector is shared with the previous item
                    const int q = r + role;
                    if (role < 3 && q < 0 && q < e) {
                        v = sf_row<PAY, SROW>(sb, q - x);
                        dst = o + q;
                    }
                } else if ((r & 3) && e >= a) {
                    // the pending sector completes: its earlier rows, then this chunk's
                    const int q = (r & ~3) + role;
                    v = q < r ? sf_row<PAY, FMAX * 4>(pend, p * 4 + role) : sf_row<PAY, SROW>(sb, q - x);
                    dst = o + q;
                }
            } else if (role < 7) {
                const int q = (lim > r ? lim : r) + role - 4;
                if (q < e) {
                    v = sf_row<PAY, SROW>(sb, q - x);
                    slot = p * 4 + (q & 3);
                }
            }
        }
        __syncwarp();
        if (dst && QE_DCHECK(A.st, dst >= outK && dst < outK + A.n, dst - outK)) {
            __stcs(dst, v.x);
            if (PAY) __stcs(dst + dP, v.y);
        }
        if (slot >= 0) sf_put<PAY, FMAX * 4>(pend, slot, v);
    }
    // whole sectors: lane j of the warp stores digit warp + NWARP j's run
    // [a, lim) of keys (and of payloads) with one bulk copy each, from the
    // sorted buffer (16-byte aligned: q - x is even) to its 32-byte-aligned
    // output rows; payload columns not 16-byte aligned beside the keys take
    // two rows per lane instead (SF_BULK), as every column does without bulk
    // stores
    if (SF_BULK) {
        const int j = lane < NJ ? lane : 0;
        const int p = warp + NWARP * j;
        const int r = sf_get<NCL>(rr, p < F ? p : 0);
        const int h = static_cast<int>(sf_get<NCL>(tot, p < F ? p : 0));
        const int s = static_cast<int>(sf_get<NCL>(s0, p < F ? p : 0));
        if (lane < NJ && p < F) {
            long long *o = ob[p];
            const int e = r + h;
            const int x = r - s;
            const int lim = e > 0 ? (e & ~3) : 0;
            const int a = r > 0 ? ((r + 3) & ~3) : 0;
            if (lim > a && QE_DCHECK(A.st, o + a >= outK && o + lim <= outK + A.n, (o + a) - outK)) {
                const int t = a - x;
                const uint32_t bytes = static_cast<uint32_t>(lim - a) * 8u;
                tma_store_1d(o + a, reinterpret_cast<const long long *>(sb) + t, bytes);
                if (PAY && vecP) tma_store_1d(o + a + dP, reinterpret_cast<const long long *>(sb) + SROW + t, bytes);
            }
        }
        if (lane < NJ) tma_store_commit();
    }
    if (!SF_BULK || (PAY && !vecP)) {
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const int p = warp + NWARP * j;
            if (p >= F) break;
            const int kk = p >> 5, src = p & 31;
            const int r = __shfl_sync(QE_FULL_MASK, kk ? rr[NCL - 1] : rr[0], src);
            const int h = static_cast<int>(__shfl_sync(QE_FULL_MASK, kk ? tot[NCL - 1] : tot[0], src));
            const int s = static_cast<int>(__shfl_sync(QE_FULL_MASK, kk ? s0[NCL - 1] : s0[0], src));
            long long *o = ob[p];
            const int e = r + h;
            const int x = r - s;
            const int lim = e > 0 ? (e & ~3) : 0;
            const int a = r > 0 ? ((r + 3) & ~3) : 0;
            for (int q = a + 2 * lane; q < lim; q += 64) {
                if (!QE_DCHECK(A.st, o + q >= outK && o + q + 1 < outK + A.n, (o + q) - outK)) continue;
                if (!SF_BULK)
                    __stcs(reinterpret_cast<longlong2 *>(o + q), reinterpret_cast<const longlong2 *>(sb)[(q - x) >> 1]);
                if (PAY) {
                    const longlong2 v2 = reinterpret_cast<const longlong2 *>(sb)[(SROW + q - x) >> 1];
                    if (vecP) {
                        __stcs(reinterpret_cast<longlong2 *>(o + q + dP), v2);
                    } else {
                        __stcs(o + q + dP, v2.x);
                        __stcs(o + q + 1 + dP, v2.y);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NCL; k++) rr[k] += static_cast<int>(tot[k]);
}

template <bool PAY, int BITS, int T, int IT, int MINB>
__global__ void __launch_bounds__(T, MINB) k_part_scatter_sf(PartArgs A)
{
    using L = SfLayout<PAY, BITS, T, IT>;
    constexpr int NWARP = L::NWARP, CH = L::CH, NCL = L::NCL;
    static_assert(L::FMAX % NWARP == 0, "digits per warp");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *pend = smem + L::pend;
    long long **ob = reinterpret_cast<long long **>(smem + L::ob);
    const int F = static_cast<int>(A.dmask) + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Ffull = 1 << A.log2f;
    long long *outK = reinterpret_cast<long long *>(A.out_keys);
    const int64_t dP = PAY ? static_cast<long long *>(A.out_pay[0]) - outK : 0;
    const bool vecP = (dP & 1) == 0;
    const int aoff = static_cast<int>((reinterpret_cast<uintptr_t>(outK) >> 3) & 3);

    for (int64_t item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        int64_t lo, hi;
        int b = static_cast<int>(item), qhi = 0;
        if (A.omode == WC_PASS2) {
            const int nspan = (A.g1 + A.span - 1) / A.span;
            qhi = static_cast<int>(item / nspan);
            b = static_cast<int>(item % nspan) * A.span;
            const int b1 = b + A.span < A.g1 ? b + A.span : A.g1;
            const int64_t F1 = Ffull >> A.sub_bits;
            lo = A.t1[static_cast<int64_t>(b) * F1 + qhi];
            hi = A.t1[static_cast<int64_t>(b1 - 1) * F1 + qhi] + A.h1[static_cast<int64_t>(b1 - 1) * F1 + qhi];
        } else {
            lo = static_cast<int64_t>(b) * A.rows_per_block;
            hi = min(A.n, lo + A.rows_per_block);
        }
        if (hi <= lo) continue;
        // every warp: q of the next row of its lanes' digits (-hl, where hl
        // rows fill the key sector the digit's output run starts in); the
        // owner warp keeps the key address of q = 0
        int rr[NCL];
        // the previous item's bulk stores have read their rows
        if (BITS <= 5 && lane < L::FMAX / NWARP) tma_store_wait_read<0>();
        __syncthreads();                              // the previous item's pending rows are written
#pragma unroll
        for (int k = 0; k < NCL; k++) {
            const int p = lane + 32 * k;
            rr[k] = 0;
            if (p < F) {
                int64_t g;
                if (A.omode == WC_SINGLE) {
                    g = A.base[p] + A.off[static_cast<int64_t>(b) * Ffull + p];
                } else if (A.omode == WC_PASS1) {
                    g = A.t1[static_cast<int64_t>(b) * F + p];
                } else {
                    const int dst = (qhi << A.sub_bits) | p;
                    g = A.base[dst] + A.off[static_cast<int64_t>(b) * Ffull + dst];
                }
                const int hl = static_cast<int>((4 - ((g + aoff) & 3)) & 3);
                rr[k] = -hl;
                if (p % NWARP == warp) ob[p] = outK + g + hl;
            }
        }
        const int64_t nch = (hi - lo + CH - 1) / CH;
        // one register set: every step fetches the next chunk into L2 first
        // and loads it into kv once this chunk's rows are in shared memory
        longlong2 kv[IT];
        if (hi - lo >= CH) sf_load_full<PAY, IT>(A, lo, kv);
        else wc_load<PAY, IT>(A, lo, hi, kv);
        for (int64_t c = 0; c < nch; c++) {
            const int64_t r0 = lo + c * CH;
            const int buf = static_cast<int>(c & 1);
            part_prefetch_l2<PAY, T, CH>(A, r0 + CH, hi);
            if (r0 + CH <= hi)
                sf_chunk<PAY, BITS, T, IT, true>(A, smem, buf, kv, 0, CH, F, rr, outK, dP, vecP, r0 + CH, hi);
            else
                sf_chunk<PAY, BITS, T, IT, false>(A, smem, buf, kv, 0, static_cast<int>(hi - r0), F, rr, outK, dP, vecP,
                                                  r0 + CH, hi);
        }
        __syncwarp();
        // rows still pending at the end of the item (owner lanes)
#pragma unroll
        for (int k = 0; k < NCL; k++) {
            const int p = lane + 32 * k;
            if (p < F && p % NWARP == warp && rr[k] > 0) {
                const int r = rr[k];
                long long *o = ob[p] + (r & ~3);
                for (int j = 0; j < (r & 3); j++) {
                    if (!QE_DCHECK(A.st, o + j >= outK && o + j < outK + A.n, (o + j) - outK)) continue;
                    const longlong2 v = sf_row<PAY, L::FMAX * 4>(pend, p * 4 + j);
                    __stcs(o + j, v.x);
                    if (PAY) __stcs(o + dP + j, v.y);
                }
            }
        }
    }
    // every bulk store done before the block's memory is released
    if (BITS <= 5 && lane < L::FMAX / NWARP) tma_store_wait_all();
}

// Two passes: per first-pass range b and high digit q, the rows and the
// scratch start: h1[b][q] = sum over the low digits r of hist[b][q, r] and
// t1[b][q] = base[q, 0] + sum over r of off[b][q, r] (range b's rows with
// high digit q follow those of the earlier ranges, inside the run of q).
__global__ void k_part_two_pass_tables(const uint32_t *hist, const int64_t *off, const int64_t *base, int G, int F,
                                       int sub_bits, int64_t *t1, uint32_t *h1)
{
    const int F1 = F >> sub_bits, F2 = 1 << sub_bits;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= static_cast<int64_t>(G) * F1) return;
    const int b = static_cast<int>(i / F1), q = static_cast<int>(i % F1);
    uint32_t h = 0;
    int64_t o = 0;
    for (int r = 0; r < F2; r++) {
        const int64_t j = static_cast<int64_t>(b) * F + (q << sub_bits) + r;
        h += hist[j];
        o += off[j];
    }
    h1[i] = h;
    t1[i] = base[q << sub_bits] + o;
}

// Block shapes of the write-combining scatters, by digits per launch
// (measured on GB300).  Up to 32 digits, two blocks of 256 threads x 11 rows
// per SM (125 registers, one register set).  At 600M pairs, fan-out 1024,
// whole call: 9, 10, 11 and 12 rows per thread with two blocks per SM took
// 7.41, 7.27, 7.11 and 7.56 ms; 8 rows with three blocks 7.68 ms, 6 rows with
// four 7.86 ms.  Before the L2 fetches, two blocks of 256 x 8 with a second
// register set for the next chunk (9.3 ms) beat one block of 512 x 8
// (9.9 ms), 512 x 4 and 1024 x 4 at 32 warps per SM (10.0 / 10.9 ms; 64
// registers with spills), 256 x 6 (10.1 ms), and three blocks of 256 x 8
// without the second set (9.7 ms).  From 64 digits a chunk of 256 threads
// gives each digit runs too short for the per-digit work, so one block of
// 512 x 8 runs per SM (its one register set measured faster than two:
// fan-out 4096 in 10.46 against 11.02 ms, fan-out 64 in 5.57 against
// 5.82 ms; 10 and 12 rows per thread 10.55 / 11.21 ms); and every block writes
// one output page per destination and column at a time, so beyond a few
// hundred pages per SM (measured at 256 digits) the address translation
// caches miss.
struct WcShape {
    int threads, items;
    const void *kernel;
    size_t smem;
};

template <bool PAY>
static WcShape wc_shape(int log2f)
{
    if (log2f <= 5)
        return {256, 11, reinterpret_cast<const void *>(k_part_scatter_sf<PAY, 5, 256, 11, 2>),
                SfLayout<PAY, 5, 256, 11>::total};
    if (log2f <= 6)
        return {512, 8, reinterpret_cast<const void *>(k_part_scatter_sf<PAY, 6, 512, 8, 1>),
                SfLayout<PAY, 6, 512, 8>::total};
    return {0, 0, nullptr, 0};   // beyond one write-combining pass: not taken
}

// General scatter (any payload columns, any fan-out up to 4096), at 1024
// threads per block where its shared memory fits and at 512 otherwise.
namespace gen1024 {
constexpr int PT = 1024;
constexpr bool EVICT_LAST = false;
#include "qe_part_general.cuh"
}  // namespace gen1024
namespace gen512 {
constexpr int PT = 512;
constexpr bool EVICT_LAST = true;
#include "qe_part_general.cuh"
}  // namespace gen512

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
    // Plan.  The write-combining scatter takes keys with one int64 payload or
    // none: in one pass up to fan-out 2^WC_MAX_LOG2F, and in two passes of
    // at most 64 digits each beyond (the first by the high bits of the
    // destination into scratch, the second by the low bits), which keeps the
    // output pages an SM writes at a time within the translation caches.
    // Everything else takes the general scatter.
    const bool wc = !ctx->tune_part_general && (npayload == 0 || fast);
    const bool two = wc && log2_fanout > WC_MAX_LOG2F;
    const int sub_bits = two ? log2_fanout / 2 : 0;
    const int F1 = F >> sub_bits;
    const WcShape ws = fast ? wc_shape<true>(log2_fanout - sub_bits) : wc_shape<false>(log2_fanout - sub_bits);
    const WcShape ws2 = fast ? wc_shape<true>(sub_bits) : wc_shape<false>(sub_bits);
    const bool big = gen1024::scatter_smem(log2_fanout, fast) <= ctx->smem_optin;
    const size_t smem = wc ? ws.smem
                           : (big ? gen1024::scatter_smem(log2_fanout, fast) : gen512::scatter_smem(log2_fanout, fast));
    const size_t smem2 = two ? ws2.smem : 0;
    if (smem > ctx->smem_optin || smem2 > ctx->smem_optin)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "partition: fan-out too large");
    const void *kscatter;
    if (wc)
        kscatter = ws.kernel;
    else if (big)
        kscatter = fast ? reinterpret_cast<const void *>(gen1024::k_part_scatter<true>)
                        : reinterpret_cast<const void *>(gen1024::k_part_scatter<false>);
    else
        kscatter = fast ? reinterpret_cast<const void *>(gen512::k_part_scatter<true>)
                        : reinterpret_cast<const void *>(gen512::k_part_scatter<false>);
    const int threads = wc ? ws.threads : (big ? gen1024::PT : gen512::PT);
    const int64_t chunk = wc ? static_cast<int64_t>(ws.threads) * ws.items : (big ? gen1024::CHUNK : gen512::CHUNK);
    // (both passes may use the same kernel: allow the larger footprint)
    const size_t smem_attr = two && ws2.kernel == kscatter && smem2 > smem ? smem2 : smem;
    QE_CUDA(ctx, cudaFuncSetAttribute(kscatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem_attr)));
    int per_sm = 0;
    QE_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kscatter, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t G = static_cast<int64_t>(ctx->num_sms) * per_sm;
    int64_t need = qe_ceil_div(nrows, chunk);
    if (G > need) G = need;
    // whole chunks per block
    A.rows_per_block = qe_ceil_div(qe_ceil_div(nrows, G), chunk) * chunk;
    G = qe_ceil_div(nrows, A.rows_per_block);
    A.tma = !wc && qe_aligned(keys, 16) && (!fast || qe_aligned(A.pay[0], 16));
    A.spin_limit = ctx->spin_limit;
    A.st = ctx->dstat;
    int64_t G2 = 0;
    if (two) {
        if (ws2.kernel != kscatter)
            QE_CUDA(ctx, cudaFuncSetAttribute(ws2.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(smem2)));
        int per_sm2 = 0;
        QE_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, ws2.kernel, ws2.threads, smem2));
        G2 = static_cast<int64_t>(ctx->num_sms) * (per_sm2 < 1 ? 1 : per_sm2);
    }

    // scratch: hist | off | tot, and for two passes t1 | h1 | keys | payload
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t hist_bytes = up(static_cast<size_t>(G) * F * sizeof(uint32_t));
    const size_t off_bytes = up(static_cast<size_t>(G) * F * sizeof(int64_t));
    const size_t tot_bytes = up(static_cast<size_t>(F) * sizeof(int64_t));
    const size_t t1_bytes = two ? up(static_cast<size_t>(G) * F1 * sizeof(int64_t)) : 0;
    const size_t h1_bytes = two ? up(static_cast<size_t>(G) * F1 * sizeof(uint32_t)) : 0;
    const size_t col_bytes = two ? up(static_cast<size_t>(nrows) * sizeof(int64_t)) : 0;
    void *scratch = nullptr;
    qe_status st = qe_alloc(ctx, &scratch,
                            hist_bytes + off_bytes + tot_bytes + t1_bytes + h1_bytes + col_bytes * (fast ? 2 : 1), s);
    if (st != QE_OK) return st;
    unsigned char *sp = static_cast<unsigned char *>(scratch);
    A.off = reinterpret_cast<int64_t *>(sp);
    int64_t *tot = reinterpret_cast<int64_t *>(sp + off_bytes);
    A.hist = reinterpret_cast<uint32_t *>(sp + off_bytes + tot_bytes);
    A.base = out_offsets;
    int64_t *t1 = reinterpret_cast<int64_t *>(sp + off_bytes + tot_bytes + hist_bytes);
    uint32_t *h1 = reinterpret_cast<uint32_t *>(sp + off_bytes + tot_bytes + hist_bytes + t1_bytes);
    int64_t *tmpK = reinterpret_cast<int64_t *>(sp + off_bytes + tot_bytes + hist_bytes + t1_bytes + h1_bytes);
    int64_t *tmpP = tmpK + col_bytes / sizeof(int64_t);

    cudaError_t e = cudaMemsetAsync(A.hist, 0, static_cast<size_t>(G) * F * sizeof(uint32_t), s);
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
    if (e == cudaSuccess && two) {
        const int64_t cells = G * F1;
        k_part_two_pass_tables<<<static_cast<unsigned>((cells + 255) / 256), 256, 0, s>>>(
            A.hist, A.off, out_offsets, static_cast<int>(G), F, sub_bits, t1, h1);
        QE_LAUNCHED(ctx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ProfScope prof(ctx, "part_scatter", s);
        PartArgs A1 = A;
        A1.dshift = sub_bits;
        A1.dmask = static_cast<uint32_t>(F1 - 1);
        A1.omode = two ? WC_PASS1 : WC_SINGLE;
        A1.nitems = G;
        if (two) {
            A1.t1 = t1;
            A1.out_keys = tmpK;
            if (fast) A1.out_pay[0] = tmpP;
        }
        void *args[] = {&A1};
        e = cudaLaunchKernel(kscatter, dim3(static_cast<unsigned>(G)), dim3(threads), args, smem, s);
        QE_LAUNCHED(ctx);
        if (e == cudaSuccess && two) {
            PartArgs A2 = A;
            A2.keys = tmpK;
            if (fast) A2.pay[0] = tmpP;
            A2.dshift = 0;
            A2.dmask = static_cast<uint32_t>((1 << sub_bits) - 1);
            A2.omode = WC_PASS2;
            A2.sub_bits = sub_bits;
            A2.g1 = static_cast<int>(G);
            A2.span = ctx->tune_part_span > 0 ? ctx->tune_part_span : 8;
            A2.t1 = t1;
            A2.h1 = h1;
            A2.nitems = qe_ceil_div(G, A2.span) * F1;
            void *args2[] = {&A2};
            e = cudaLaunchKernel(ws2.kernel, dim3(static_cast<unsigned>(G2)), dim3(ws2.threads), args2, smem2, s);
            QE_LAUNCHED(ctx);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    qe_free(ctx, scratch, s);
    if (e != cudaSuccess) return qe_cuda_fail(ctx, e, "partition launch");
    return QE_OK;
}
