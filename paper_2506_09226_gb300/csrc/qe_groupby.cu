// qe_groupby.cu -- hash group-by with exact SUM / COUNT / MIN / MAX
// (Sec. 2.3: sum, min and max among the reduction kinds; Sec. 2.4: group-by
// inside the per-GPU program).
//
// Each block of a persistent grid aggregates its rows into a private
// shared-memory table (when the expected group count fits) and merges it into
// one HBM table at the end; rows whose key cannot be placed in the
// shared-memory table go straight to the HBM table.  The HBM table is then
// compacted into the caller's output.
#include "qe_pipe_core.cuh"

namespace {

constexpr int GB_THREADS = 1024;   // one block per SM shares the shared-memory table
constexpr int GB_ITEMS = 4;

struct ColRef {
    const void *data;
    int32_t type;
    int32_t gather;
};

struct GroupbyArgs {
    int64_t n;
    const int32_t *rows;
    ColRef key_hi, key_lo;
    ColRef a[QE_MAX_AGGS], b[QE_MAX_AGGS];
    AggOps ops;
    GTable g;
    int S;
    int log2S;
};

__device__ __forceinline__ int64_t col_at(const ColRef &c, int64_t i, int64_t r)
{
    return dev_col(c.data, c.type, c.gather ? r : i);
}

__global__ void __launch_bounds__(GB_THREADS) k_groupby(GroupbyArgs A)
{
    extern __shared__ unsigned long long sm[];
    if (A.S) st_zero(sm, A.S, A.ops.n);
    __syncthreads();
    const int64_t tile_rows = static_cast<int64_t>(GB_THREADS) * GB_ITEMS;
    const int64_t ntiles = (A.n + tile_rows - 1) / tile_rows;
    const uint32_t mask = A.S ? static_cast<uint32_t>(A.S - 1) : 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int64_t r[GB_ITEMS];
#pragma unroll
        for (int k = 0; k < GB_ITEMS; k++) {
            const int64_t i = tile * tile_rows + k * GB_THREADS + threadIdx.x;
            r[k] = i < A.n ? (A.rows ? static_cast<int64_t>(__ldg(A.rows + i)) : i) : -1;
        }
#pragma unroll
        for (int k = 0; k < GB_ITEMS; k++) {
            const int64_t i = tile * tile_rows + k * GB_THREADS + threadIdx.x;
            if (r[k] < 0) continue;
            const int64_t lo = col_at(A.key_lo, i, r[k]);
            int64_t key = lo;
            if (A.key_hi.data)
                key = static_cast<int64_t>((static_cast<uint64_t>(col_at(A.key_hi, i, r[k])) << 32) |
                                           static_cast<uint32_t>(lo));
            const unsigned long long kx = static_cast<unsigned long long>(key) ^ GB_SIGN;
            if (kx == 0) {
                dev_report(A.g.st, QE_ERR_RESERVED_KEY, 0);
                continue;
            }
            unsigned long long e[QE_MAX_AGGS];
#pragma unroll
            for (int a = 0; a < QE_MAX_AGGS; a++) {
                e[a] = 0;
                if (a < A.ops.n) {
                    int64_t v = 0;
                    if (A.ops.op[a] != QE_COUNT) {
                        uint64_t x = static_cast<uint64_t>(col_at(A.a[a], i, r[k]));
                        if (A.b[a].data) x *= static_cast<uint64_t>(col_at(A.b[a], i, r[k]));
                        v = static_cast<int64_t>(x);
                    }
                    e[a] = agg_encode(A.ops.op[a], v);
                }
            }
            if (A.S) {
                const uint32_t h = st_hash(kx, A.log2S);
                const int slot = sm[h] == kx ? static_cast<int>(h) : st_find_slow(sm, mask, kx, h);
                if (slot >= 0) {
#pragma unroll
                    for (int a = 0; a < QE_MAX_AGGS; a++)
                        if (a < A.ops.n) st_update(sm + (a + 1) * A.S + slot, A.ops.op[a], e[a]);
                    continue;
                }
            }
            spill_row_ni(A.g, A.ops, kx, e[0], e[1], e[2], e[3]);
        }
    }
    if (A.S) {
        __syncthreads();
        st_flush(sm, A.S, A.ops, A.g);
    }
}

bool col_ok(const qe_col &c, int64_t n, const int32_t *rows)
{
    if (!c.data) return false;
    if (!qe_valid_type(c.type) || !qe_aligned(c.data, c.type)) return false;
    if (c.gather && !rows) return false;
    (void)n;
    return true;
}

}  // namespace

extern "C" qe_status qe_groupby(qe_ctx *ctx, int64_t n, const int32_t *rows, qe_col key_hi, qe_col key_lo,
                                const qe_agg *aggs, int naggs, int placement, const qe_groups_out *out, void *stream)
{
    if (!ctx) return QE_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n < 0 || naggs < 0 || naggs > QE_MAX_AGGS || (naggs > 0 && !aggs) || placement < QE_GB_AUTO ||
        placement > QE_GB_HBM)
        return qe_fail(ctx, QE_ERR_INVALID_ARG, "groupby: bad argument");
    GroupbyArgs A{};
    A.n = n;
    A.rows = rows;
    if (n > 0) {
        if (!col_ok(key_lo, n, rows) || (key_hi.data && !col_ok(key_hi, n, rows)))
            return qe_fail(ctx, QE_ERR_INVALID_ARG, "groupby: bad key column");
    }
    A.key_lo = {key_lo.data, key_lo.type, key_lo.gather};
    A.key_hi = {key_hi.data, key_hi.type, key_hi.gather};
    A.ops.n = naggs;
    for (int a = 0; a < naggs; a++) {
        const qe_agg &g = aggs[a];
        if (g.op < QE_SUM || g.op > QE_MAX) return qe_fail(ctx, QE_ERR_INVALID_ARG, "groupby: bad aggregate");
        A.ops.op[a] = g.op;
        if (g.op != QE_COUNT && n > 0) {
            if (!col_ok(g.a, n, rows) || (g.b.data && !col_ok(g.b, n, rows)))
                return qe_fail(ctx, QE_ERR_INVALID_ARG, "groupby: bad aggregate column");
        }
        A.a[a] = {g.a.data, g.a.type, g.a.gather};
        A.b[a] = {g.op == QE_COUNT ? nullptr : g.b.data, g.b.type, g.b.gather};
    }
    qe_status st = gt_check_out(ctx, out, A.ops);
    if (st != QE_OK) return st;
    cudaSetDevice(ctx->device);
    GroupTableHost t;
    st = gt_create(ctx, out->capacity, naggs, t, s);
    if (st != QE_OK) return st;
    A.g.words = t.words;
    A.g.mask = t.slots - 1;
    A.g.stride = t.stride;
    A.g.capacity = out->capacity;
    A.g.st = ctx->dstat;
    const size_t budget = ctx->smem_optin > 4096 ? ctx->smem_optin - 4096 : 0;
    A.S = 0;
    if (placement != QE_GB_HBM) {
        // The capacity bounds the number of groups, so a table of
        // pow2 >= capacity slots cannot fill up; a table that does not fit
        // the budget is used only when shared memory is asked for, as a
        // cache in front of the HBM table.
        uint64_t want = 64;
        while (want < static_cast<uint64_t>(out->capacity)) want <<= 1;
        if (want * 8 * (1 + naggs) <= budget) A.S = static_cast<int>(want);
        else if (placement == QE_GB_SMEM) A.S = st_slots_max(naggs, budget);
    }
    A.log2S = 0;
    while ((1 << A.log2S) < A.S) A.log2S++;
    const size_t smem = static_cast<size_t>(A.S) * 8 * (1 + naggs);
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaFuncSetAttribute(k_groupby, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        int per_sm = 1;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_groupby, GB_THREADS, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t grid = static_cast<int64_t>(ctx->num_sms) * per_sm;
        int64_t need = qe_ceil_div(n, GB_THREADS * GB_ITEMS);
        if (grid > need) grid = need;
        if (e == cudaSuccess) {
            ProfScope prof(ctx, "groupby", s);
            k_groupby<<<static_cast<unsigned>(grid), GB_THREADS, smem, s>>>(A);
            QE_LAUNCHED(ctx);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        st = gt_finalize(ctx, t, A.ops, out, s);
    } else {
        st = qe_cuda_fail(ctx, e, "groupby launch");
    }
    qe_free(ctx, t.words, s);
    return st;
}
