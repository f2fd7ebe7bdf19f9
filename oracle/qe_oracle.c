/*
 * qe_oracle.c -- plain, single-threaded CPU oracle for the relational
 * operator pipeline of "Terabyte-Scale Analytics in the Blink of an Eye"
 * (arxiv 2506.09226).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU operators compute.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * code, header, table or constant generator with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Every operator is written as its plain relational definition:
 *   - selection:  keep row i (ascending i) when every predicate holds
 *                 (Sec. 2.1: relational operators over column tensors);
 *   - partition:  apply one partitioning function to every row's key and lay
 *                 rows out as one contiguous run per destination, with a
 *                 start offset per destination (Sec. 2.2, Fig. 1; Sec. 2.3,
 *                 the per-sender offsets into one contiguous tensor per
 *                 column);
 *   - join:       inner equi-join of a probe column against unique build
 *                 keys (Sec. 2.2, the local join after exchange), and the
 *                 semi- and anti-join (membership in the build keys), and
 *                 the many-to-many join (build keys may repeat), and the join
 *                 on a pair of key columns;
 *   - group-by:   SUM / COUNT / MIN / MAX per distinct key (Sec. 2.3, the
 *                 aggregation kinds of the final reduction; Sec. 2.4, group
 *                 by in the compiled tensor program);
 *   - average:    AVG of a group derived from its exact integer SUM and
 *                 COUNT (Sec. 2.3 lists average among the final aggregation
 *                 kinds);
 *   - pipeline:   group-by(join(filter(fact), dim)), one tensor program per
 *                 GPU (Sec. 2.4).
 *
 * Readings where the paper is silent (the hash, stable order, sentinels,
 * fixed-point decimals) are stated at each function.  Parity pins: brute
 * force on tiny inputs (nested-loop join, dictionary group-by, per-row
 * partition loop) and invariants, in tests/test_oracle_pins.py.
 *
 * Integer arithmetic on aggregates wraps modulo 2^64 (two's complement); it
 * is done on uint64_t so that the wrap is defined behaviour in C.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Column element types (oracle's own numbering). */
enum { OR_I8 = 0, OR_I32 = 1, OR_I64 = 2 };
/* Comparison operators of a predicate; BETWEEN is lo <= x <= hi. */
enum { OR_LT = 0, OR_LE, OR_GT, OR_GE, OR_EQ, OR_NE, OR_BETWEEN };
/* Aggregate kinds. */
enum { OR_SUM = 0, OR_COUNT = 1, OR_MIN = 2, OR_MAX = 3 };
/* Status codes returned by the oracle. */
enum { OR_OK = 0, OR_DUPLICATE_KEY = 5, OR_BAD_ARG = 1 };

/* Value of element i of a column, sign-extended to int64. */
static int64_t col_get(const void *col, int type, int64_t i)
{
    if (type == OR_I8)  return (int64_t)((const int8_t *)col)[i];
    if (type == OR_I32) return (int64_t)((const int32_t *)col)[i];
    return ((const int64_t *)col)[i];
}

static int pred_holds(int64_t x, int op, int64_t lo, int64_t hi)
{
    switch (op) {
    case OR_LT: return x < lo;
    case OR_LE: return x <= lo;
    case OR_GT: return x > lo;
    case OR_GE: return x >= lo;
    case OR_EQ: return x == lo;
    case OR_NE: return x != lo;
    case OR_BETWEEN: return lo <= x && x <= hi;
    }
    return 0;
}

/*
 * Selection (Sec. 2.1; the filters of Sec. 2.2's Q19 example and Sec. 7.3's
 * Q12).  Conjunction of npreds comparisons; predicate p compares column
 * pred_col[p] with lo[p] (and hi[p] for BETWEEN).  Writes the ids of the
 * surviving rows in ascending order to out_sel and returns their number.
 */
int64_t oracle_filter(int64_t n, const void *const *cols, const int *types,
                      int npreds, const int *pred_col, const int *pred_op,
                      const int64_t *lo, const int64_t *hi, int32_t *out_sel)
{
    int64_t count = 0;
    for (int64_t i = 0; i < n; i++) {
        int keep = 1;
        for (int p = 0; p < npreds; p++) {
            int c = pred_col[p];
            if (!pred_holds(col_get(cols[c], types[c], i), pred_op[p], lo[p], hi[p]))
                keep = 0;
        }
        if (keep) out_sel[count++] = (int32_t)i;
    }
    return count;
}

/*
 * The partitioning function (Sec. 2.2: every process applies the same
 * partitioning function to its keys).  The paper does not name it.  Reading:
 * the 64-bit finalizer of MurmurHash3 (A. Appleby, public domain), whose
 * top log2(F) bits select the destination; it is a bijection on 64-bit
 * words, so equal keys always go to the same destination.
 */
uint64_t oracle_fmix64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* mode 0: hash (top bits of fmix64); mode 1: raw radix bits of the key
 * starting at bit `shift`. */
int64_t oracle_partition_of(int64_t key, int log2f, int mode, int shift)
{
    uint64_t fanout = (uint64_t)1 << log2f;
    if (log2f == 0) return 0;
    if (mode == 0) return (int64_t)(oracle_fmix64((uint64_t)key) >> (64 - log2f));
    return (int64_t)(((uint64_t)key >> shift) & (fanout - 1));
}

static int type_size(int t) { return t == OR_I8 ? 1 : (t == OR_I32 ? 4 : 8); }

/*
 * Partition (Sec. 2.2, Fig. 1; Sec. 2.3: one contiguous tensor per column,
 * with a start offset per destination).  Rows go to destination
 * part(key_i); within a destination they keep their input order (the paper
 * is silent on order; reading: stable).  out_offsets[p] is the first row of
 * destination p and out_offsets[F] = n.
 *
 * Plain form: count rows per destination, turn the counts into start
 * offsets, then place rows in ascending input order.
 */
void oracle_partition(int64_t n, const int64_t *keys, int npay,
                      const void *const *pay, const int *pay_types,
                      int log2f, int mode, int shift,
                      int64_t *out_keys, void *const *out_pay,
                      int64_t *out_offsets)
{
    int64_t fanout = (int64_t)1 << log2f;
    int64_t *next = (int64_t *)calloc((size_t)fanout, sizeof(int64_t));
    for (int64_t p = 0; p <= fanout; p++) out_offsets[p] = 0;
    for (int64_t i = 0; i < n; i++)
        out_offsets[oracle_partition_of(keys[i], log2f, mode, shift) + 1] += 1;
    for (int64_t p = 0; p < fanout; p++) out_offsets[p + 1] += out_offsets[p];
    for (int64_t p = 0; p < fanout; p++) next[p] = out_offsets[p];
    for (int64_t i = 0; i < n; i++) {
        int64_t p = oracle_partition_of(keys[i], log2f, mode, shift);
        int64_t dst = next[p]++;
        out_keys[dst] = keys[i];
        for (int c = 0; c < npay; c++) {
            int sz = type_size(pay_types[c]);
            memcpy((char *)out_pay[c] + dst * sz, (const char *)pay[c] + i * sz, (size_t)sz);
        }
    }
    free(next);
}

typedef struct { int32_t key; int32_t payload; } build_row;

static int cmp_build_row(const void *a, const void *b)
{
    int32_t x = ((const build_row *)a)->key, y = ((const build_row *)b)->key;
    return (x > y) - (x < y);
}

/*
 * Inner equi-join (Sec. 2.2: the local join once both inputs are
 * co-located).  For each probe position i in order (the row sel[i], or i when
 * sel is NULL), every build row j with key_j == probe_key gives one output
 * (probe row, payload_j).  Build keys must be unique (reading: the paper is
 * silent; duplicates are reported as OR_DUPLICATE_KEY and nothing is
 * emitted).  The lookup is a binary search of the build rows sorted by key.
 */
int oracle_join(int64_t nb, const int32_t *bkeys, const int32_t *bpay,
                int64_t np, const int32_t *pkeys, const int32_t *sel,
                int32_t *out_row, int32_t *out_pay, int64_t *out_count)
{
    build_row *b = (build_row *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(build_row));
    for (int64_t j = 0; j < nb; j++) { b[j].key = bkeys[j]; b[j].payload = bpay[j]; }
    qsort(b, (size_t)nb, sizeof(build_row), cmp_build_row);
    for (int64_t j = 1; j < nb; j++)
        if (b[j].key == b[j - 1].key) { free(b); *out_count = 0; return OR_DUPLICATE_KEY; }
    int64_t count = 0;
    for (int64_t i = 0; i < np; i++) {
        int32_t row = sel ? sel[i] : (int32_t)i;
        int32_t k = pkeys[row];
        int64_t lo = 0, hi = nb;           /* first index with key >= k */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (b[mid].key < k) lo = mid + 1; else hi = mid;
        }
        if (lo < nb && b[lo].key == k) {
            out_row[count] = row;
            out_pay[count] = b[lo].payload;
            count++;
        }
    }
    free(b);
    *out_count = count;
    return OR_OK;
}

/*
 * Many-to-many inner equi-join (the local join of Sec. 2.2 when build keys
 * repeat).  For each probe position i in order (the row sel[i], or i when sel
 * is NULL), every build row j with key_j == probe_key gives one output
 * (probe row, payload_j), in ascending j.  Plain nested loop over a sorted
 * copy: the build rows sorted by (key, j), then a binary search for the
 * first row of the probe key.  When the output would exceed `capacity`,
 * nothing past it is written; returns the full number of matches.
 */
static int cmp_build_row_stable(const void *a, const void *b)
{
    const build_row *x = (const build_row *)a, *y = (const build_row *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->payload > y->payload) - (x->payload < y->payload);   /* payload holds j here */
}

int64_t oracle_join_multi(int64_t nb, const int32_t *bkeys, const int32_t *bpay,
                          int64_t np, const int32_t *pkeys, const int32_t *sel,
                          int32_t *out_row, int32_t *out_pay, int64_t capacity)
{
    build_row *b = (build_row *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(build_row));
    for (int64_t j = 0; j < nb; j++) { b[j].key = bkeys[j]; b[j].payload = (int32_t)j; }
    qsort(b, (size_t)nb, sizeof(build_row), cmp_build_row_stable);
    int64_t count = 0;
    for (int64_t i = 0; i < np; i++) {
        int32_t row = sel ? sel[i] : (int32_t)i;
        int32_t k = pkeys[row];
        int64_t lo = 0, hi = nb;           /* first index with key >= k */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (b[mid].key < k) lo = mid + 1; else hi = mid;
        }
        for (int64_t t = lo; t < nb && b[t].key == k; t++) {
            if (count < capacity) {
                out_row[count] = row;
                out_pay[count] = bpay[b[t].payload];
            }
            count++;
        }
    }
    free(b);
    return count;
}

/*
 * Inner equi-join on a pair of key columns: the composite keys of joins
 * such as a (part, supplier) pair in the TPC-H queries the paper runs
 * (Sec. 6.1), joined locally as in Sec. 2.2.  Build row j matches probe row
 * r when bhi[j] == phi[r] and blo[j] == plo[r].  Build pairs must be unique
 * (OR_DUPLICATE_KEY, nothing emitted).  Output as oracle_join: for each
 * probe position in order, (probe row, payload) on a match.  The lookup is
 * a binary search of the build rows sorted by (hi, lo).
 */
typedef struct { int32_t hi, lo, payload; } pair_row;

static int cmp_pair_row(const void *a, const void *b)
{
    const pair_row *x = (const pair_row *)a, *y = (const pair_row *)b;
    if (x->hi != y->hi) return (x->hi > y->hi) - (x->hi < y->hi);
    return (x->lo > y->lo) - (x->lo < y->lo);
}

int oracle_join_pair(int64_t nb, const int32_t *bhi, const int32_t *blo, const int32_t *bpay,
                     int64_t np, const int32_t *phi, const int32_t *plo, const int32_t *sel,
                     int32_t *out_row, int32_t *out_pay, int64_t *out_count)
{
    pair_row *b = (pair_row *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(pair_row));
    for (int64_t j = 0; j < nb; j++) { b[j].hi = bhi[j]; b[j].lo = blo[j]; b[j].payload = bpay[j]; }
    qsort(b, (size_t)nb, sizeof(pair_row), cmp_pair_row);
    for (int64_t j = 1; j < nb; j++)
        if (b[j].hi == b[j - 1].hi && b[j].lo == b[j - 1].lo) { free(b); *out_count = 0; return OR_DUPLICATE_KEY; }
    int64_t count = 0;
    for (int64_t i = 0; i < np; i++) {
        int32_t row = sel ? sel[i] : (int32_t)i;
        pair_row key = { phi[row], plo[row], 0 };
        int64_t lo = 0, hi = nb;           /* first index with (hi, lo) >= key */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (cmp_pair_row(&b[mid], &key) < 0) lo = mid + 1; else hi = mid;
        }
        if (lo < nb && cmp_pair_row(&b[lo], &key) == 0) {
            const pair_row *hit = &b[lo];
            out_row[count] = row;
            out_pay[count] = hit->payload;
            count++;
        }
    }
    free(b);
    *out_count = count;
    return OR_OK;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Semi- and anti-join: the EXISTS and NOT EXISTS forms of the local join
 * (Sec. 2.2), which the TPC-H queries the paper runs (Sec. 6.1) contain.
 * For each probe position i in order (the row sel[i], or i when sel is
 * NULL) the row is emitted when some build key equals its key (anti = 0),
 * or when no build key does (anti = 1).  Build keys may repeat: only
 * membership matters.  The lookup is a binary search of the sorted build
 * keys.  Returns the number of rows written to out_row.
 */
int64_t oracle_semi_join(int64_t nb, const int32_t *bkeys, int64_t np, const int32_t *pkeys,
                         const int32_t *sel, int anti, int32_t *out_row)
{
    int32_t *b = (int32_t *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(int32_t));
    if (nb > 0) memcpy(b, bkeys, (size_t)nb * sizeof(int32_t));
    qsort(b, (size_t)nb, sizeof(int32_t), cmp_i32);
    int64_t count = 0;
    for (int64_t i = 0; i < np; i++) {
        int32_t row = sel ? sel[i] : (int32_t)i;
        int32_t k = pkeys[row];
        int64_t lo = 0, hi = nb;           /* first index with key >= k */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (b[mid] < k) lo = mid + 1; else hi = mid;
        }
        int found = lo < nb && b[lo] == k;
        if (found != (anti != 0)) out_row[count++] = row;
    }
    free(b);
    return count;
}

typedef struct { int64_t key; int64_t idx; } key_idx;

static int cmp_key_idx(const void *a, const void *b)
{
    const key_idx *x = (const key_idx *)a, *y = (const key_idx *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/*
 * Hash group-by, stated without a hash (Sec. 2.3: sum, min, max as the
 * aggregation kinds; Sec. 2.4: group by in the compiled program).  Groups
 * are the distinct keys; aggregate a of group g is, over the rows i with
 * keys[i] == g: SUM of vals[a][i] (wrapping int64), COUNT of rows, MIN or
 * MAX of vals[a][i].  Output is in ascending signed key order (reading: a
 * hash table has no order, so this is the canonical order both sides are
 * compared in).  Returns the number of groups.
 */
int64_t oracle_groupby(int64_t n, const int64_t *keys, int naggs,
                       const int *ops, const int64_t *const *vals,
                       int64_t *out_keys, int64_t *const *out_aggs)
{
    key_idx *r = (key_idx *)malloc((size_t)(n > 0 ? n : 1) * sizeof(key_idx));
    for (int64_t i = 0; i < n; i++) { r[i].key = keys[i]; r[i].idx = i; }
    qsort(r, (size_t)n, sizeof(key_idx), cmp_key_idx);
    int64_t ng = 0;
    for (int64_t s = 0; s < n; ) {
        int64_t e = s;
        while (e < n && r[e].key == r[s].key) e++;
        out_keys[ng] = r[s].key;
        for (int a = 0; a < naggs; a++) {
            uint64_t sum = 0;
            int64_t mn = INT64_MAX, mx = INT64_MIN;
            for (int64_t t = s; t < e; t++) {
                int64_t v = ops[a] == OR_COUNT ? 0 : vals[a][r[t].idx];
                sum += (uint64_t)v;
                if (v < mn) mn = v;
                if (v > mx) mx = v;
            }
            int64_t res = 0;
            if (ops[a] == OR_SUM) res = (int64_t)sum;
            else if (ops[a] == OR_COUNT) res = e - s;
            else if (ops[a] == OR_MIN) res = mn;
            else if (ops[a] == OR_MAX) res = mx;
            out_aggs[a][ng] = res;
        }
        ng++;
        s = e;
    }
    free(r);
    return ng;
}

/*
 * Average of each group (Sec. 2.3: average is one of the aggregation kinds
 * of the final reduction).  Reading: decimals are fixed-point int64, so the
 * exact aggregates are the int64 SUM and COUNT, and the average is derived
 * from them in FP64 as (double)sum / (double)count -- one rounding of the
 * sum to double, then one IEEE division.  Deriving it from SUM and COUNT
 * (never averaging partial averages) keeps it exact up to those two
 * roundings however the rows were split between blocks or GPUs.  A group
 * with count 0 gets 0/0 (NaN); groups of a group-by always have count >= 1.
 */
void oracle_avg(int64_t n, const int64_t *sum, const int64_t *count, double *out)
{
    for (int64_t g = 0; g < n; g++) out[g] = (double)sum[g] / (double)count[g];
}

/*
 * Group key of a joined row: (int64)hi << 32 | (uint32)lo when a high part
 * is given, else lo sign-extended (reading: the key packing is not in the
 * paper; two 32-bit attributes form one int64 key).
 */
int64_t oracle_group_key(int has_hi, int64_t hi, int64_t lo)
{
    if (!has_hi) return lo;
    return (int64_t)(((uint64_t)hi << 32) | (uint64_t)(uint32_t)lo);
}

/* Value fed to an aggregate: a, or a*b (wrapping) when b is given. */
static int64_t agg_value(const void *const *cols, const int *types, int a, int b, int64_t row)
{
    if (a < 0) return 0;
    uint64_t v = (uint64_t)col_get(cols[a], types[a], row);
    if (b >= 0) v *= (uint64_t)col_get(cols[b], types[b], row);
    return (int64_t)v;
}

/*
 * The operator pipeline (Sec. 2.4: one tensor program per GPU over its local
 * columns): group-by(join(filter(fact), dim)).
 *
 *   filter   : the fact-side conjunction of predicates;
 *   join     : fact column fk_col probes the dim (key -> payload) rows; when
 *              fk_col < 0 there is no join and the payload is absent;
 *              join_kind 0 is the inner join, 1 the semi-join (keep rows
 *              with a match) and 2 the anti-join (keep rows without one);
 *              the latter two carry no payload and allow repeated dim keys;
 *   group key: oracle_group_key over fact column key_hi_col (or none when
 *              < 0) and key_lo_col (a fact column, or the join payload when
 *              key_lo_col == -2);
 *   aggregate: agg_op[a] over fact columns agg_a[a] (times agg_b[a] when
 *              >= 0); COUNT takes no column.
 *
 * Output in ascending key order; returns the number of groups, -1 on a
 * duplicate build key of an inner join, or -2 when a semi- or anti-join asks
 * for the join payload as key.  out_nsel / out_njoin, when not NULL, receive the
 * row counts after the filter and after the join.
 */
int64_t oracle_pipeline(int64_t n_fact, const void *const *fact, const int *types,
                        int npreds, const int *pred_col, const int *pred_op,
                        const int64_t *lo, const int64_t *hi,
                        int fk_col, int64_t n_dim, const int32_t *dim_key,
                        const int32_t *dim_pay, int join_kind,
                        int key_hi_col, int key_lo_col,
                        int naggs, const int *agg_op, const int *agg_a, const int *agg_b,
                        int64_t *out_keys, int64_t *const *out_aggs,
                        int64_t *out_nsel, int64_t *out_njoin)
{
    if (fk_col >= 0 && join_kind != 0 && key_lo_col == -2) return -2;
    int32_t *sel = (int32_t *)malloc((size_t)(n_fact > 0 ? n_fact : 1) * sizeof(int32_t));
    int64_t nsel = oracle_filter(n_fact, fact, types, npreds, pred_col, pred_op, lo, hi, sel);
    int32_t *rows = sel, *pay = NULL;
    int64_t nj = nsel;
    if (fk_col >= 0 && join_kind != 0) {
        rows = (int32_t *)malloc((size_t)(nsel > 0 ? nsel : 1) * sizeof(int32_t));
        nj = oracle_semi_join(n_dim, dim_key, nsel, (const int32_t *)fact[fk_col], sel,
                              join_kind == 2, rows);
    } else if (fk_col >= 0) {
        rows = (int32_t *)malloc((size_t)(nsel > 0 ? nsel : 1) * sizeof(int32_t));
        pay = (int32_t *)malloc((size_t)(nsel > 0 ? nsel : 1) * sizeof(int32_t));
        int st = oracle_join(n_dim, dim_key, dim_pay, nsel, (const int32_t *)fact[fk_col],
                             sel, rows, pay, &nj);
        if (st != OR_OK) { free(sel); free(rows); free(pay); return -1; }
    }
    int64_t *keys = (int64_t *)malloc((size_t)(nj > 0 ? nj : 1) * sizeof(int64_t));
    int64_t *vals[8];
    for (int a = 0; a < naggs; a++)
        vals[a] = (int64_t *)malloc((size_t)(nj > 0 ? nj : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nj; i++) {
        int64_t row = rows[i];
        int64_t hiv = key_hi_col >= 0 ? col_get(fact[key_hi_col], types[key_hi_col], row) : 0;
        int64_t lov = key_lo_col == -2 ? (int64_t)pay[i]
                                       : col_get(fact[key_lo_col], types[key_lo_col], row);
        keys[i] = oracle_group_key(key_hi_col >= 0, hiv, lov);
        for (int a = 0; a < naggs; a++)
            vals[a][i] = agg_op[a] == OR_COUNT ? 0 : agg_value(fact, types, agg_a[a], agg_b[a], row);
    }
    int64_t ng = oracle_groupby(nj, keys, naggs, agg_op, (const int64_t *const *)vals,
                                out_keys, out_aggs);
    if (out_nsel) *out_nsel = nsel;
    if (out_njoin) *out_njoin = nj;
    for (int a = 0; a < naggs; a++) free(vals[a]);
    free(keys);
    if (rows != sel) free(rows);
    free(pay);
    free(sel);
    return ng;
}

/*
 * One output group of the pipeline, computed on its own over the whole
 * input: the aggregates of group `gkey` are accumulated row by row over the
 * fact rows that pass the predicates, join (join_kind as in
 * oracle_pipeline), and map to gkey.  Used for
 * sampled checks of results too large for the full oracle.  The join lookup
 * goes through the dim rows whose payload could produce gkey, sorted by key.
 * Returns the group's row count (0 when the group is absent).
 */
int64_t oracle_pipeline_group(int64_t n_fact, const void *const *fact, const int *types,
                              int npreds, const int *pred_col, const int *pred_op,
                              const int64_t *lo, const int64_t *hi,
                              int fk_col, int64_t n_dim, const int32_t *dim_key,
                              const int32_t *dim_pay, int join_kind,
                              int key_hi_col, int key_lo_col,
                              int naggs, const int *agg_op, const int *agg_a, const int *agg_b,
                              int64_t gkey, int64_t *out_aggs)
{
    /* dim rows whose payload matches the low half of gkey (all of them when
     * the low half does not come from the join) */
    build_row *b = (build_row *)malloc((size_t)(n_dim > 0 ? n_dim : 1) * sizeof(build_row));
    int64_t nb = 0;
    for (int64_t j = 0; j < n_dim; j++) {
        if (key_lo_col == -2) {
            int can_match = key_hi_col >= 0 ? (uint32_t)dim_pay[j] == (uint32_t)gkey
                                            : (int64_t)dim_pay[j] == gkey;
            if (!can_match) continue;
        }
        b[nb].key = dim_key[j];
        b[nb].payload = dim_pay ? dim_pay[j] : 0;
        nb++;
    }
    qsort(b, (size_t)nb, sizeof(build_row), cmp_build_row);
    uint64_t sum[8] = {0};
    int64_t mn[8], mx[8], count = 0;
    for (int a = 0; a < naggs; a++) { mn[a] = INT64_MAX; mx[a] = INT64_MIN; }
    for (int64_t i = 0; i < n_fact; i++) {
        int keep = 1;
        for (int p = 0; p < npreds && keep; p++) {
            int c = pred_col[p];
            keep = pred_holds(col_get(fact[c], types[c], i), pred_op[p], lo[p], hi[p]);
        }
        if (!keep) continue;
        int64_t payload = 0;
        if (fk_col >= 0) {
            int32_t k = ((const int32_t *)fact[fk_col])[i];
            int64_t l = 0, h = nb;
            while (l < h) {
                int64_t m = l + (h - l) / 2;
                if (b[m].key < k) l = m + 1; else h = m;
            }
            int found = l < nb && b[l].key == k;
            if (join_kind != 0) {
                if (found == (join_kind == 2)) continue;     /* semi: needs a match, anti: none */
            } else {
                if (!found) continue;
                payload = b[l].payload;
            }
        }
        int64_t hiv = key_hi_col >= 0 ? col_get(fact[key_hi_col], types[key_hi_col], i) : 0;
        int64_t lov = key_lo_col == -2 ? payload : col_get(fact[key_lo_col], types[key_lo_col], i);
        if (oracle_group_key(key_hi_col >= 0, hiv, lov) != gkey) continue;
        count++;
        for (int a = 0; a < naggs; a++) {
            int64_t v = agg_op[a] == OR_COUNT ? 0 : agg_value(fact, types, agg_a[a], agg_b[a], i);
            sum[a] += (uint64_t)v;
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    }
    for (int a = 0; a < naggs; a++) {
        if (agg_op[a] == OR_SUM) out_aggs[a] = (int64_t)sum[a];
        else if (agg_op[a] == OR_COUNT) out_aggs[a] = count;
        else if (agg_op[a] == OR_MIN) out_aggs[a] = mn[a];
        else out_aggs[a] = mx[a];
    }
    free(b);
    return count;
}
