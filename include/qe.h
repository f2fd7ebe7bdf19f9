/*
 * qe.h -- C ABI of libqe, a single-GPU relational operator library for
 * NVIDIA GB300 (sm_103a).
 *
 * It implements the per-GPU operator layer of the query engine in
 * "Terabyte-Scale Analytics in the Blink of an Eye" (arxiv 2506.09226): the
 * paper runs relational operators over one tensor per column on each GPU
 * (Sec. 2.1) and composes them into one program per GPU (Sec. 2.4).  The
 * operators here are selection with stream compaction, the radix/hash
 * partition that lays rows out per destination with start offsets (Sec. 2.2,
 * Fig. 1; Sec. 2.3), hash-join build and probe (Sec. 2.2), hash group-by with
 * exact SUM / COUNT / MIN / MAX (Sec. 2.3, Sec. 2.4), a fused pipeline of
 * them, and a batched form that runs many pipelines in one persistent launch.
 *
 * Conventions for every call
 *   - Memory: every column, selection vector and output buffer is a DEVICE
 *     pointer owned by the caller; no call keeps or frees a caller pointer.
 *     Columns may start at any address (unaligned views are read with scalar
 *     loads).  The library owns hash tables, batch plans and per-call scratch,
 *     which it allocates from the context's stream-ordered pool under the
 *     context's HBM budget.
 *   - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *     Calls enqueue work and return; outputs, counts included, are valid once
 *     the stream reaches that point.  Counts are written to device memory.
 *   - Errors: argument errors are returned at once as a qe_status and leave
 *     nothing enqueued.  Errors found by the kernels (output capacity too
 *     small, duplicate or reserved build key, a bounded device wait that
 *     expired) are recorded in the context; qe_sync_status() waits for the
 *     stream and returns and clears the first one.  qe_last_error() gives a
 *     message for the last non-OK status.
 *   - Sizes: row counts are int64_t; selection vectors and join outputs hold
 *     int32 row ids, so inputs that produce row ids are limited to
 *     nrows < 2^31.  Integer aggregates wrap modulo 2^64.
 *   - Threads: a context may be used from one host thread at a time.
 *     Different streams may run calls of one context concurrently.
 */
#ifndef QE_H
#define QE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QE_OK = 0,
    QE_ERR_INVALID_ARG = 1,   /* bad pointer, size, type or option           */
    QE_ERR_CAPACITY = 2,      /* output too small; required size recorded    */
    QE_ERR_OOM = 3,           /* HBM budget of the context exceeded          */
    QE_ERR_DUPLICATE_KEY = 4, /* join build saw a key twice                  */
    QE_ERR_RESERVED_KEY = 5,  /* key equal to the table's empty-slot marker  */
    QE_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up          */
    QE_ERR_CUDA = 7,          /* a CUDA runtime call failed                  */
    QE_ERR_NO_DEVICE = 8,     /* no usable sm_103a device                     */
    QE_ERR_DEVICE_CHECK = 9   /* a bounds check of the checked build failed  */
} qe_status;

/* Element type of a column; the value is the element size in bytes. */
typedef enum { QE_I8 = 1, QE_I32 = 4, QE_I64 = 8 } qe_type;

/* Column view: device pointer + element type.  When `gather` is nonzero the
 * column is read through a row-id list (element i is data[rows[i]]); the
 * calls that accept a row-id list say so. */
typedef struct {
    const void *data;
    int32_t type;     /* qe_type */
    int32_t gather;
} qe_col;

/* One comparison of a conjunctive selection predicate (Sec. 2.1).  The column
 * value, sign-extended to int64, is compared with lo (BETWEEN: lo <= x <= hi,
 * both inclusive). */
typedef enum { QE_LT = 0, QE_LE, QE_GT, QE_GE, QE_EQ, QE_NE, QE_BETWEEN } qe_cmp;
typedef struct {
    int32_t col;      /* index into the call's column array */
    int32_t op;       /* qe_cmp */
    int64_t lo, hi;
} qe_pred;

#define QE_MAX_COLS 8
#define QE_MAX_PREDS 4
#define QE_MAX_AGGS 4

/* Aggregates (Sec. 2.3 lists sum, min, max among the reduction kinds).  The
 * value of row i is column a, or a*b (int64, wrapping) when b is given;
 * COUNT takes no column. */
typedef enum { QE_SUM = 0, QE_COUNT = 1, QE_MIN = 2, QE_MAX = 3 } qe_agg_op;

/* Output of a group-by: one row per distinct key, in unspecified order.
 * keys and aggs[a] (for a < the number of aggregates) are device arrays of
 * `capacity` int64; *ngroups (device) receives the number of groups.  If the
 * groups exceed `capacity`, QE_ERR_CAPACITY is recorded with the number of
 * groups seen (a lower bound when the table overflowed) as the required
 * size, and only `capacity` rows are written.
 *
 * Averages (Sec. 2.3 lists average among the aggregation kinds of the final
 * reduction): avg[a] (nullable; device double [capacity]) asks for the
 * average of aggregate a, which must be a SUM, over the group's row count,
 * which some aggregate of the same call must provide as a COUNT:
 *     avg[a][g] = (double)aggs[a][g] / (double)count[g]
 * derived in FP64 from the exact int64 SUM and COUNT (one rounding of the
 * sum to double, one IEEE division), so the average of rows split across
 * blocks is exact to those two roundings.  A non-NULL avg[a] whose
 * aggregate is not a SUM, or with no COUNT among the aggregates, returns
 * QE_ERR_INVALID_ARG.  Entries a >= the number of aggregates must be NULL. */
typedef struct {
    int64_t capacity;
    int64_t *keys;
    int64_t *aggs[QE_MAX_AGGS];
    int64_t *ngroups;
    double *avg[QE_MAX_AGGS];
} qe_groups_out;

typedef struct qe_ctx qe_ctx;
typedef struct qe_hash_table qe_hash_table;
typedef struct qe_batch qe_batch;

/* ------------------------------------------------------------ context */

/* Create a context on CUDA device `device` (which must be sm_103a).  All
 * library-owned device memory of the context is capped at hbm_budget_bytes
 * (0 = no cap).  Returns QE_ERR_NO_DEVICE when the device is absent or not a
 * GB300-class part. */
qe_status qe_create(qe_ctx **out, int device, size_t hbm_budget_bytes);
qe_status qe_destroy(qe_ctx *ctx);

/* Message for the last non-OK status of this context (never NULL). */
const char *qe_last_error(const qe_ctx *ctx);

/* Wait for `stream`, then return and clear the first error the kernels
 * recorded since the last call.  *required (nullable) receives the size the
 * failing output needed (QE_ERR_CAPACITY) or 0. */
qe_status qe_sync_status(qe_ctx *ctx, void *stream, int64_t *required);

/* Device bytes currently held by library-owned objects of the context. */
size_t qe_bytes_in_use(const qe_ctx *ctx);

/* Host-side fault injection for tests: the n-th library allocation from now
 * (1 = the next one) fails with QE_ERR_OOM; n = 0 disables. */
void qe_debug_fail_alloc(qe_ctx *ctx, int n);

/* Limit, in iterations, of every bounded device-side wait of this context's
 * kernels (0 = the default).  Tests shorten it to make a wait expire. */
void qe_debug_set_spin_limit(qe_ctx *ctx, int64_t iterations);

/* Tuning knobs of the context (the autotuner sets them):
 *   "star_items"    rows per thread of the star-shape pipeline kernel: 2 or 3
 *                   (0 = default 3);
 *   "force_generic" nonzero: run every pipeline through the generic kernel.
 *   "part_general"  nonzero: qe_partition always uses its general scatter
 *                   kernel (chunks ranked over one or two digits, any
 *                   payload types, one pass at every fan-out) instead of the
 *                   write-combining one.
 *   "l2_hint"       nonzero: the star pipeline loads fact columns with an
 *                   L2 evict-first policy and looks payloads up with an
 *                   evict-last one (measured no faster; off by default).
 *   "gb_partition"  pipelines whose groups need an HBM hash table: 0 = the
 *                   partitioned group-by when that table would exceed 256 MB
 *                   and the fact table has 4M rows or more, 1 = never,
 *                   2 = always.
 *   "gb_part_log2p" / "gb_part_log2q"
 *                   log2 of the partitioned group-by's parts (1..10; 0 =
 *                   planned) and sub-parts per part (0..8; -1 = planned).
 *   "join_partition" join builds into tables of 256 MB or more: 0 = rows
 *                   reordered region by region (the top bits of the slot
 *                   they hash to) before the inserts for the multimap and
 *                   pair-key builds of 4M rows or more, input order
 *                   otherwise; 1 = always input order; 2 = always reordered
 *                   (every build kind).
 *   "join_part_log2" log2 of the regions of a reordered build (1..8; 0 =
 *                   planned: regions of about 32 MB).
 * Unknown names return QE_ERR_INVALID_ARG. */
qe_status qe_set_tuning(qe_ctx *ctx, const char *name, int64_t value);

/* Nonzero when this library is the bounds-checked build (libqe_checked.so,
 * compiled with QE_CHECKED): its kernels test the indices of their scatter
 * writes, segment ranges and shared-memory table slots against the bounds
 * they derive them from, and instead of an access out of bounds record
 * QE_ERR_DEVICE_CHECK (with the offending index as the required size) and
 * skip it.  It stands in for a memory checker; the plain build omits the
 * tests. */
int qe_build_checked(void);

/* Number of kernels this context has launched so far (host-side counter). */
int64_t qe_launch_count(const qe_ctx *ctx);

/* Per-kernel timing.  While enabled, the library brackets each launch of
 * its main kernels with CUDA events recorded on the launch stream.
 * qe_profile_read waits for those events and returns, for the kernel named
 * `name` ("filter", "probe", "build", "part_hist", "part_scatter", "groupby",
 * "pipeline", "batch"), the launches and their total device time in ms
 * since the last reset.  Unknown names give zero launches. */
qe_status qe_profile_enable(qe_ctx *ctx, int on);
qe_status qe_profile_read(qe_ctx *ctx, const char *name, int64_t *launches, double *total_ms);
qe_status qe_profile_reset(qe_ctx *ctx);

/* ------------------------------------------------------------ filter */

/* Selection with stable stream compaction (Sec. 2.1; the filters before a
 * join in Sec. 2.2's example).  A row i in [0, nrows) survives when every
 * predicate holds.  Writes the surviving row ids in ascending order to
 * out_sel[0 .. count) and count to *out_count (device int64).
 *   cols:   ncols column views (gather must be 0), each nrows long;
 *   preds:  npreds (0..QE_MAX_PREDS) comparisons over those columns;
 *   out_sel: device int32 [sel_capacity]; rows past the capacity are not
 *            written and QE_ERR_CAPACITY is recorded (required = count).
 * nrows must be < 2^31.  From 4M rows on the filter runs in two passes
 * (count per 512-row segment, then write), with scratch of about 8 bytes per
 * 512 rows from the context's budget. */
qe_status qe_filter(qe_ctx *ctx, const qe_col *cols, int ncols, const qe_pred *preds,
                    int npreds, int64_t nrows, int32_t *out_sel, int64_t sel_capacity,
                    int64_t *out_count, void *stream);

/* Largest nrows accepted by qe_filter_noalloc: 65,536 tiles of 4,096 rows. */
#define QE_FILTER_NOALLOC_MAX_ROWS (65536LL * 4096LL)

/* qe_filter without any device allocation.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory
 * from inside the call: a host whose device memory is entirely owned by its
 * own allocator (a library cudaMalloc would fail or fragment that pool), and
 * latency-critical callers that cannot afford an allocator call, which may
 * synchronize the device.  Arguments, result and errors are those of
 * qe_filter; the rows are computed by the one-pass compaction kernel (the
 * one qe_filter uses below 4M rows; above, qe_filter runs two passes with
 * allocated scratch).
 *
 * Its scratch (a tile counter and one look-back status word per 4,096-row
 * tile, about 512 KB) is a static device array inside libqe, which every GPU
 * that loads the library holds until the process exits.  The call clears the
 * part it uses before each launch, allocates and frees nothing, and rejects
 * nrows > QE_FILTER_NOALLOC_MAX_ROWS with QE_ERR_INVALID_ARG.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.  Every call shares the one array, so
 * calls whose work overlaps on the GPU (on different streams, or from
 * different contexts of one device) race: order them on one stream or
 * synchronize between them. */
qe_status qe_filter_noalloc(qe_ctx *ctx, const qe_col *cols, int ncols, const qe_pred *preds,
                            int npreds, int64_t nrows, int32_t *out_sel, int64_t sel_capacity,
                            int64_t *out_count, void *stream);

/* ------------------------------------------------------------ partition */

typedef enum {
    QE_PART_HASH = 0,  /* p = top log2_fanout bits of fmix64(key)           */
    QE_PART_RADIX = 1  /* p = (key >> shift) & (F - 1) on the key's 64 bits */
} qe_part_mode;

/* Radix / hash partition (Sec. 2.2, Fig. 1: every process applies the same
 * partitioning function to its rows; Sec. 2.3: the data for each destination
 * is one contiguous run per column, located by a start offset).  With
 * F = 2^log2_fanout destinations, row i goes to destination p(key_i); rows
 * keep their input order inside a destination (stable).  fmix64 is the
 * MurmurHash3 64-bit finalizer.
 *   keys:        device int64 [nrows];
 *   payload:     npayload (0..QE_MAX_COLS-1) columns of nrows (gather = 0);
 *   out_keys, out_payload[c]: device arrays of nrows, same types; must not
 *                overlap the inputs;
 *   out_offsets: device int64 [F + 1]; out_offsets[p] is the first output
 *                row of destination p, out_offsets[F] = nrows.
 * log2_fanout in [0, 12]; shift in [0, 63] (radix mode).
 * Scratch, taken from the context's HBM budget for the duration of the call:
 * per-block histograms and offsets (about 12 bytes x F x 304), and, when the
 * rows are int64 keys with one int64 payload or none and F > 64, a copy of
 * the keys and payload (16 bytes per row), because such fan-outs run as two
 * passes of at most 64 destinations each.  QE_ERR_OOM when the budget does
 * not hold it. */
qe_status qe_partition(qe_ctx *ctx, const int64_t *keys, const qe_col *payload, int npayload,
                       int64_t nrows, int log2_fanout, int mode, int shift, int64_t *out_keys,
                       void *const *out_payload, int64_t *out_offsets, void *stream);

/* ------------------------------------------------------------ join */

typedef enum {
    QE_HT_AUTO = 0,   /* dense when the key range is at most 4x the row count */
    QE_HT_DENSE = 1,  /* direct-mapped on key - key_min (perfect hash)        */
    QE_HT_OPEN = 2    /* open addressing, linear probing, 8-byte slots, CAS   */
} qe_ht_layout;

/* Optional build hints.  When have_range is nonzero, [key_min, key_max] is
 * a caller-known bound on the build keys (column statistics), so the build
 * needs no device-to-host read; a key outside it records
 * QE_ERR_INVALID_ARG.  When have_range is zero the build reads the key range
 * back from the device and synchronizes `stream` once. */
typedef struct {
    int32_t layout;       /* qe_ht_layout */
    int32_t have_range;
    int32_t key_min, key_max;
} qe_build_opts;

typedef struct {
    int32_t layout;       /* QE_HT_DENSE or QE_HT_OPEN */
    int32_t full;         /* dense table whose every slot is occupied */
    int64_t nkeys;        /* build rows (a key set counts repeats) */
    int64_t slots;
    int64_t bytes;
    int32_t key_min, key_max;
    int32_t have_payload_range;   /* payload range known (read back with the key range) */
    int32_t payload_min, payload_max;
    int32_t key_set;      /* 1: built by qe_join_build_set (membership only);
                             2: built by qe_join_build_multi (a multimap);
                             3: built by qe_join_build_pair (pair keys) */
} qe_ht_info;

/* Hash-join build (Sec. 2.2: the local join once both inputs are
 * co-located; Sec. 7.2 on build sizes).  Inserts key[j] -> payload[j] for
 * j < nrows into a library-owned table returned in *out.  Build keys must
 * be unique (QE_ERR_DUPLICATE_KEY is recorded otherwise).  For the
 * open-addressing layout INT32_MIN is the empty-slot marker and records
 * QE_ERR_RESERVED_KEY.  opts may be NULL (AUTO layout, range read back). */
qe_status qe_join_build(qe_ctx *ctx, const int32_t *keys, const int32_t *payload, int64_t nrows,
                        const qe_build_opts *opts, qe_hash_table **out, void *stream);

/* Hash-join probe (inner join).  For each probe position i < n in order,
 * row r = sel ? sel[i] : i is looked up with key probe_keys[r]; on a match
 * (r, payload) is appended; misses are dropped.  Output is in ascending
 * position order (stable compaction).
 *   out_probe_row, out_build_payload: device int32 [capacity];
 *   *out_count (device int64): number of matches; past the capacity nothing
 *   is written and QE_ERR_CAPACITY is recorded.
 * From 4M positions on the probe runs in two passes: the first looks every
 * position up once, counts matches per 256-position segment and keeps each
 * match's payload and every segment's match masks; the second writes them.
 * Scratch from the context's budget: about 4.2 bytes per position (0.2 for
 * qe_join_semi, which keeps the masks only). */
qe_status qe_join_probe(qe_ctx *ctx, const qe_hash_table *ht, const int32_t *probe_keys,
                        const int32_t *sel, int64_t n, int32_t *out_probe_row,
                        int32_t *out_build_payload, int64_t capacity, int64_t *out_count,
                        void *stream);

/* Key-set build for the semi- and anti-join: the EXISTS / NOT EXISTS forms
 * of the local join (Sec. 2.2) that the TPC-H queries the paper runs
 * (Sec. 6.1) contain.  Inserts key[j] for j < nrows; keys may repeat and no
 * payload is stored (a dense set is its occupancy bitmap alone, range/8
 * bytes).  opts as for qe_join_build (have_range skips the range read-back).
 * The open-addressing layout reserves INT32_MIN (QE_ERR_RESERVED_KEY).
 * A key set serves qe_join_semi and pipelines with a semi- or anti-join;
 * qe_join_probe rejects it (QE_ERR_INVALID_ARG: it has no payloads). */
qe_status qe_join_build_set(qe_ctx *ctx, const int32_t *keys, int64_t nrows, const qe_build_opts *opts,
                            qe_hash_table **out, void *stream);

/* Semi-join (anti = 0) or anti-join (anti = 1).  For each probe position
 * i < n in order, row r = sel ? sel[i] : i is kept when probe_keys[r] is
 * among the table's keys (semi) or is not (anti); the kept rows' ids are
 * written in ascending position order (stable compaction).  `ht` may be a
 * key set or a table from qe_join_build.
 *   out_rows: device int32 [capacity]; *out_count (device int64) receives
 *   the number of kept rows; past the capacity nothing is written and
 *   QE_ERR_CAPACITY is recorded.
 * From 4M positions on it runs in two passes, like qe_join_probe. */
qe_status qe_join_semi(qe_ctx *ctx, const qe_hash_table *ht, const int32_t *probe_keys, const int32_t *sel,
                       int64_t n, int anti, int32_t *out_rows, int64_t capacity, int64_t *out_count,
                       void *stream);

/* Many-to-many build (Sec. 2.2's local join when build keys repeat): a
 * multimap from key to the run of its build rows' payloads.  Every key
 * counts its rows (a dense slot key - key_min, or an open-addressing slot
 * holding the key and its count), a scan of the counts gives each key the
 * start of its run in one payload array, and a second pass places the rows;
 * the order of payloads inside a run is unspecified.  Layout and opts as for
 * qe_join_build (AUTO: dense when the key range is at most 4x the row count).
 * Memory: dense 12 bytes per key-range slot, open 20 bytes per slot (slots =
 * the power of two >= 2 x rows), plus 4 bytes per row; a probe reads one
 * 8-byte word (run start and length) per key.  The open layout
 * reserves INT32_MIN (QE_ERR_RESERVED_KEY).  A multimap serves only
 * qe_join_probe_multi (the other probes and the pipelines return
 * QE_ERR_INVALID_ARG for it). */
qe_status qe_join_build_multi(qe_ctx *ctx, const int32_t *keys, const int32_t *payload, int64_t nrows,
                              const qe_build_opts *opts, qe_hash_table **out, void *stream);

/* Many-to-many probe.  For each probe position i < n in order, row r = sel ?
 * sel[i] : i is looked up with key probe_keys[r]; each of the key's build
 * rows gives one output (r, payload).  Positions come out in ascending
 * order; the outputs of one position are in unspecified order.
 *   out_probe_row, out_build_payload: device int32 [capacity];
 *   *out_count (device int64): the number of outputs; past the capacity
 *   nothing is written and QE_ERR_CAPACITY is recorded with that number.
 * Two passes: the first looks every position up once, keeps its run (start,
 * length) and counts matches per segment of 256 positions; after a scan the
 * second writes the runs, a warp's outputs as consecutive stores.  Scratch:
 * 8 bytes per position plus 16 per segment. */
qe_status qe_join_probe_multi(qe_ctx *ctx, const qe_hash_table *ht, const int32_t *probe_keys,
                              const int32_t *sel, int64_t n, int32_t *out_probe_row,
                              int32_t *out_build_payload, int64_t capacity, int64_t *out_count,
                              void *stream);

/* Join on a pair of int32 key columns: the composite keys of joins such as a
 * (part, supplier) pair in the TPC-H queries the paper runs (Sec. 6.1),
 * joined locally as in Sec. 2.2.  The pair is packed as (uint32)hi << 32 |
 * (uint32)lo into an open-addressing table (load factor <= 0.5, 16-byte
 * slots holding key and payload); (INT32_MIN, INT32_MIN) is the empty-slot
 * marker and records
 * QE_ERR_RESERVED_KEY.  Build pairs must be unique (QE_ERR_DUPLICATE_KEY).
 * The probe matches row r = sel ? sel[i] : i on (probe_hi[r], probe_lo[r])
 * and writes (r, payload) in ascending position order, as qe_join_probe
 * (two passes from 4M positions on).  Pair-key tables serve only
 * qe_join_probe_pair. */
qe_status qe_join_build_pair(qe_ctx *ctx, const int32_t *key_hi, const int32_t *key_lo, const int32_t *payload,
                             int64_t nrows, qe_hash_table **out, void *stream);
qe_status qe_join_probe_pair(qe_ctx *ctx, const qe_hash_table *ht, const int32_t *probe_hi,
                             const int32_t *probe_lo, const int32_t *sel, int64_t n, int32_t *out_probe_row,
                             int32_t *out_build_payload, int64_t capacity, int64_t *out_count, void *stream);

qe_status qe_join_info(const qe_hash_table *ht, qe_ht_info *info);

/* Release the table once the work on `stream` that uses it is ordered
 * before this call. */
qe_status qe_join_destroy(qe_ctx *ctx, qe_hash_table *ht, void *stream);

/* ------------------------------------------------------------ group-by */

typedef struct {
    int32_t op;       /* qe_agg_op */
    int32_t pad;
    qe_col a, b;      /* b.data == NULL: value = a; else value = a * b */
} qe_agg;

typedef enum {
    QE_GB_AUTO = 0,   /* shared-memory tables when the capacity fits, else HBM */
    QE_GB_SMEM = 1,   /* per-block shared-memory table, spilling to HBM       */
    QE_GB_HBM = 2     /* HBM table only                                       */
} qe_gb_placement;

/* Hash group-by with exact aggregates (Sec. 2.3: sum, min and max as the
 * reduction kinds; Sec. 2.4: group-by in the per-GPU program).  For i < n,
 * the group key of row i is
 *     (int64)key_hi[i] << 32 | (uint32)key_lo[i]   when key_hi.data != NULL,
 *     (int64)key_lo[i]                             otherwise,
 * and each aggregate folds its value into the group.  Columns with gather
 * set are read at rows[i] (rows: device int32 [n], required then).
 *   placement: qe_gb_placement (AUTO picks by group_capacity);
 *   out: see qe_groups_out; out->capacity bounds the groups.
 * INT64_MIN is the table's empty-key marker and records
 * QE_ERR_RESERVED_KEY. */
qe_status qe_groupby(qe_ctx *ctx, int64_t n, const int32_t *rows, qe_col key_hi, qe_col key_lo,
                     const qe_agg *aggs, int naggs, int placement, const qe_groups_out *out,
                     void *stream);

/* ------------------------------------------------------------ pipeline */

#define QE_JOIN_PAYLOAD (-2)

/* Join of a pipeline: the inner join, or the semi- / anti-join that keeps
 * the fact rows whose foreign key has a match / has none (no payload). */
typedef enum { QE_JOIN_INNER = 0, QE_JOIN_SEMI = 1, QE_JOIN_ANTI = 2 } qe_join_kind;

typedef struct {
    int32_t op;       /* qe_agg_op */
    int32_t a, b;     /* fact column indices; -1 = absent */
    int32_t pad;
} qe_agg_spec;

/* One query of the paper's per-GPU shape (Sec. 2.4): a selection on the fact
 * table, an inner join of one fact column with a dimension table, and a
 * group-by with aggregates -- group-by(join(filter(fact), dim)).
 *   fact[0..n_fact_cols): fact columns, n_fact rows each (gather = 0);
 *   preds: conjunction over fact columns;
 *   fk_col: int32 fact column joined with the dimension keys, or -1 (no
 *           join);
 *   join_kind: qe_join_kind.  A semi- or anti-join has no payload (so
 *           key_lo_col may not be QE_JOIN_PAYLOAD), accepts repeated
 *           dimension keys, and takes dim_payload = NULL;
 *   dim_key/dim_payload/n_dim: dimension columns (device int32), built into a
 *           table by the call when ht is NULL (a key set for a semi- or
 *           anti-join); or a prebuilt resident table (a key set only with a
 *           semi- or anti-join);
 *   group key: key_hi_col (fact column or -1) and key_lo_col (fact column or
 *           QE_JOIN_PAYLOAD), packed as in qe_groupby;
 *   aggs: over fact columns.
 *   expected_groups: sizing hint for the group table (0 = use the output
 *           capacity); est_selectivity: hint in (0, 1] (0 = unknown). */
typedef struct {
    int64_t n_fact;
    qe_col fact[QE_MAX_COLS];
    int32_t n_fact_cols;
    int32_t n_preds;
    qe_pred preds[QE_MAX_PREDS];
    int32_t fk_col;
    int32_t key_hi_col;
    int32_t key_lo_col;
    int32_t n_aggs;
    qe_agg_spec aggs[QE_MAX_AGGS];
    const int32_t *dim_key;
    const int32_t *dim_payload;
    int64_t n_dim;
    const qe_hash_table *ht;
    qe_build_opts build;
    int64_t expected_groups;
    double est_selectivity;
    /* Optional bounds of the group key's parts (column statistics): when
     * have_key_range is nonzero, key_hi in [key_hi_min, key_hi_max] and
     * key_lo in [key_lo_min, key_lo_max] let the group table be a direct
     * (perfect-hash) array; rows outside the bounds still aggregate
     * correctly through the hash table.  Without it, a join-payload low part
     * takes its bounds from the join table when they are known. */
    int32_t have_key_range;
    int32_t join_kind;    /* qe_join_kind (0 = inner) */
    int64_t key_hi_min, key_hi_max, key_lo_min, key_lo_max;
} qe_pipeline_desc;

/* Run one pipeline: (build), then one fused pass over the fact table that
 * filters, probes and aggregates each row, then the group output.  Result
 * as in qe_groupby.  Groups are kept in a direct array indexed by the key's
 * parts when their ranges are known and small (in shared memory when it
 * fits), else in hash tables. */
qe_status qe_pipeline(qe_ctx *ctx, const qe_pipeline_desc *desc, const qe_groups_out *out,
                      void *stream);

/* ------------------------------------------------------------ batch */

/* Launch shape of a batch; zeros pick the tuned defaults. */
typedef struct {
    int32_t block_threads;   /* threads per block (multiple of 32) */
    int32_t tile_rows;       /* fact rows per work item            */
    int32_t smem_slots;      /* shared-memory group-table slots    */
    int32_t use_graph;       /* capture the launch in a CUDA graph */
    int64_t build_ahead_bytes;  /* join-table bytes built ahead of their
                                   probes (0 = 32 MB): the work items of a
                                   pipeline's in-kernel build are placed that
                                   far ahead of its probe items, so tables are
                                   probed while still in L2 */
} qe_batch_opts;

/* Plan a batch of n pipelines that share one persistent launch: every
 * pipeline's build, fused fact pass and group output run as work items of
 * one kernel, ordered per pipeline by device counters (bounded waits).  A
 * pipeline joins either a prebuilt resident table (desc.ht) or dimension
 * columns with build.have_range set (built inside the kernel, dense).  The
 * descs and outs are copied; the pointed-to device buffers must stay valid
 * until qe_batch_destroy.  Allocates all per-pipeline tables on `stream`
 * without synchronizing the host. */
qe_status qe_batch_create(qe_ctx *ctx, const qe_pipeline_desc *descs, const qe_groups_out *outs,
                          int n, const qe_batch_opts *opts, qe_batch **out, void *stream);

/* Run the planned batch on `stream` (through its CUDA graph when planned
 * with use_graph).  May be called repeatedly. */
qe_status qe_batch_launch(qe_ctx *ctx, qe_batch *batch, void *stream);

/* Synchronizes `stream`, then frees the batch. */
qe_status qe_batch_destroy(qe_ctx *ctx, qe_batch *batch, void *stream);

/* Plan, launch once and destroy. */
qe_status qe_batch_run(qe_ctx *ctx, const qe_pipeline_desc *descs, const qe_groups_out *outs,
                       int n, const qe_batch_opts *opts, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QE_H */
