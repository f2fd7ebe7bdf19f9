/*
 * qe_plan.h -- host-side exchange planner of libqe.
 *
 * Evaluates the analytical data-exchange models of "Terabyte-Scale Analytics
 * in the Blink of an Eye" (arxiv 2506.09226, Sec. 3) so that a distributed
 * query plan can choose how to bring join inputs together: keep co-partitioned
 * inputs local, broadcast the smaller table, or shuffle both (Sec. 3.4).
 *
 * Model (Sec. 3.1, Table 1): V machines of k GPUs each, N = k*V GPUs.  A
 * dataset of S bytes is spread S/N per GPU.  Machines are joined by a network
 * of unidirectional bandwidth B_n per machine; inside a machine a GPU sends to
 * its local peers at an aggregate rate B_g; the two kinds of transfer overlap.
 * Link speed may depend on the message size (Sec. 3.6, Hockney's model): an
 * m-byte message takes L + c*m seconds, so B(m) = m / (L + c*m).  A link of
 * constant bandwidth B is {L = 0, c = 1/B}; {0, 0} is an infinitely fast link.
 * Broadcast and shuffle carry separate link parameters because the paper fits
 * them separately (Sec. 3.6).
 *
 * Conventions for every call
 *   - No call touches a GPU or needs a context.  All pointers are HOST
 *     pointers owned by the caller; nothing is kept after a call returns.
 *   - Sizes are bytes and times seconds, as IEEE doubles.
 *   - Errors: a bad argument (NULL required pointer, k or V < 1, a negative,
 *     NaN or infinite size, time or link parameter, an unknown enum) returns
 *     QE_ERR_INVALID_ARG and writes no output; qe_plan_last_error() then
 *     describes it (per calling thread).
 *   - Threads: every call is reentrant.
 */
#ifndef QE_PLAN_H
#define QE_PLAN_H

#include "qe.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One link under Hockney's model (Sec. 3.6): an m-byte message takes
 * L + c*m seconds.  L >= 0 (seconds), c >= 0 (seconds per byte). */
typedef struct {
    double L;
    double c;
} qe_link;

/* A cluster of V machines with k GPUs each (Sec. 3.1). */
typedef struct {
    int32_t k;            /* GPUs per machine, >= 1 */
    int32_t V;            /* machines, >= 1 */
    qe_link bcast_net;    /* network link as seen by the broadcast (B_n)   */
    qe_link bcast_gpu;    /* intra-machine link as seen by the broadcast (B_g) */
    qe_link shuf_net;     /* network link as seen by the shuffle (B_n)     */
    qe_link shuf_gpu;     /* intra-machine link as seen by the shuffle (B_g) */
} qe_cluster;

typedef enum { QE_EXCH_BROADCAST = 0, QE_EXCH_SHUFFLE = 1 } qe_exchange;

typedef enum {
    QE_JOIN_LOCAL = 0,         /* co-partitioned inputs or one GPU: no exchange */
    QE_JOIN_BROADCAST_R = 1,   /* broadcast R (the smaller table, or equal size) */
    QE_JOIN_BROADCAST_S = 2,   /* broadcast S (strictly smaller than R)          */
    QE_JOIN_SHUFFLE_BOTH = 3   /* shuffle R and S                                */
} qe_join_strategy;

/* Time of one exchange of `bytes` bytes held bytes/N per GPU.
 *  QE_EXCH_BROADCAST (Sec. 3.2, Eq. 1): a ring of N-1 steps, each moving a
 *    bytes/N message over every hop; a hop runs at the slower of the network
 *    and intra-machine links, at B_g alone when V = 1, at B_n alone when
 *    k = 1 (no hop stays inside a machine):
 *    T = (N-1) * (bytes/N) / B(bytes/N).
 *  QE_EXCH_SHUFFLE (Sec. 3.3, Eq. 2): every GPU sends bytes/N^2 to every GPU;
 *    V >= 2: the network bounds it, T = bytes (V-1) / (V^2 B_n(bytes/N^2));
 *    V = 1:  T = bytes (N-1) / (N^2 B_g(bytes/N^2)).
 * N = 1 or bytes = 0 gives 0.  Throughput (the paper's Thpt) is bytes / T. */
qe_status qe_plan_exchange_time(const qe_cluster *cluster, int32_t op, double bytes, double *seconds);

/* Shuffle time under skew (Sec. 3.5.2).  With PXN, data leaves a machine
 * through any of its NICs, so only per-machine totals matter:
 *   S_i = sum over GPUs j of machine i, machines p != i, GPUs q of p of m_{ij->pq}
 *   R_i = the same sum of m_{pq->ij}
 *   T   = max(S_0..S_{V-1}, R_0..R_{V-1}) / B_n.
 * msg: N*N row-major bytes, msg[g*N + h] = bytes GPU g sends GPU h, with
 * g = machine*k + gpu (the sums of Sec. 3.5.2 index a GPU by machine first).
 * Entries >= 0.  bn: network bandwidth in bytes/s, > 0.  Requires V >= 2 (the
 * model covers the network only).  node_send / node_recv: NULL or V doubles,
 * receiving S_i / R_i. */
qe_status qe_plan_shuffle_skew(int32_t k, int32_t V, const double *msg, double bn, double *seconds,
                               double *node_send, double *node_recv);

/* Join strategy for tables of r_bytes and s_bytes (Sec. 3.4).
 * Broadcasting the smaller table costs one broadcast of it; shuffling both
 * costs one shuffle of each table.  The broadcast is chosen only when it is
 * strictly faster; with constant bandwidths and B_n <= B_g this is Eq. 3:
 * broadcast R iff |S|/|R| > (N-1)/(N-k) * V - 1, and |S|/|R| > N-1 when V = 1.
 * copartitioned != 0, or N = 1, gives QE_JOIN_LOCAL with both times 0.
 * r_msg / s_msg: NULL, or (V >= 2 only) an N*N message matrix as in
 * qe_plan_shuffle_skew whose entries sum to that table's size (to a relative
 * 1e-6, else QE_ERR_INVALID_ARG); the table's
 * shuffle is then timed by the skew model with B_n = the shuffle network link
 * read at the mean message size (sum / N^2).  Skew leaves the broadcast
 * unchanged (Sec. 3.5.1).  Outputs: strategy (qe_join_strategy); t_broadcast
 * and t_shuffle may be NULL. */
qe_status qe_plan_join(const qe_cluster *cluster, double r_bytes, double s_bytes, int32_t copartitioned,
                       const double *r_msg, const double *s_msg, int32_t *strategy, double *t_broadcast,
                       double *t_shuffle);

/* Fit Hockney parameters to n measured (bytes[i], seconds[i]) pairs of one
 * exchange `op` on a V x k cluster (Sec. 3.6).  The model time is linear in
 * (L, c), so this is an ordinary least-squares line through the points,
 * mapped back to (L, c).  At V = 1 the result is the intra-machine link, at
 * V >= 2 the network link (taken as the ring's bottleneck for a broadcast).
 * Requires N >= 2, n >= 2, bytes[i] > 0 and at least two distinct sizes.  A
 * fitted L may come out negative on noisy data; it is returned as fitted. */
qe_status qe_plan_fit_link(int32_t op, int32_t k, int32_t V, const double *bytes, const double *seconds,
                           int64_t n, qe_link *out);

/* Skew-gradient placement of the paper's skew experiments (Sec. 5, skew
 * case): GPU i of n_gpus holds x (1 + i f), x chosen so the sizes sum to
 * `total`.  f >= 0, total >= 0; sizes receives n_gpus doubles. */
qe_status qe_plan_skew_gradient(int32_t n_gpus, double f, double total, double *sizes);

/* Message of the last failed qe_plan_* call on this thread ("" if none). */
const char *qe_plan_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QE_PLAN_H */
