// Host-side exchange planner: the data-exchange cost models of Sec. 3
// (broadcast Eq. 1, shuffle Eq. 2, join choice Eq. 3, skew Sec. 3.5,
// Hockney message-size model Sec. 3.6).  Pure host arithmetic in double; no
// CUDA call.  Each time is computed as (messages on the bottleneck link) x
// (L + c*m), the per-message form of bytes / B(m).
#include <cmath>
#include <string>
#include <vector>

#include "qe_plan.h"

namespace {

thread_local std::string g_plan_error;

qe_status bad(const char *msg)
{
    g_plan_error = msg;
    return QE_ERR_INVALID_ARG;
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

bool link_ok(const qe_link &l) { return finite_nonneg(l.L) && finite_nonneg(l.c); }

bool cluster_ok(const qe_cluster *c)
{
    return c && c->k >= 1 && c->V >= 1 && link_ok(c->bcast_net) && link_ok(c->bcast_gpu) &&
           link_ok(c->shuf_net) && link_ok(c->shuf_gpu);
}

// Seconds one m-byte message occupies a link.
double msg_time(const qe_link &l, double m) { return l.L + l.c * m; }

// Eq. 1: N-1 ring steps, each a bytes/N message over every hop at once; the
// step lasts as long as the slowest kind of hop present in the ring.
double broadcast_seconds(int64_t k, int64_t V, double bytes, const qe_link &net, const qe_link &gpu)
{
    const int64_t N = k * V;
    if (N == 1 || bytes == 0.0) return 0.0;
    const double m = bytes / (double)N;
    double hop;
    if (V == 1) hop = msg_time(gpu, m);
    else if (k == 1) hop = msg_time(net, m);
    else hop = std::fmax(msg_time(net, m), msg_time(gpu, m));
    return (double)(N - 1) * hop;
}

// Eq. 2: each GPU sends bytes/N^2 to every GPU.  For V >= 2 each machine's
// NIC carries k*k*(V-1) of those messages; for V = 1 each GPU's local link
// carries N-1.
double shuffle_seconds(int64_t k, int64_t V, double bytes, const qe_link &net, const qe_link &gpu)
{
    const int64_t N = k * V;
    if (N == 1 || bytes == 0.0) return 0.0;
    const double m = bytes / ((double)N * (double)N);
    if (V == 1) return (double)(N - 1) * msg_time(gpu, m);
    return (double)(k * k * (V - 1)) * msg_time(net, m);
}

// Per-machine network totals of a message matrix (Sec. 3.5.2).
void node_totals(int64_t k, int64_t V, const double *msg, double *send, double *recv)
{
    const int64_t N = k * V;
    for (int64_t i = 0; i < V; i++) send[i] = recv[i] = 0.0;
    for (int64_t g = 0; g < N; g++) {
        const int64_t mg = g / k;
        for (int64_t h = 0; h < N; h++) {
            const int64_t mh = h / k;
            if (mg == mh) continue;
            send[mg] += msg[g * N + h];
            recv[mh] += msg[g * N + h];
        }
    }
}

bool matrix_ok(const double *msg, int64_t N, double *sum)
{
    double s = 0.0;
    for (int64_t i = 0; i < N * N; i++) {
        if (!finite_nonneg(msg[i])) return false;
        s += msg[i];
    }
    *sum = s;
    return true;
}

// Largest machine count whose N x N matrices and loops stay reasonable on
// the host (a 2^16-GPU cluster already needs a 32 GB matrix).
constexpr int64_t kMaxGpus = 1 << 16;

}  // namespace

extern "C" const char *qe_plan_last_error(void) { return g_plan_error.c_str(); }

extern "C" qe_status qe_plan_exchange_time(const qe_cluster *cluster, int32_t op, double bytes, double *seconds)
{
    if (!cluster_ok(cluster)) return bad("qe_plan_exchange_time: cluster is NULL or has k, V < 1 or a bad link");
    if (!seconds) return bad("qe_plan_exchange_time: seconds is NULL");
    if (!finite_nonneg(bytes)) return bad("qe_plan_exchange_time: bytes must be finite and >= 0");
    const int64_t k = cluster->k, V = cluster->V;
    if (op == QE_EXCH_BROADCAST) *seconds = broadcast_seconds(k, V, bytes, cluster->bcast_net, cluster->bcast_gpu);
    else if (op == QE_EXCH_SHUFFLE) *seconds = shuffle_seconds(k, V, bytes, cluster->shuf_net, cluster->shuf_gpu);
    else return bad("qe_plan_exchange_time: op must be QE_EXCH_BROADCAST or QE_EXCH_SHUFFLE");
    return QE_OK;
}

extern "C" qe_status qe_plan_shuffle_skew(int32_t k, int32_t V, const double *msg, double bn, double *seconds,
                                          double *node_send, double *node_recv)
{
    if (k < 1 || V < 2) return bad("qe_plan_shuffle_skew: needs k >= 1 and V >= 2");
    if ((int64_t)k * V > kMaxGpus) return bad("qe_plan_shuffle_skew: more than 65536 GPUs");
    if (!msg || !seconds) return bad("qe_plan_shuffle_skew: msg and seconds must not be NULL");
    if (!(std::isfinite(bn) && bn > 0.0)) return bad("qe_plan_shuffle_skew: bn must be finite and > 0");
    const int64_t N = (int64_t)k * V;
    double total;
    if (!matrix_ok(msg, N, &total)) return bad("qe_plan_shuffle_skew: message sizes must be finite and >= 0");
    std::vector<double> buf(2 * (size_t)V);
    double *send = buf.data(), *recv = send + V;
    node_totals(k, V, msg, send, recv);
    double mx = 0.0;
    for (int64_t i = 0; i < V; i++) mx = std::fmax(mx, std::fmax(send[i], recv[i]));
    *seconds = mx / bn;
    for (int64_t i = 0; i < V; i++) {
        if (node_send) node_send[i] = send[i];
        if (node_recv) node_recv[i] = recv[i];
    }
    return QE_OK;
}

extern "C" qe_status qe_plan_join(const qe_cluster *cluster, double r_bytes, double s_bytes, int32_t copartitioned,
                                  const double *r_msg, const double *s_msg, int32_t *strategy, double *t_broadcast,
                                  double *t_shuffle)
{
    if (!cluster_ok(cluster)) return bad("qe_plan_join: cluster is NULL or has k, V < 1 or a bad link");
    if (!strategy) return bad("qe_plan_join: strategy is NULL");
    if (!finite_nonneg(r_bytes) || !finite_nonneg(s_bytes))
        return bad("qe_plan_join: table sizes must be finite and >= 0");
    const int64_t k = cluster->k, V = cluster->V, N = k * V;
    if ((r_msg || s_msg) && V < 2) return bad("qe_plan_join: message matrices need V >= 2");
    if ((r_msg || s_msg) && N > kMaxGpus) return bad("qe_plan_join: more than 65536 GPUs");
    double msum[2] = {0.0, 0.0};
    const double *mats[2] = {r_msg, s_msg};
    const double sizes[2] = {r_bytes, s_bytes};
    for (int t = 0; t < 2; t++) {
        if (!mats[t]) continue;
        if (!matrix_ok(mats[t], N, &msum[t])) return bad("qe_plan_join: message sizes must be finite and >= 0");
        if (std::fabs(msum[t] - sizes[t]) > 1e-6 * std::fmax(msum[t], sizes[t]))
            return bad("qe_plan_join: a message matrix does not sum to its table's size");
    }

    if (copartitioned || N == 1) {
        *strategy = QE_JOIN_LOCAL;
        if (t_broadcast) *t_broadcast = 0.0;
        if (t_shuffle) *t_shuffle = 0.0;
        return QE_OK;
    }
    const bool r_small = r_bytes <= s_bytes;
    const double tb = broadcast_seconds(k, V, r_small ? r_bytes : s_bytes, cluster->bcast_net, cluster->bcast_gpu);
    double ts = 0.0;
    std::vector<double> buf(2 * (size_t)V);
    double *send = buf.data(), *recv = send + V;
    for (int t = 0; t < 2; t++) {
        if (!mats[t]) {
            ts += shuffle_seconds(k, V, sizes[t], cluster->shuf_net, cluster->shuf_gpu);
            continue;
        }
        if (msum[t] == 0.0) continue;
        // B_n at the mean message size, as seconds per byte: (L + c m) / m
        const double m = msum[t] / ((double)N * (double)N);
        const double sec_per_byte = msg_time(cluster->shuf_net, m) / m;
        node_totals(k, V, mats[t], send, recv);
        double mx = 0.0;
        for (int64_t i = 0; i < V; i++) mx = std::fmax(mx, std::fmax(send[i], recv[i]));
        ts += mx * sec_per_byte;
    }
    *strategy = tb < ts ? (r_small ? QE_JOIN_BROADCAST_R : QE_JOIN_BROADCAST_S) : QE_JOIN_SHUFFLE_BOTH;
    if (t_broadcast) *t_broadcast = tb;
    if (t_shuffle) *t_shuffle = ts;
    return QE_OK;
}

extern "C" qe_status qe_plan_fit_link(int32_t op, int32_t k, int32_t V, const double *bytes, const double *seconds,
                                      int64_t n, qe_link *out)
{
    if (op != QE_EXCH_BROADCAST && op != QE_EXCH_SHUFFLE) return bad("qe_plan_fit_link: unknown op");
    if (k < 1 || V < 1 || (int64_t)k * V < 2) return bad("qe_plan_fit_link: needs k, V >= 1 and N >= 2");
    if (!bytes || !seconds || !out) return bad("qe_plan_fit_link: NULL pointer");
    if (n < 2) return bad("qe_plan_fit_link: needs at least two measurements");
    for (int64_t i = 0; i < n; i++)
        if (!(std::isfinite(bytes[i]) && bytes[i] > 0.0) || !std::isfinite(seconds[i]))
            return bad("qe_plan_fit_link: sizes must be finite and > 0, times finite");
    const double N = (double)k * (double)V;
    // T = a*L + b*c*bytes for the link the exchange is charged to
    double a, b;
    if (op == QE_EXCH_BROADCAST) {
        a = N - 1.0;
        b = (N - 1.0) / N;
    } else if (V == 1) {
        a = N - 1.0;
        b = (N - 1.0) / (N * N);
    } else {
        a = (double)k * (double)k * (double)(V - 1);
        b = a / (N * N);
    }
    // least-squares line T = alpha + beta * bytes, with centred sums
    double mx = 0.0, my = 0.0;
    for (int64_t i = 0; i < n; i++) {
        mx += bytes[i];
        my += seconds[i];
    }
    mx /= (double)n;
    my /= (double)n;
    double sxx = 0.0, sxy = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double dx = bytes[i] - mx;
        sxx += dx * dx;
        sxy += dx * (seconds[i] - my);
    }
    if (!(sxx > 0.0)) return bad("qe_plan_fit_link: needs at least two distinct sizes");
    const double beta = sxy / sxx;
    const double alpha = my - beta * mx;
    out->L = alpha / a;
    out->c = beta / b;
    return QE_OK;
}

extern "C" qe_status qe_plan_skew_gradient(int32_t n_gpus, double f, double total, double *sizes)
{
    if (n_gpus < 1) return bad("qe_plan_skew_gradient: n_gpus must be >= 1");
    if (!finite_nonneg(f) || !finite_nonneg(total)) return bad("qe_plan_skew_gradient: f and total must be >= 0");
    if (!sizes) return bad("qe_plan_skew_gradient: sizes is NULL");
    // sum of (1 + i f) over i < n is n + f n (n-1) / 2
    const double n = (double)n_gpus;
    const double x = total / (n + f * n * (n - 1.0) * 0.5);
    for (int32_t i = 0; i < n_gpus; i++) sizes[i] = x * (1.0 + (double)i * f);
    return QE_OK;
}
