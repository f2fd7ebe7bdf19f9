"""CPU oracle for the data-exchange cost models of Sec. 3 (arxiv 2506.09226).

TEST INFRASTRUCTURE ONLY: the test-suite is the only caller.  Plain Python
floats (IEEE fp64), no vectorisation, written in the order and notation of
the paper.  It shares no code with the planner in the operator library.

Notation (Sec. 3.1, Table 1): k GPUs per machine, V machines, N = k*V GPUs,
B_n the unidirectional network bandwidth of one machine, B_g the aggregate
rate at which one GPU sends to its local peers, S the total bytes exchanged
(spread evenly over the N GPUs unless a message matrix says otherwise).

Message-size dependence (Sec. 3.6, Hockney's model): an m-byte message over
a link takes L + c*m seconds, so the link's effective bandwidth is
B(m) = m / (L + c*m).  A constant bandwidth B is the link L = 0, c = 1/B.
Broadcast and shuffle have separate link parameters because the paper fits
them separately.

Readings where the paper is silent or inconsistent:
* m_{ij->pq}: Table 1 names G_ij the i-th GPU of machine j, but the per-node
  sums of Sec. 3.5.2 let the first index run over machines and the second
  over GPUs; the oracle follows the sums (i, p machines; j, q GPUs) and
  stores the matrix with flat GPU index g = machine*k + gpu.
* Message sizes: a broadcast moves S/N per ring step (Sec. 3.2), a shuffle
  moves S/N^2 per GPU pair (Sec. 3.3); those are the m at which B(m) is read.
* Shuffle-both costs one shuffle of R and one of S (Sec. 3.4); with constant
  bandwidth their sum is the paper's (V-1)/(V^2 B_n) (|R|+|S|).
* Broadcast is charged to the smaller table (Sec. 3.4 assumes |R| <= |S|);
  broadcast is chosen only when strictly faster than shuffle.
* With one GPU per machine (k = 1) no ring hop stays inside a machine, so
  the broadcast runs at B_n alone (Eq. 1 takes min(B_n, B_g) for V > 1).
* The skewed shuffle (Sec. 3.5.2) models the network only and needs V >= 2;
  its B_n is the shuffle network link read at the mean message size.
* Fitting (Sec. 3.6): at V = 1 the measurements fit the GPU link, at V >= 2
  the network link (taken as the bottleneck of the broadcast ring).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BROADCAST, SHUFFLE = 0, 1
LOCAL, BROADCAST_R, BROADCAST_S, SHUFFLE_BOTH = 0, 1, 2, 3


@dataclass
class Link:
    """Hockney link: an m-byte message takes L + c*m seconds (Sec. 3.6)."""
    L: float = 0.0
    c: float = 0.0

    def bw(self, m: float) -> float:
        d = self.L + self.c * m
        return math.inf if d == 0.0 else m / d


def constant(B: float) -> Link:
    """A link of bandwidth B bytes/s independent of message size (Sec. 3.1)."""
    return Link(0.0, 1.0 / B)


@dataclass
class Cluster:
    k: int
    V: int
    bcast_net: Link
    bcast_gpu: Link
    shuf_net: Link
    shuf_gpu: Link


def broadcast_time(k: int, V: int, S: float, net: Link, gpu: Link) -> float:
    """Ring broadcast of S bytes held S/N per GPU (Sec. 3.2, Eq. 1).

    N-1 steps, each moving S/N over every hop of the ring; a hop runs at the
    slower of the network and the intra-machine link, at B_g alone when
    V = 1 and at B_n alone when k = 1 (no hop stays inside a machine)."""
    N = k * V
    if N == 1 or S == 0.0:
        return 0.0
    m = S / N
    if V == 1:
        B = gpu.bw(m)
    elif k == 1:
        B = net.bw(m)
    else:
        B = min(net.bw(m), gpu.bw(m))
    return (N - 1) * (S / N) / B


def shuffle_time(k: int, V: int, S: float, net: Link, gpu: Link) -> float:
    """All-to-all shuffle of S bytes held S/N per GPU (Sec. 3.3, Eq. 2).

    Each GPU sends S/N^2 to every GPU.  For V >= 2 the remote sends bound
    the time: every machine pushes (V-1) k^2 messages through B_n, so
    T = S (V-1) / (V^2 B_n).  For V = 1 each GPU sends N-1 messages at B_g:
    T = S (N-1) / (N^2 B_g)."""
    N = k * V
    if N == 1 or S == 0.0:
        return 0.0
    m = S / (N * N)
    if V == 1:
        return S * (N - 1) / (N * N * gpu.bw(m))
    return S * (V - 1) / (V * V * net.bw(m))


def exchange_time(cl: Cluster, op: int, S: float) -> float:
    if op == BROADCAST:
        return broadcast_time(cl.k, cl.V, S, cl.bcast_net, cl.bcast_gpu)
    return shuffle_time(cl.k, cl.V, S, cl.shuf_net, cl.shuf_gpu)


def throughput(cl: Cluster, op: int, S: float) -> float:
    """S / T, the throughput the paper plots (Sec. 3.1)."""
    T = exchange_time(cl, op, S)
    return math.inf if T == 0.0 else S / T


def eq3_threshold(k: int, V: int) -> float:
    """|S|/|R| above which broadcasting R beats shuffling both (Sec. 3.4,
    Eq. 3); N - 1 when V = 1.  Holds for constant bandwidths with the
    network the slower link."""
    N = k * V
    if V == 1:
        return float(N - 1)
    return (N - 1) / (N - k) * V - 1


def shuffle_skew(k: int, V: int, msg, Bn: float):
    """Shuffle time under skew (Sec. 3.5.2): with PXN only per-machine totals
    matter.  msg[g][h] is m_{ij->pq} with g = i*k + j, h = p*k + q.

    Returns (T, send, recv) with send[i] = S_i, recv[i] = R_i and
    T = max(S_0..S_{V-1}, R_0..R_{V-1}) / B_n."""
    send = [0.0] * V
    recv = [0.0] * V
    for i in range(V):
        for j in range(k):
            for p in range(V):
                if p == i:
                    continue
                for q in range(k):
                    send[i] += msg[i * k + j][p * k + q]
                    recv[i] += msg[p * k + q][i * k + j]
    return max(send + recv) / Bn, send, recv


def plan_join(cl: Cluster, r_bytes: float, s_bytes: float, copartitioned: bool = False,
              r_msg=None, s_msg=None):
    """Join strategy (Sec. 3.4): broadcast the smaller table, or shuffle both.

    Returns (strategy, T_broadcast, T_shuffle).  A co-partitioned input or a
    single GPU needs no exchange.  When a table's message matrix is given
    (V >= 2) its shuffle is timed by the skew model (Sec. 3.5.2); skew does
    not change the broadcast (Sec. 3.5.1)."""
    k, V = cl.k, cl.V
    N = k * V
    if copartitioned or N == 1:
        return LOCAL, 0.0, 0.0
    small = min(r_bytes, s_bytes)
    t_b = broadcast_time(k, V, small, cl.bcast_net, cl.bcast_gpu)
    t_s = 0.0
    for size, msg in ((r_bytes, r_msg), (s_bytes, s_msg)):
        if msg is None:
            t_s += shuffle_time(k, V, size, cl.shuf_net, cl.shuf_gpu)
        else:
            total = sum(sum(row) for row in msg)
            if total > 0.0:
                Bn = cl.shuf_net.bw(total / (N * N))
                t_s += shuffle_skew(k, V, msg, Bn)[0]
    if t_b < t_s:
        return (BROADCAST_R if r_bytes <= s_bytes else BROADCAST_S), t_b, t_s
    return SHUFFLE_BOTH, t_b, t_s


def fit_link(op: int, k: int, V: int, sizes, times) -> Link:
    """Hockney parameters from measured (bytes, seconds) of one exchange at
    one cluster shape (Sec. 3.6).  The model time is linear in (L, c), so
    its columns are the model evaluated at (1, 0) and (0, 1); least squares
    via numpy.linalg.lstsq."""
    unit_L, unit_c, free = Link(1.0, 0.0), Link(0.0, 1.0), Link(0.0, 0.0)
    rows = []
    for S in sizes:
        if op == BROADCAST:
            if V == 1:
                a = broadcast_time(k, V, S, free, unit_L)
                b = broadcast_time(k, V, S, free, unit_c)
            else:
                a = broadcast_time(k, V, S, unit_L, free)
                b = broadcast_time(k, V, S, unit_c, free)
        else:
            a = shuffle_time(k, V, S, unit_L, unit_L)
            b = shuffle_time(k, V, S, unit_c, unit_c)
        rows.append([a, b])
    sol = np.linalg.lstsq(np.array(rows, dtype=np.float64), np.array(times, dtype=np.float64), rcond=None)[0]
    return Link(float(sol[0]), float(sol[1]))


def skew_gradient(n_gpus: int, f: float, total: float):
    """Initial placement of the skew experiments (Sec. 5, skew case): GPU i holds
    x (1 + i f), with x chosen so the sizes add up to total."""
    x = total / sum(1.0 + i * f for i in range(n_gpus))
    return [x * (1.0 + i * f) for i in range(n_gpus)]


def uniform_messages(sizes):
    """Each GPU sends the same amount to every GPU (Sec. 5, skew case): m_g->h = size_g / N."""
    N = len(sizes)
    return [[sizes[g] / N for _ in range(N)] for g in range(N)]
