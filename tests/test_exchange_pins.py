"""Pins of the exchange-model oracle (oracle/exchange.py) against things
other than itself.

* Values and claims the paper prints (tests/golden/exchange_models.json): the
  skew-gradient placement of Sec. 5, the V = 1 join rule of Sec. 3.4, the
  skew claims of Sec. 5, the broadcast and shuffle trends of Sec. 3.2-3.3.
* Eq. 3, a closed form the oracle's planner never evaluates, against the
  planner's decision on both sides of the threshold.
* Independent accounting: the shuffle timed message by message per NIC and
  per local link under the assumptions of Sec. 3.1; the broadcast simulated
  ring step by ring step.
* The skew model (Sec. 3.5.2) with a uniform message matrix against Eq. 2.
* The Hockney fit against hand-derived linear forms and numpy.polyfit.

tests/test_exchange_mutants.py plants mistakes in copies of the oracle and
checks that this file catches each of them (QE_EXCHANGE_ORACLE names the
copy to load).
"""
import importlib.util
import json
import math
import os
import sys

import numpy as np
import pytest

_OVERRIDE = os.environ.get("QE_EXCHANGE_ORACLE")
if _OVERRIDE:
    _spec = importlib.util.spec_from_file_location("exchange_under_test", _OVERRIDE)
    X = importlib.util.module_from_spec(_spec)
    sys.modules["exchange_under_test"] = X
    _spec.loader.exec_module(X)
else:
    from oracle import exchange as X

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "exchange_models.json")))
GiB, MiB, GB = float(1 << 30), float(1 << 20), 1e9


def rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def const_cluster(k, V, Bn, Bg):
    n, g = X.constant(Bn), X.constant(Bg)
    return X.Cluster(k, V, n, g, n, g)


# ---------------------------------------------------------------- printed values and claims
def test_skew_gradient_worked_example():
    e = GOLD["skew_gradient"]
    N = e["k"] * e["V"]
    sizes = X.skew_gradient(N, e["f"], N * e["gib_per_gpu"] * GiB)
    assert round(sizes[0] / MiB) == e["first_mib_approx"]
    assert round(sizes[-1] / GiB, 2) == e["last_gib_approx"]
    assert rel(sum(sizes), N * GiB) < 1e-12
    flat = X.skew_gradient(N, 0.0, N * GiB)
    assert all(rel(s, e["f0_gib_each"] * GiB) < 1e-12 for s in flat)
    # the sizes step by f*x from x
    assert all(rel(sizes[i + 1] - sizes[i], e["f"] * sizes[0]) < 1e-9 for i in range(N - 1))


@pytest.mark.parametrize("k", GOLD["eq3_v1"]["ks"])
def test_join_rule_single_machine(k):
    cl = const_cluster(k, 1, 25 * GB, 400 * GB)
    R = 1e9
    above = X.plan_join(cl, R, (k - 1) * R * (1 + 1e-9))[0]
    below = X.plan_join(cl, R, (k - 1) * R * (1 - 1e-9))[0]
    assert above == X.BROADCAST_R
    assert below == X.SHUFFLE_BOTH
    # N = 2: the rule is |S| > |R|, so the smaller table is always broadcast; a tie shuffles
    cl2 = const_cluster(2, 1, 25 * GB, 400 * GB)
    assert X.plan_join(cl2, R, R * (1 + 1e-9))[0] == X.BROADCAST_R
    assert X.plan_join(cl2, R * (1 + 1e-9), R)[0] == X.BROADCAST_S
    assert X.plan_join(cl2, R, R)[0] == X.SHUFFLE_BOTH


def test_skew_claims_of_the_skew_experiment():
    e = GOLD["skew_claims"]
    k = e["k"]
    for V in e["Vs"]:
        N = k * V
        total = N * GiB
        t0 = X.shuffle_skew(k, V, X.uniform_messages([GiB] * N), 50 * GB)[0]
        for f in e["fs"]:
            sizes = X.skew_gradient(N, f, total)
            T, send, recv = X.shuffle_skew(k, V, X.uniform_messages(sizes), 50 * GB)
            assert int(np.argmax(send)) == V - 1          # last node sends the most
            assert int(np.argmax(recv)) == 0              # first node receives the most
            assert T > t0                                 # skew across VMs slows the shuffle
            # skew inside each VM only: x, x+fx, ..., x+(k-1)fx on every VM
            per_vm = X.skew_gradient(k, f, total / V)
            T_in, s_in, r_in = X.shuffle_skew(k, V, X.uniform_messages(per_vm * V), 50 * GB)
            assert rel(T_in, t0) < 1e-12
            assert all(rel(a, s_in[0]) < 1e-12 for a in s_in + r_in)


def test_broadcast_trend():
    e = GOLD["broadcast_trend"]
    k, Bg = e["k"], e["Bg_gbs"] * GB
    for Bn in (b * GB for b in e["Bn_gbs"]):
        th = [X.throughput(const_cluster(k, V, Bn, Bg), X.BROADCAST, 1e12) for V in range(2, 40)]
        assert all(a > b for a, b in zip(th, th[1:]))            # falls as V grows
        lim = X.throughput(const_cluster(k, 4000, Bn, Bg), X.BROADCAST, 1e12)
        assert rel(lim, min(Bn, Bg)) < 1e-4                       # converges to the ring's bottleneck
    lo = X.throughput(const_cluster(k, 4, e["Bn_gbs"][0] * GB, Bg), X.BROADCAST, 1e12)
    hi = X.throughput(const_cluster(k, 4, e["Bn_gbs"][1] * GB, Bg), X.BROADCAST, 1e12)
    assert rel(hi / lo, Bg / (e["Bn_gbs"][0] * GB)) < 1e-12      # the intra-VM link caps the gain


def test_shuffle_trend():
    e = GOLD["shuffle_trend"]
    k, Bg = e["k"], e["Bg_gbs"] * GB
    for Bn in (b * GB for b in e["Bn_gbs"]):
        th = [X.throughput(const_cluster(k, V, Bn, Bg), X.SHUFFLE, 1e12) for V in range(2, 40)]
        assert all(a < b for a, b in zip(th, th[1:]))             # grows with V for V >= 2
        th2 = X.throughput(const_cluster(k, 5, 2 * Bn, Bg), X.SHUFFLE, 1e12)
        assert rel(th2, 2 * X.throughput(const_cluster(k, 5, Bn, Bg), X.SHUFFLE, 1e12)) < 1e-12
        for V in (4, 16, 64):
            cl = const_cluster(k, V, Bn, Bg)
            ratio = X.throughput(cl, X.SHUFFLE, 1e12) / X.throughput(cl, X.BROADCAST, 1e12)
            assert V <= ratio <= V * V / (V - 1) * (1 + 1e-12)    # "almost V times"


# ---------------------------------------------------------------- Eq. 3
@pytest.mark.parametrize("k", [1, 2, 4, 8])
@pytest.mark.parametrize("V", [1, 2, 3, 5, 8])
def test_planner_matches_eq3(k, V):
    if k * V == 1:
        return
    N = k * V
    thr = (N - 1) / (N - k) * V - 1 if V > 1 else N - 1        # Eq. 3 as printed
    assert rel(X.eq3_threshold(k, V), thr) < 1e-15
    rng = np.random.default_rng(k * 100 + V)
    for _ in range(20):
        Bn = float(rng.uniform(5, 100)) * GB
        Bg = Bn * float(rng.uniform(1, 20))                      # the network is the slower link
        cl = const_cluster(k, V, Bn, Bg)
        R = float(rng.uniform(1e6, 1e11))
        assert X.plan_join(cl, R, R * thr * (1 + 1e-9))[0] == X.BROADCAST_R
        # thr = 1 only at N = 2, where |S| just below |R| makes S the broadcast side
        below = X.BROADCAST_S if N == 2 else X.SHUFFLE_BOTH
        assert X.plan_join(cl, R, R * thr * (1 - 1e-9))[0] == below


def test_planner_broadcasts_the_smaller_table_and_local_cases():
    cl = const_cluster(8, 4, 50 * GB, 400 * GB)
    s, tb, ts = X.plan_join(cl, 1e12, 1e9)
    assert s == X.BROADCAST_S
    assert rel(tb, X.broadcast_time(8, 4, 1e9, X.constant(50 * GB), X.constant(400 * GB))) < 1e-15
    assert X.plan_join(cl, 1e9, 1e12, copartitioned=True) == (X.LOCAL, 0.0, 0.0)
    assert X.plan_join(const_cluster(1, 1, GB, GB), 1e9, 1e12)[0] == X.LOCAL


# ---------------------------------------------------------------- independent accounting
def random_links(rng, hockney):
    """A network link and a faster local link (Sec. 3.1: local sends are faster)."""
    Ln = float(rng.uniform(1e-6, 1e-4)) if hockney else 0.0
    cn = 1.0 / (float(rng.uniform(5, 100)) * GB)
    net = X.Link(Ln, cn)
    gpu = X.Link(Ln * float(rng.uniform(0, 1)), cn * float(rng.uniform(0.02, 1)))
    return net, gpu


@pytest.mark.parametrize("hockney", [False, True])
def test_shuffle_against_per_message_accounting(hockney):
    """Every GPU sends S/N^2 to every GPU; remote messages queue on the
    sending and receiving machines' NICs, local ones on the sender's local
    link; a message costs L + c*m on its link; links run concurrently."""
    rng = np.random.default_rng(7 + hockney)
    for k in (1, 2, 4, 8):
        for V in (1, 2, 3, 5):
            N = k * V
            if N == 1:
                continue
            net, gpu = random_links(rng, hockney)
            S = float(rng.uniform(1e6, 1e12))
            m = S / N ** 2
            nic_out = [0.0] * V
            nic_in = [0.0] * V
            local = [0.0] * N
            for g in range(N):
                for h in range(N):
                    if g == h:
                        continue
                    if g // k != h // k:
                        nic_out[g // k] += net.L + net.c * m
                        nic_in[h // k] += net.L + net.c * m
                    else:
                        local[g] += gpu.L + gpu.c * m
            T = max(nic_out + nic_in + local)
            assert rel(X.shuffle_time(k, V, S, net, gpu), T) < 1e-12, (k, V)


@pytest.mark.parametrize("hockney", [False, True])
def test_broadcast_against_ring_simulation(hockney):
    """GPUs in a ring in machine order; in each of the steps every GPU
    forwards one S/N chunk to its successor and a step lasts as long as its
    slowest hop, a hop between machines running at B_n and one inside a
    machine at B_g; the broadcast ends when every GPU holds every chunk."""
    rng = np.random.default_rng(11 + hockney)
    for k in (1, 2, 4, 8):
        for V in (1, 2, 3, 5):
            N = k * V
            if N == 1:
                continue
            net, gpu = random_links(rng, hockney)
            if rng.uniform() < 0.5:
                net, gpu = gpu, net                              # either link may be the slower
            S = float(rng.uniform(1e6, 1e12))
            chunk = S / N
            have = [{g} for g in range(N)]
            T, s = 0.0, 0
            while any(len(h) < N for h in have):
                step, moves = 0.0, []
                for g in range(N):
                    c = (g - s) % N              # the chunk g received last (its own at the first step)
                    assert c in have[g]
                    h = (g + 1) % N
                    link = net if g // k != h // k else gpu
                    step = max(step, chunk / link.bw(chunk))
                    moves.append((h, c))
                for h, c in moves:
                    have[h].add(c)
                T += step
                s += 1
            assert s == N - 1
            assert rel(X.broadcast_time(k, V, S, net, gpu), T) < 1e-12, (k, V)


def test_skew_model_with_uniform_messages_is_eq2():
    rng = np.random.default_rng(3)
    for k in (1, 2, 8):
        for V in (2, 3, 6):
            N = k * V
            S = float(rng.uniform(1e9, 1e12))
            Bn = float(rng.uniform(5, 100)) * GB
            msg = [[S / N ** 2] * N for _ in range(N)]
            T, send, recv = X.shuffle_skew(k, V, msg, Bn)
            assert rel(T, S * (V - 1) / (V ** 2 * Bn)) < 1e-12      # Eq. 2 as printed: S / Thpt
            assert rel(T, X.shuffle_time(k, V, S, X.constant(Bn), X.constant(10 * Bn))) < 1e-12
            # every byte a machine sends another machine receives
            assert rel(sum(send), sum(recv)) < 1e-12


def test_skew_model_against_brute_force_matrix():
    """Per-machine send/receive totals of a random matrix, computed by masking
    the diagonal machine blocks out of numpy row/column sums."""
    rng = np.random.default_rng(5)
    for k, V in ((1, 3), (2, 2), (4, 3), (8, 4)):
        N = k * V
        M = rng.exponential(1e6, size=(N, N))
        T, send, recv = X.shuffle_skew(k, V, M.tolist(), 25 * GB)
        mach = np.arange(N) // k
        remote = mach[:, None] != mach[None, :]
        R = np.where(remote, M, 0.0)
        s_ref = np.bincount(mach, weights=R.sum(axis=1), minlength=V)
        r_ref = np.bincount(mach, weights=R.sum(axis=0), minlength=V)
        assert np.allclose(send, s_ref, rtol=1e-12)
        assert np.allclose(recv, r_ref, rtol=1e-12)
        assert rel(T, max(s_ref.max(), r_ref.max()) / (25 * GB)) < 1e-12


# ---------------------------------------------------------------- Hockney fit
def linear_form(op, k, V, S, L, c):
    """The model time written out by hand for a link (L, c)."""
    N = k * V
    if op == X.BROADCAST:
        return (N - 1) * (L + c * S / N)
    if V == 1:
        return (N - 1) * (L + c * S / N ** 2)
    return (V - 1) / V ** 2 * (N ** 2 * L + c * S)


@pytest.mark.parametrize("op", [0, 1])
def test_fit_recovers_link_and_matches_polyfit(op):
    rng = np.random.default_rng(op)
    for k, V in ((8, 1), (8, 2), (4, 4), (1, 3)):
        L, c = float(rng.uniform(1e-6, 1e-4)), 1.0 / (float(rng.uniform(5, 400)) * GB)
        sizes = [float(s) for s in np.geomspace(1e5, 1e11, 13)]
        times = [linear_form(op, k, V, S, L, c) for S in sizes]
        for S, t in zip(sizes, times):
            net = X.Link(L, c) if V > 1 else X.Link(0.0, 0.0)
            gpu = X.Link(L, c) if V == 1 else X.Link(0.0, 0.0)
            model = X.broadcast_time(k, V, S, net, gpu) if op == X.BROADCAST else X.shuffle_time(k, V, S, net, gpu)
            assert rel(model, t) < 1e-12
        got = X.fit_link(op, k, V, sizes, times)
        assert rel(got.L, L) < 1e-6 and rel(got.c, c) < 1e-9
        # noisy times: the least-squares line through (S, T), mapped back to (L, c)
        noisy = [t * float(rng.uniform(0.9, 1.1)) for t in times]
        slope, icpt = np.polyfit(sizes, noisy, 1)
        a = linear_form(op, k, V, 0.0, 1.0, 0.0)
        b = linear_form(op, k, V, 1.0, 0.0, 1.0)
        got = X.fit_link(op, k, V, sizes, noisy)
        assert rel(got.c, slope / b) < 1e-6
        assert abs(got.L - icpt / a) < 1e-6 * abs(icpt / a) + 1e-12


def test_link_bandwidth_limits():
    ln = X.Link(1e-5, 1.0 / (50 * GB))
    assert rel(ln.bw(1e15), 50 * GB) < 1e-4                    # large messages: 1/c
    assert rel(ln.bw(1.0) * 1e-5, 1.0) < 1e-4                  # small messages: m/L
    assert rel(X.constant(7 * GB).bw(123.0), 7 * GB) < 1e-15
