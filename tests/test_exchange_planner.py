"""Parity of the library's exchange planner (include/qe_plan.h, host code in
libqe) with the exchange-model oracle (oracle/exchange.py) on seeded random
clusters, links, sizes and message matrices, plus its argument checks.

Both sides compute in fp64 with different operation orders, so times agree
to a relative 1e-12; the join decision is compared wherever the two times
differ by more than a relative 1e-9 (nearer ties may round either way), and
exact ties are checked separately.
"""
import ctypes
import math
import os

import numpy as np
import pytest

from oracle import exchange as X
from paper_2506_09226_gb300 import qe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2506_09226_gb300", "libqe.so")
GB = 1e9
RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(LIB):
        from paper_2506_09226_gb300 import build
        build.build()
    return qe.load_library()


def rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def rand_link(rng, kind):
    if kind == "zero":
        return 0.0, 0.0
    c = 1.0 / (float(rng.uniform(1, 1000)) * GB)
    L = float(rng.uniform(1e-7, 1e-3)) if kind == "hockney" else 0.0
    return L, c


def rand_cluster(rng, k=None, V=None):
    k = int(rng.integers(1, 17)) if k is None else k
    V = int(rng.integers(1, 13)) if V is None else V
    kinds = ["constant", "hockney", "hockney", "zero"]
    links = [rand_link(rng, kinds[int(rng.integers(0, 4)) if rng.uniform() < 0.1 else int(rng.integers(0, 3))])
             for _ in range(4)]
    c_cl = qe.qe_cluster(k, V, *[qe.qe_link(*l) for l in links])
    o_cl = X.Cluster(k, V, *[X.Link(*l) for l in links])
    return c_cl, o_cl


def rand_bytes(rng):
    r = rng.uniform()
    if r < 0.05:
        return 0.0
    return float(10 ** rng.uniform(0, 13))


def test_exchange_time_matches_oracle():
    rng = np.random.default_rng(1)
    for _ in range(3000):
        c_cl, o_cl = rand_cluster(rng)
        S = rand_bytes(rng)
        for op in (X.BROADCAST, X.SHUFFLE):
            got = qe.qe_plan_exchange_time(c_cl, op, S)
            ref = X.exchange_time(o_cl, op, S)
            assert rel(got, ref) < RTOL, (c_cl.k, c_cl.V, S, op, got, ref)


@pytest.mark.parametrize("k,V", [(1, 1), (4, 1), (1, 6), (8, 2), (8, 5)])
def test_exchange_time_edges(k, V):
    rng = np.random.default_rng(k * 10 + V)
    c_cl, o_cl = rand_cluster(rng, k, V)
    for op in (0, 1):
        assert qe.qe_plan_exchange_time(c_cl, op, 0.0) == 0.0
        if k * V == 1:
            assert qe.qe_plan_exchange_time(c_cl, op, 1e12) == 0.0
    # infinitely fast links take no time
    z = qe.qe_cluster(k, V, *[qe.qe_link(0.0, 0.0)] * 4)
    assert qe.qe_plan_exchange_time(z, 0, 1e12) == 0.0
    assert qe.qe_plan_exchange_time(z, 1, 1e12) == 0.0


def rand_matrix(rng, N, total=None):
    kind = int(rng.integers(0, 4))
    if kind == 0:
        M = rng.exponential(1e6, size=(N, N))
    elif kind == 1:                                   # sparse, some zero rows
        M = rng.exponential(1e6, size=(N, N)) * (rng.uniform(size=(N, N)) < 0.3)
        M[rng.integers(0, N)] = 0.0
    elif kind == 2:                                   # skew-gradient placement, equal sends
        f = float(rng.uniform(0, 4))
        M = np.array(X.uniform_messages(X.skew_gradient(N, f, float(N) * 2 ** 30)))
    else:                                             # one hot sender
        M = np.zeros((N, N))
        M[rng.integers(0, N)] = rng.uniform(1e3, 1e9, size=N)
    if M.sum() == 0:
        M = np.ones((N, N))
    if total is not None:
        M *= total / M.sum()
    return M


def test_shuffle_skew_matches_oracle():
    rng = np.random.default_rng(2)
    for _ in range(400):
        k, V = int(rng.integers(1, 9)), int(rng.integers(2, 7))
        N = k * V
        M = rand_matrix(rng, N)
        bn = float(rng.uniform(1, 500)) * GB
        t, s, r = qe.qe_plan_shuffle_skew(k, V, M, bn)
        T, s_ref, r_ref = X.shuffle_skew(k, V, M.tolist(), bn)
        assert rel(t, T) < RTOL
        assert np.allclose(s, s_ref, rtol=RTOL, atol=0) and np.allclose(r, r_ref, rtol=RTOL, atol=0)


def test_plan_join_matches_oracle():
    rng = np.random.default_rng(3)
    compared = 0
    for i in range(3000):
        c_cl, o_cl = rand_cluster(rng)
        N = c_cl.k * c_cl.V
        R, S = rand_bytes(rng), rand_bytes(rng)
        copart = rng.uniform() < 0.05
        rm = sm = None
        if c_cl.V >= 2 and N <= 64 and rng.uniform() < 0.3:
            rm = rand_matrix(rng, N, R) if R > 0 else np.zeros((N, N))
            if rng.uniform() < 0.5:
                sm = rand_matrix(rng, N, S) if S > 0 else np.zeros((N, N))
        got = qe.qe_plan_join(c_cl, R, S, copart, rm, sm)
        ref = X.plan_join(o_cl, R, S, copart, None if rm is None else rm.tolist(),
                          None if sm is None else sm.tolist())
        assert rel(got[1], ref[1]) < RTOL and rel(got[2], ref[2]) < RTOL, (i, got, ref)
        if abs(ref[1] - ref[2]) > 1e-9 * max(ref[1], ref[2]) or ref[0] == X.LOCAL:
            assert got[0] == ref[0], (i, got, ref)
            compared += 1
        else:
            assert got[0] in (X.SHUFFLE_BOTH, X.BROADCAST_R if R <= S else X.BROADCAST_S)
    assert compared > 2900


def test_plan_join_eq3_and_ties():
    # constant links with the network slower: the decision is Eq. 3
    for k in (1, 2, 4, 8):
        for V in (1, 2, 3, 6):
            if k * V == 1:
                continue
            cl = qe.cluster(k, V, qe.link(40 * GB), qe.link(320 * GB))
            thr = X.eq3_threshold(k, V)
            R = 3e9
            assert qe.qe_plan_join(cl, R, R * thr * (1 + 1e-9))[0] == qe.JOIN_BROADCAST_R
            below = qe.JOIN_BROADCAST_S if k * V == 2 else qe.JOIN_SHUFFLE_BOTH
            assert qe.qe_plan_join(cl, R, R * thr * (1 - 1e-9))[0] == below
    # an exact tie shuffles: zero-size tables, and equal tables on two GPUs with power-of-two sizes
    cl = qe.cluster(2, 1, qe.link(L=0.0, c=2.0 ** -33), qe.link(L=0.0, c=2.0 ** -35))
    st, tb, ts = qe.qe_plan_join(cl, 2.0 ** 30, 2.0 ** 30)
    assert tb == ts and st == qe.JOIN_SHUFFLE_BOTH
    assert qe.qe_plan_join(cl, 0.0, 0.0)[0] == qe.JOIN_SHUFFLE_BOTH
    assert qe.qe_plan_join(cl, 1e9, 1e12, copartitioned=True) == (qe.JOIN_LOCAL, 0.0, 0.0)


def test_fit_link_matches_oracle():
    rng = np.random.default_rng(4)
    for _ in range(300):
        op = int(rng.integers(0, 2))
        k, V = int(rng.integers(1, 9)), int(rng.integers(1, 6))
        if k * V == 1:
            continue
        L, c = float(rng.uniform(1e-6, 1e-4)), 1.0 / (float(rng.uniform(5, 400)) * GB)
        n = int(rng.integers(2, 20))
        sizes = np.geomspace(float(10 ** rng.uniform(2, 6)), float(10 ** rng.uniform(7, 11)), n)
        net = X.Link(L, c) if V > 1 else X.Link(0.0, 0.0)
        gpu = X.Link(L, c) if V == 1 else X.Link(0.0, 0.0)
        f = X.broadcast_time if op == X.BROADCAST else X.shuffle_time
        times = np.array([f(k, V, float(s), net, gpu) for s in sizes]) * rng.uniform(0.95, 1.05, n)
        got = qe.qe_plan_fit_link(op, k, V, sizes, times)
        ref = X.fit_link(op, k, V, sizes.tolist(), times.tolist())
        assert rel(got.c, ref.c) < 1e-8
        scale = abs(ref.L) + c * float(sizes.mean())
        assert abs(got.L - ref.L) < 1e-8 * scale


def test_skew_gradient_matches_oracle():
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(1, 300))
        f = float(rng.uniform(0, 10)) if rng.uniform() < 0.9 else 0.0
        total = float(10 ** rng.uniform(0, 14))
        got = qe.qe_plan_skew_gradient(n, f, total)
        ref = X.skew_gradient(n, f, total)
        assert np.allclose(got, ref, rtol=1e-13, atol=0)


# ---------------------------------------------------------------- argument checks
def _raises_invalid(fn, *a, **kw):
    with pytest.raises(qe.QeError) as e:
        fn(*a, **kw)
    assert e.value.status == qe.ERR_INVALID_ARG
    assert str(e.value).split(": ", 1)[1]          # a message from qe_plan_last_error


def test_invalid_arguments_are_rejected(lib):
    good = qe.cluster(4, 2, qe.link(50 * GB), qe.link(400 * GB))
    for k, V in ((0, 2), (2, 0), (-1, 3)):
        _raises_invalid(qe.qe_plan_exchange_time, qe.qe_cluster(k, V, good.bcast_net, good.bcast_gpu,
                                                                good.shuf_net, good.shuf_gpu), 0, 1e9)
    for bad in (-1.0, math.nan, math.inf):
        _raises_invalid(qe.qe_plan_exchange_time, good, 0, bad)
        _raises_invalid(qe.qe_plan_join, good, bad, 1e9)
        b = qe.cluster(4, 2, qe.qe_link(bad, 1e-9), qe.link(400 * GB))
        _raises_invalid(qe.qe_plan_exchange_time, b, 1, 1e9)
    _raises_invalid(qe.qe_plan_exchange_time, good, 2, 1e9)
    # skew model: V >= 2, bn > 0, entries >= 0
    _raises_invalid(qe.qe_plan_shuffle_skew, 4, 1, np.ones((4, 4)), GB)
    _raises_invalid(qe.qe_plan_shuffle_skew, 2, 2, np.ones((4, 4)), 0.0)
    m = np.ones((4, 4))
    m[1, 2] = -1.0
    _raises_invalid(qe.qe_plan_shuffle_skew, 2, 2, m, GB)
    # join: matrices only for V >= 2 and summing to the table size
    one = qe.cluster(4, 1, qe.link(50 * GB), qe.link(400 * GB))
    _raises_invalid(qe.qe_plan_join, one, 16.0, 16.0, False, np.ones((4, 4)))
    _raises_invalid(qe.qe_plan_join, good, 1e9, 1e9, False, np.ones((8, 8)))
    # fit: two distinct positive sizes, N >= 2, known op
    _raises_invalid(qe.qe_plan_fit_link, 0, 4, 2, [1e6], [1e-3])
    _raises_invalid(qe.qe_plan_fit_link, 0, 4, 2, [1e6, 1e6], [1e-3, 2e-3])
    _raises_invalid(qe.qe_plan_fit_link, 0, 4, 2, [0.0, 1e6], [1e-3, 2e-3])
    _raises_invalid(qe.qe_plan_fit_link, 0, 1, 1, [1e5, 1e6], [1e-3, 2e-3])
    _raises_invalid(qe.qe_plan_fit_link, 3, 4, 2, [1e5, 1e6], [1e-3, 2e-3])
    _raises_invalid(qe.qe_plan_skew_gradient, 0, 1.0, 1.0)
    _raises_invalid(qe.qe_plan_skew_gradient, 4, -0.5, 1.0)
    # NULL outputs through the raw ABI, and no output written on error
    assert lib.qe_plan_exchange_time(ctypes.byref(good), 0, 1e9, None) == qe.ERR_INVALID_ARG
    assert lib.qe_plan_join(None, 1.0, 1.0, 0, None, None, None, None, None) == qe.ERR_INVALID_ARG
    out = ctypes.c_double(-7.0)
    assert lib.qe_plan_exchange_time(ctypes.byref(good), 0, -1.0, ctypes.byref(out)) == qe.ERR_INVALID_ARG
    assert out.value == -7.0
    st = ctypes.c_int32(-7)
    assert lib.qe_plan_join(ctypes.byref(good), -1.0, 1.0, 0, None, None, ctypes.byref(st), None, None) \
        == qe.ERR_INVALID_ARG
    assert st.value == -7
