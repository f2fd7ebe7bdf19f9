"""Pins of the CPU oracle against things other than itself.

Each operator of the oracle is checked against an independent brute-force
restatement on tiny inputs (per-row predicate loop, per-row partition loop,
nested-loop join, dictionary group-by), against hand-worked fixtures in
tests/golden/, and against invariants that hold at any size (partition output
is a permutation with monotone offsets; a foreign-key join yields exactly one
match per probe row; SUM and COUNT totals are preserved).  The planted-mistake
tests at the end show that a dropped term, a wrong index or a wrong sign in
the kind of code the oracle contains is caught by these checks.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_09226_gb300 import datagen

GOLD = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def wrap64(x: int) -> int:
    x &= M64
    return x - (1 << 64) if x >> 63 else x


# ---------------------------------------------------------------- brute force
def bf_pred(x, op, lo, hi):
    return [x < lo, x <= lo, x > lo, x >= lo, x == lo, x != lo, lo <= x <= hi][op]


def bf_filter(cols, preds):
    n = len(cols[0])
    return [i for i in range(n)
            if all(bf_pred(int(cols[p.col][i]), p.op, p.lo, p.hi) for p in preds)]


def bf_partition(keys, pays, part):
    buckets = {}
    for i, k in enumerate(keys):
        buckets.setdefault(part(int(k)), []).append(i)
    F = max(buckets) + 1 if buckets else 1
    order, offs = [], [0]
    for p in range(F):
        order += buckets.get(p, [])
        offs.append(len(order))
    return order, offs


def bf_join(bkeys, bpay, pkeys, sel):
    rows = list(range(len(pkeys))) if sel is None else [int(s) for s in sel]
    out = []
    for r in rows:                                   # nested loop
        for j in range(len(bkeys)):
            if int(bkeys[j]) == int(pkeys[r]):
                out.append((r, int(bpay[j])))
    return out


def bf_groupby(keys, aggs):
    d = {}
    for i, k in enumerate(keys):
        d.setdefault(int(k), []).append(i)
    res = {}
    for k, idx in d.items():
        row = []
        for op, v in aggs:
            if op == O.SUM:
                row.append(wrap64(sum(int(v[i]) for i in idx)))
            elif op == O.COUNT:
                row.append(len(idx))
            elif op == O.MIN:
                row.append(min(int(v[i]) for i in idx))
            else:
                row.append(max(int(v[i]) for i in idx))
        res[k] = row
    return res


# ---------------------------------------------------------------- filter
@pytest.mark.parametrize("seed", range(4))
def test_filter_matches_row_loop(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 300))
    cols = [rng.integers(-50, 50, n).astype(np.int32),
            rng.integers(-100, 100, n).astype(np.int8),
            rng.integers(-2 ** 62, 2 ** 62, n, dtype=np.int64)]
    for op in range(7):
        preds = [O.Pred(0, op, int(rng.integers(-40, 40)), int(rng.integers(0, 40)))]
        preds.append(O.Pred(1, int(rng.integers(0, 7)), int(rng.integers(-60, 60)), 90))
        got = O.filter(cols, preds)
        assert got.dtype == np.int32
        assert got.tolist() == bf_filter(cols, preds)


def test_filter_edges():
    d = np.arange(10, dtype=np.int32)
    assert O.filter([d], [O.Pred(0, O.LT, 0)]).tolist() == []           # 0 %
    assert O.filter([d], [O.Pred(0, O.LT, 10)]).tolist() == list(range(10))  # 100 %
    assert O.filter([d], [O.Pred(0, O.LT, 5)]).tolist() == [0, 1, 2, 3, 4]   # strict
    assert O.filter([d], [O.Pred(0, O.BETWEEN, 3, 5)]).tolist() == [3, 4, 5]
    assert O.filter([np.empty(0, np.int32)], [O.Pred(0, O.LT, 5)]).tolist() == []
    assert O.filter([d], []).tolist() == list(range(10))                # no predicate


def test_filter_count_closed_form():
    # date uniform in [0, 2557): E|date < c| = n c / 2557 (binomial, 5 sigma)
    n, c = 200_000, 1278
    f = datagen.star_fact(n, 1000, seed=11)
    got = len(O.filter([f["date"].numpy()], [O.Pred(0, O.LT, c)]))
    p = c / datagen.DATE_SPAN
    assert abs(got - n * p) < 5 * (n * p * (1 - p)) ** 0.5
    assert got == int((f["date"].numpy() < c).sum())


# ---------------------------------------------------------------- hash
def test_fmix64_fixed_point_and_bijection():
    assert O.fmix64(0) == 0
    # invert the published step sequence with modular inverses computed here;
    # a changed constant or shift makes the round trip fail
    c1, c2 = 0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53
    i1, i2 = pow(c1, -1, 1 << 64), pow(c2, -1, 1 << 64)

    def unxorshift33(h):
        return h ^ (h >> 33)          # 33 >= 32, so one step inverts it

    rng = np.random.default_rng(5)
    for k in [1, 2, 3, 2 ** 63, M64] + [int(x) for x in rng.integers(0, 2 ** 63, 200)]:
        h = O.fmix64(k)
        x = unxorshift33(h)
        x = (x * i2) & M64
        x = unxorshift33(x)
        x = (x * i1) & M64
        x = unxorshift33(x)
        assert x == k


def test_fmix64_avalanche():
    # each input bit flip changes each output bit with probability ~1/2
    rng = np.random.default_rng(7)
    keys = [int(x) for x in rng.integers(0, 2 ** 63, 300)]
    flips = np.zeros(64)
    trials = 0
    for k in keys:
        h = O.fmix64(k)
        for b in range(0, 64, 3):
            d = h ^ O.fmix64(k ^ (1 << b))
            flips += [(d >> j) & 1 for j in range(64)]
            trials += 1
    p = flips / trials
    assert p.min() > 0.42 and p.max() < 0.58


# ---------------------------------------------------------------- partition
def test_partition_golden():
    g = json.load(open(os.path.join(GOLD, "tiny_partition.json")))
    k, (p,), offs = O.partition(np.array(g["keys"]), [np.array(g["payload"], np.int64)],
                                g["log2f"], mode=1, shift=g["shift"])
    assert k.tolist() == g["expect"]["keys"]
    assert p.tolist() == g["expect"]["payload"]
    assert offs.tolist() == g["expect"]["offsets"]


@pytest.mark.parametrize("log2f,mode,shift", [(0, 0, 0), (1, 0, 0), (4, 0, 0), (8, 0, 0),
                                              (3, 1, 0), (4, 1, 5), (6, 1, 58)])
def test_partition_matches_row_loop(log2f, mode, shift):
    rng = np.random.default_rng(log2f * 10 + mode)
    n = 700
    keys = rng.integers(-2 ** 63, 2 ** 63 - 1, n, dtype=np.int64)
    keys[::7] = keys[3]                                    # repeated keys
    pay32 = rng.integers(-2 ** 31, 2 ** 31 - 1, n).astype(np.int32)
    pay8 = rng.integers(-128, 127, n).astype(np.int8)
    rowid = np.arange(n, dtype=np.int64)
    F = 1 << log2f

    def part(k):
        if log2f == 0:
            return 0
        if mode == 0:
            return O.fmix64(k) >> (64 - log2f)
        return ((k & M64) >> shift) & (F - 1)

    ok, (op32, op8, orow), offs = O.partition(keys, [pay32, pay8, rowid], log2f, mode, shift)
    order, boffs = bf_partition(keys, None, part)
    boffs = boffs + [boffs[-1]] * (F + 1 - len(boffs))
    assert offs.tolist() == boffs
    assert orow.tolist() == order
    assert ok.tolist() == keys[order].tolist()
    assert op32.tolist() == pay32[order].tolist()
    assert op8.tolist() == pay8[order].tolist()


def test_partition_invariants():
    key, pay = datagen.key_payload_pairs(50_000, seed=2)
    key, pay = key.numpy(), pay.numpy()
    for log2f in (0, 8, 10, 12):
        F = 1 << log2f
        ok, (op,), offs = O.partition(key, [pay], log2f)
        assert offs[0] == 0 and offs[-1] == len(key) and np.all(np.diff(offs) >= 0)
        assert np.array_equal(np.sort(op), pay)                 # permutation
        assert np.array_equal(key[op], ok)                      # pairs stay together
        seg = np.repeat(np.arange(F), np.diff(offs))
        for i in range(0, len(ok), 997):                        # destination check
            assert O.partition_of(int(ok[i]), log2f) == seg[i]
        d = np.diff(op)                                         # stable: ascending rows
        assert np.all((d > 0) | (np.diff(seg) > 0))
    ok, (op,), offs = O.partition(key, [pay], 0)                # F = 1 is the identity
    assert np.array_equal(ok, key) and np.array_equal(op, pay)


# ---------------------------------------------------------------- join
@pytest.mark.parametrize("seed", range(3))
def test_join_matches_nested_loop(seed):
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(1, 120))
    bkeys = rng.choice(np.arange(-300, 300), nb, replace=False).astype(np.int32)
    bpay = rng.integers(-2 ** 31, 2 ** 31 - 1, nb).astype(np.int32)
    pkeys = rng.integers(-320, 320, 400).astype(np.int32)
    sel = np.sort(rng.choice(400, 150, replace=False)).astype(np.int32)
    for s in (None, sel):
        rows, pay = O.join(bkeys, bpay, pkeys, s)
        assert list(zip(rows.tolist(), pay.tolist())) == bf_join(bkeys, bpay, pkeys, s)


def test_join_duplicate_and_empty():
    with pytest.raises(ValueError):
        O.join(np.array([1, 2, 1], np.int32), np.array([0, 0, 0], np.int32),
               np.array([1], np.int32))
    rows, pay = O.join(np.empty(0, np.int32), np.empty(0, np.int32), np.array([1, 2], np.int32))
    assert len(rows) == 0
    rows, pay = O.join(np.array([1], np.int32), np.array([5], np.int32), np.empty(0, np.int32))
    assert len(rows) == 0
    # extreme keys are ordinary keys for the oracle
    bk = np.array([-2 ** 31, 2 ** 31 - 1], np.int32)
    rows, pay = O.join(bk, np.array([7, 8], np.int32), np.array([2 ** 31 - 1, -2 ** 31], np.int32))
    assert rows.tolist() == [0, 1] and pay.tolist() == [8, 7]


def test_join_fk_invariant():
    dim = datagen.star_dim(5000, 25, seed=0)
    fact = datagen.star_fact(40_000, 5000, seed=0)
    dk, da, fk = dim["key"].numpy(), dim["attr"].numpy(), fact["fk"].numpy()
    sel = O.filter([fact["date"].numpy()], [O.Pred(0, O.LT, 1278)])
    rows, pay = O.join(dk, da, fk, sel)
    assert np.array_equal(rows, sel)                       # exactly one match per row
    direct = np.empty(5000, np.int32)
    direct[dk] = da                                        # keys are a permutation
    assert np.array_equal(pay, direct[fk[sel]])


# ---------------------------------------------------------------- join on a pair of key columns
def bf_join_pair(bhi, blo, bpay, phi, plo, sel):
    rows = range(len(phi)) if sel is None else [int(r) for r in sel]
    out = []
    for r in rows:
        m = [int(bpay[j]) for j in range(len(bhi)) if int(bhi[j]) == int(phi[r]) and int(blo[j]) == int(plo[r])]
        assert len(m) <= 1
        out += [(int(r), m[0])] if m else []
    return out


@pytest.mark.parametrize("seed", range(3))
def test_join_pair_matches_nested_loop(seed):
    rng = np.random.default_rng(400 + seed)
    pairs = rng.choice(40 * 40, int(rng.integers(1, 300)), replace=False)
    bhi, blo = (pairs // 40 - 20).astype(np.int32), (pairs % 40 - 20).astype(np.int32)
    bpay = rng.integers(-2 ** 31, 2 ** 31 - 1, len(pairs)).astype(np.int32)
    phi, plo = rng.integers(-22, 22, 500).astype(np.int32), rng.integers(-22, 22, 500).astype(np.int32)
    sel = np.sort(rng.choice(500, 200, replace=False)).astype(np.int32)
    for s in (None, sel):
        rows, pay = O.join_pair(bhi, blo, bpay, phi, plo, s)
        assert list(zip(rows.tolist(), pay.tolist())) == bf_join_pair(bhi, blo, bpay, phi, plo, s)


def test_join_pair_invariants():
    rng = np.random.default_rng(41)
    bk = rng.choice(np.arange(-500, 500), 300, replace=False).astype(np.int32)
    bp = rng.integers(0, 1000, 300).astype(np.int32)
    pk = rng.integers(-600, 600, 2000).astype(np.int32)
    # one key column constant: the single-column join
    z = np.zeros_like(bk)
    r1, p1 = O.join_pair(z, bk, bp, np.zeros_like(pk), pk)
    r2, p2 = O.join(bk, bp, pk)
    assert np.array_equal(r1, r2) and np.array_equal(p1, p2)
    # the halves are not interchangeable: (a, b) does not match (b, a)
    rows, _ = O.join_pair(np.array([1], np.int32), np.array([2], np.int32), np.array([9], np.int32),
                          np.array([2, 1], np.int32), np.array([1, 2], np.int32))
    assert rows.tolist() == [1]
    # extreme values are ordinary keys; a repeated pair is an error, a repeated half is not
    m = -2 ** 31
    rows, pay = O.join_pair(np.array([m, m], np.int32), np.array([m, 7], np.int32), np.array([1, 2], np.int32),
                            np.array([m, m, 0], np.int32), np.array([7, m, m], np.int32))
    assert rows.tolist() == [0, 1] and pay.tolist() == [2, 1]
    with pytest.raises(ValueError):
        O.join_pair(np.array([3, 3], np.int32), np.array([4, 4], np.int32), np.array([1, 2], np.int32),
                    np.array([3], np.int32), np.array([4], np.int32))


# ---------------------------------------------------------------- many-to-many join
def bf_join_multi(bkeys, bpay, pkeys, sel):
    """Nested loop: every (position, build row) pair with equal keys, build
    rows in ascending order within a position."""
    rows = range(len(pkeys)) if sel is None else [int(r) for r in sel]
    return [(int(r), int(bpay[j])) for r in rows for j in range(len(bkeys)) if int(bkeys[j]) == int(pkeys[r])]


@pytest.mark.parametrize("seed", range(3))
def test_join_multi_matches_nested_loop(seed):
    rng = np.random.default_rng(200 + seed)
    nb = int(rng.integers(0, 200))
    bkeys = rng.integers(-40, 40, nb).astype(np.int32)            # many repeats
    bpay = rng.integers(-2 ** 31, 2 ** 31 - 1, nb).astype(np.int32)
    pkeys = rng.integers(-50, 50, 300).astype(np.int32)
    sel = np.sort(rng.choice(300, 100, replace=False)).astype(np.int32)
    for s in (None, sel):
        rows, pay = O.join_multi(bkeys, bpay, pkeys, s)
        assert list(zip(rows.tolist(), pay.tolist())) == bf_join_multi(bkeys, bpay, pkeys, s)


def test_join_multi_invariants():
    rng = np.random.default_rng(31)
    bkeys = rng.integers(0, 60, 500).astype(np.int32)
    bpay = np.arange(500, dtype=np.int32)
    pkeys = rng.integers(0, 80, 1000).astype(np.int32)
    rows, pay = O.join_multi(bkeys, bpay, pkeys)
    # one output per (position, equal build key); the kept positions are the semi-join's
    per_key = np.bincount(bkeys, minlength=80)
    assert len(rows) == int(per_key[pkeys].sum())
    assert np.array_equal(np.unique(rows), O.semi_join(bkeys, pkeys))
    assert np.all(bkeys[pay] == pkeys[rows])                      # payloads are build row ids here
    # unique build keys: the inner join
    ub, first = np.unique(bkeys, return_index=True)
    r1, p1 = O.join_multi(ub, bpay[first], pkeys)
    r2, p2 = O.join(ub, bpay[first], pkeys)
    assert np.array_equal(r1, r2) and np.array_equal(p1, p2)
    # empty sides
    assert len(O.join_multi(np.empty(0, np.int32), np.empty(0, np.int32), pkeys)[0]) == 0
    assert len(O.join_multi(bkeys, bpay, np.empty(0, np.int32))[0]) == 0


# ---------------------------------------------------------------- semi- and anti-join
def bf_semi(bkeys, pkeys, sel, anti):
    """Nested loop: position i keeps its row when any build key equals its key
    (or, anti, when none does)."""
    rows = range(len(pkeys)) if sel is None else [int(r) for r in sel]
    out = []
    for r in rows:
        found = any(int(b) == int(pkeys[r]) for b in bkeys)
        if found != anti:
            out.append(int(r))
    return out


@pytest.mark.parametrize("seed", range(3))
def test_semi_anti_match_nested_loop(seed):
    rng = np.random.default_rng(100 + seed)
    nb = int(rng.integers(0, 150))
    bkeys = rng.integers(-200, 200, nb).astype(np.int32)          # repeats allowed
    pkeys = rng.integers(-220, 220, 300).astype(np.int32)
    sel = np.sort(rng.choice(300, 120, replace=False)).astype(np.int32)
    for s in (None, sel):
        for anti in (False, True):
            assert O.semi_join(bkeys, pkeys, s, anti).tolist() == bf_semi(bkeys, pkeys, s, anti)


def test_semi_anti_invariants():
    rng = np.random.default_rng(9)
    bkeys = rng.integers(0, 50, 80).astype(np.int32)
    pkeys = rng.integers(0, 100, 500).astype(np.int32)
    sel = np.sort(rng.choice(500, 200, replace=False)).astype(np.int32)
    semi, anti = O.semi_join(bkeys, pkeys, sel), O.semi_join(bkeys, pkeys, sel, anti=True)
    # the two split the probe positions: disjoint, and together every position in order
    assert not set(semi.tolist()) & set(anti.tolist())
    assert sorted(semi.tolist() + anti.tolist()) == sel.tolist()
    # with unique build keys the semi-join keeps exactly the inner join's rows
    ub = np.unique(bkeys)
    rows, _ = O.join(ub, np.zeros(len(ub), np.int32), pkeys, sel)
    assert O.semi_join(ub, pkeys, sel).tolist() == rows.tolist()
    # repeated build keys change nothing
    assert O.semi_join(np.concatenate([bkeys, bkeys]), pkeys, sel).tolist() == semi.tolist()
    # empty sides
    assert O.semi_join(np.empty(0, np.int32), pkeys).tolist() == []
    assert O.semi_join(np.empty(0, np.int32), pkeys, anti=True).tolist() == list(range(500))
    assert O.semi_join(bkeys, np.empty(0, np.int32)).tolist() == []


@pytest.mark.parametrize("kind", [O.SEMI, O.ANTI])
def test_pipeline_semi_anti_matches_composition(kind):
    """group-by over filter, then EXISTS / NOT EXISTS against repeated dim
    keys, restated from the brute-force operators; and one group computed
    on its own."""
    rng = np.random.default_rng(4 + kind)
    nf = 500
    dk = rng.integers(0, 120, 90).astype(np.int32)
    fact = [rng.integers(0, 200, nf).astype(np.int32), rng.integers(0, 2557, nf).astype(np.int32),
            rng.integers(100, 10 ** 7, nf).astype(np.int64), rng.integers(1, 51, nf).astype(np.int32),
            rng.integers(0, 3, nf).astype(np.int8)]
    q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0, key_hi_col=-1, key_lo_col=4,
                aggs=[(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)], join_kind=kind)
    r = O.pipeline(fact, q, dk)
    sel = bf_filter(fact, q.preds)
    kept = bf_semi(dk, fact[0], sel, kind == O.ANTI)
    keys = [int(fact[4][i]) for i in kept]
    vals = [int(fact[2][i]) * int(fact[3][i]) for i in kept]
    price = [int(fact[2][i]) for i in kept]
    ref = bf_groupby(keys, [(O.SUM, vals), (O.COUNT, None), (O.MIN, price), (O.MAX, price)])
    assert r["keys"].tolist() == sorted(ref)
    for i, k in enumerate(r["keys"].tolist()):
        assert [int(a[i]) for a in r["aggs"]] == ref[k]
    assert r["nsel"] == len(sel) and r["njoin"] == len(kept)
    cnt, aggs = O.pipeline_group(fact, q, int(r["keys"][0]), dk)
    assert cnt == ref[int(r["keys"][0])][1] and aggs.tolist() == ref[int(r["keys"][0])]
    with pytest.raises(ValueError):
        O.pipeline(fact, O.Query(**{**q.__dict__, "key_lo_col": O.JOIN_PAYLOAD}), dk)


# ---------------------------------------------------------------- group-by
@pytest.mark.parametrize("seed", range(3))
def test_groupby_matches_dict(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 500))
    keys = rng.integers(-5, 5, n).astype(np.int64) * (2 ** 40 + 3)
    v = rng.integers(-2 ** 62, 2 ** 62, n, dtype=np.int64)     # sums wrap
    aggs = [(O.SUM, v), (O.COUNT, None), (O.MIN, v), (O.MAX, v)]
    gk, ga = O.groupby(keys, aggs)
    ref = bf_groupby(keys, [(op, v) for op, _ in aggs])
    assert gk.tolist() == sorted(ref)                       # ascending signed keys
    for i, k in enumerate(gk.tolist()):
        assert [int(a[i]) for a in ga] == ref[k]


def test_groupby_invariants():
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 3000, 100_000).astype(np.int64)
    v = rng.integers(100, 10 ** 7, 100_000).astype(np.int64)
    gk, (s, c, mn, mx) = O.groupby(keys, [(O.SUM, v), (O.COUNT, None), (O.MIN, v), (O.MAX, v)])
    assert c.sum() == len(keys) and s.sum() == v.sum()
    assert len(gk) == len(np.unique(keys))
    assert np.all(mn <= mx)
    # sort-then-run-length with numpy as a second route
    order = np.argsort(keys, kind="stable")
    uk, start = np.unique(keys[order], return_index=True)
    assert np.array_equal(uk, gk)
    assert np.array_equal(np.add.reduceat(v[order], start), s)
    assert np.array_equal(np.minimum.reduceat(v[order], start), mn)


# ---------------------------------------------------------------- pipeline
STAR_Q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0, key_hi_col=4,
                 key_lo_col=O.JOIN_PAYLOAD,
                 aggs=[(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)])


def _fact_list(f):
    return [f[c].numpy() if hasattr(f[c], "numpy") else np.asarray(f[c])
            for c in ("fk", "date", "price", "qty", "flag")]


def test_pipeline_golden():
    g = json.load(open(os.path.join(GOLD, "tiny_pipeline.json")))
    fact = [np.array(g["fact"]["fk"], np.int32), np.array(g["fact"]["date"], np.int32),
            np.array(g["fact"]["price"], np.int64), np.array(g["fact"]["qty"], np.int32),
            np.array(g["fact"]["flag"], np.int8)]
    q = O.Query(**{**STAR_Q.__dict__, "preds": [O.Pred(1, O.LT, g["date_lt"])]})
    r = O.pipeline(fact, q, np.array(g["dim"]["key"], np.int32),
                   np.array(g["dim"]["attr"], np.int32))
    e = g["expect"]
    assert r["nsel"] == e["nsel"] and r["njoin"] == e["njoin"]
    assert r["keys"].tolist() == e["keys"]
    for name, a in zip(("sum", "count", "min", "max"), r["aggs"]):
        assert a.tolist() == e[name]


def test_pipeline_matches_composition():
    rng = np.random.default_rng(3)
    nd, nf = 60, 400
    dk = rng.choice(np.arange(0, 200), nd, replace=False).astype(np.int32)
    da = rng.integers(0, 6, nd).astype(np.int32)
    fact = [rng.integers(0, 210, nf).astype(np.int32), rng.integers(0, 2557, nf).astype(np.int32),
            rng.integers(100, 10 ** 7, nf).astype(np.int64), rng.integers(1, 51, nf).astype(np.int32),
            rng.integers(0, 3, nf).astype(np.int8)]
    r = O.pipeline(fact, STAR_Q, dk, da)
    sel = bf_filter(fact, STAR_Q.preds)
    joined = bf_join(dk, da, fact[0], sel)
    keys = [wrap64((int(fact[4][i]) << 32) | (p & 0xFFFFFFFF)) for i, p in joined]
    vals = [int(fact[2][i]) * int(fact[3][i]) for i, _ in joined]
    price = [int(fact[2][i]) for i, _ in joined]
    ref = bf_groupby(keys, [(O.SUM, vals), (O.COUNT, None), (O.MIN, price), (O.MAX, price)])
    assert r["keys"].tolist() == sorted(ref)
    for i, k in enumerate(r["keys"].tolist()):
        assert [int(a[i]) for a in r["aggs"]] == ref[k]
    assert r["nsel"] == len(sel) and r["njoin"] == len(joined)


def test_pipeline_invariants_and_single_group_route():
    dim = datagen.star_dim(10_000, 25, seed=0)
    fact = datagen.star_fact(100_000, 10_000, seed=0)
    fl = _fact_list(fact)
    r = O.pipeline(fl, STAR_Q, dim["key"].numpy(), dim["attr"].numpy())
    m = fl[1] < 1278
    assert r["nsel"] == int(m.sum()) == r["njoin"]                     # FK join
    assert int(r["aggs"][1].sum()) == r["nsel"]                        # sum COUNT
    assert int(r["aggs"][0].sum()) == int((fl[2][m] * fl[3][m]).sum())  # sum SUM
    assert len(r["keys"]) == 75
    for gi in (0, 17, 74):
        cnt, aggs = O.pipeline_group(fl, STAR_Q, int(r["keys"][gi]),
                                     dim["key"].numpy(), dim["attr"].numpy())
        assert cnt == r["aggs"][1][gi]
        assert aggs.tolist() == [int(a[gi]) for a in r["aggs"]]
    cnt, _ = O.pipeline_group(fl, STAR_Q, 12345, dim["key"].numpy(), dim["attr"].numpy())
    assert cnt == 0


def test_pipeline_without_join():
    rng = np.random.default_rng(1)
    fact = [rng.integers(0, 5, 300).astype(np.int32), rng.integers(0, 100, 300).astype(np.int64)]
    q = O.Query(preds=[O.Pred(1, O.GE, 50)], fk_col=-1, key_hi_col=-1, key_lo_col=0,
                aggs=[(O.SUM, 1, -1), (O.COUNT, -1, -1)])
    r = O.pipeline(fact, q)
    sel = fact[1] >= 50
    ref = bf_groupby(fact[0][sel], [(O.SUM, fact[1][sel]), (O.COUNT, None)])
    assert r["keys"].tolist() == sorted(ref)
    assert [[int(a[i]) for a in r["aggs"]] for i in range(len(r["keys"]))] == \
        [ref[k] for k in sorted(ref)]


def test_group_key_rule():
    """The group key: the low part alone, sign-extended, without a high part;
    (hi << 32) | (uint32)lo with one.  Checked directly and through join-free
    pipelines grouped by a negative int32 column and by an int64 column."""
    assert O.group_key(False, 0, -5) == -5
    assert O.group_key(False, 0, -(1 << 40)) == -(1 << 40)
    assert O.group_key(True, -1, -2) == -2
    assert O.group_key(True, 2, -1) == (2 << 32) | 0xFFFFFFFF
    assert O.group_key(True, -3, 7) == wrap64((-3 << 32) | 7)
    rng = np.random.default_rng(5)
    v = rng.integers(0, 100, 200).astype(np.int64)
    for col in (rng.integers(-4, 4, 200).astype(np.int32),
                (rng.integers(-3, 3, 200) * (1 << 40)).astype(np.int64)):
        q = O.Query(preds=[], fk_col=-1, key_hi_col=-1, key_lo_col=0, aggs=[(O.SUM, 1, -1), (O.COUNT, -1, -1)])
        r = O.pipeline([col, v], q)
        ref = bf_groupby(col.tolist(), [(O.SUM, v), (O.COUNT, None)])
        assert r["keys"].tolist() == sorted(ref)
        assert [[int(a[i]) for a in r["aggs"]] for i in range(len(r["keys"]))] == [ref[k] for k in sorted(ref)]


# ---------------------------------------------------------------- derived averages
def test_avg_golden():
    """oracle_avg against hand-worked cases (exact rational arithmetic):
    halves, thirds, negative sums, sums past 2^53 that round before the
    division, a count-1 group with a sum near 2^62."""
    g = json.load(open(os.path.join(GOLD, "avg_cases.json")))
    sums = np.array([int(c["sum"]) for c in g["cases"]], np.int64)
    cnts = np.array([int(c["count"]) for c in g["cases"]], np.int64)
    got = O.avg(sums, cnts)
    for c, x in zip(g["cases"], got):
        assert float(x).hex() == float.fromhex(c["avg_hex"]).hex(), c["note"]


def test_avg_within_two_roundings():
    """For random sums over the whole int64 range and counts up to 10^9:
    the average is within two double roundings (2^-52 relative) of the exact
    quotient, and equal to the correctly rounded quotient whenever the sum
    converts to double exactly (|sum| <= 2^53)."""
    from fractions import Fraction
    rng = np.random.default_rng(8)
    mags = rng.integers(0, 63, 4000)
    sums = np.array([int(rng.integers(-(1 << int(m)), 1 << int(m), endpoint=True)) if m else 0 for m in mags],
                    np.int64)
    cnts = rng.integers(1, 10 ** 9, 4000).astype(np.int64)
    cnts[:500] = 1
    got = O.avg(sums, cnts)
    for s, c, x in zip(sums.tolist(), cnts.tolist(), got.tolist()):
        q = Fraction(s, c)
        assert abs(Fraction(x) - q) <= abs(q) * Fraction(1, 1 << 52)
        if abs(s) <= 1 << 53:
            assert x == float(q)


def test_avg_of_pipeline_groups():
    """The average of SUM(price*qty) over COUNT for the tiny pipeline's
    groups, and AVG(price) of a join-free pipeline against per-group means
    taken with exact fractions."""
    from fractions import Fraction
    g = json.load(open(os.path.join(GOLD, "tiny_pipeline.json")))
    e = g["expect"]
    assert O.avg(e["sum"], e["count"]).tolist() == [950.0, 1000.0, 600.0, 800.0]
    rng = np.random.default_rng(4)
    key = rng.integers(0, 7, 500).astype(np.int32)
    price = rng.integers(100, 10 ** 7, 500).astype(np.int64)
    q = O.Query(preds=[], fk_col=-1, key_hi_col=-1, key_lo_col=0, aggs=[(O.SUM, 1, -1), (O.COUNT, -1, -1)])
    r = O.pipeline([key, price], q)
    got = O.avg(r["aggs"][0], r["aggs"][1])
    for k, x in zip(r["keys"].tolist(), got.tolist()):
        rows = price[key == k].tolist()
        assert x == float(Fraction(sum(rows), len(rows)))


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes():
    """The brute-force pins reject plausible oracle mistakes: a dropped
    predicate term, an off-by-one boundary, a swapped key half, a sign error
    in the aggregate and an unstable partition."""
    d = np.arange(20, dtype=np.int32)
    preds = [O.Pred(0, O.LT, 10), O.Pred(0, O.GE, 3)]
    good = bf_filter([d], preds)
    assert good != bf_filter([d], preds[:1])                          # dropped term
    assert good != bf_filter([d], [O.Pred(0, O.LE, 10), preds[1]])    # boundary
    g = json.load(open(os.path.join(GOLD, "tiny_pipeline.json")))
    swapped = [wrap64((2 << 32) | 1), 2]                              # hi/lo swap
    assert swapped[0] != g["expect"]["keys"][0]
    keys = np.array([1, 1, 2], np.int64)
    v = np.array([5, -3, 4], np.int64)
    s_ok = bf_groupby(keys, [(O.SUM, v)])[1][0]
    assert s_ok == 2 and s_ok != 5 + 3                                # sign error
    k, (p,), _ = O.partition(np.array([4, 0, 8], np.int64), [np.arange(3, dtype=np.int64)], 2, 1)
    assert p.tolist() == [0, 1, 2]                                    # unstable order fails
