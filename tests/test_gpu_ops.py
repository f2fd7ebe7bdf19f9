"""GPU parity of each operator against the CPU oracle (bit-exact).

Every test calls libqe through its C ABI (paper_2506_09226_gb300.qe) on
seeded synthetic inputs and compares element by element with oracle/ on the
same bytes.  Sizes span several tiles and a ragged tail; edge cases cover
empty input, single rows, warp and tile boundaries, 0 % / 100 % selectivity,
unaligned column views, the largest fan-out, duplicate and reserved keys and
too-small outputs.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_09226_gb300 import datagen
from paper_2506_09226_gb300 import qe

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 31, 32, 33, 4095, 4096, 4097, 100_003]
OPMAP = {qe.LT: O.LT, qe.LE: O.LE, qe.GT: O.GT, qe.GE: O.GE, qe.EQ: O.EQ, qe.NE: O.NE, qe.BETWEEN: O.BETWEEN}


@pytest.fixture(scope="module")
def ctx():
    c = qe.Context(0)
    yield c
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------- filter
@pytest.mark.parametrize("n", SIZES)
def test_filter_sizes(ctx, n):
    f = datagen.star_fact(n, 1000, seed=n)
    date = f["date"].numpy()
    sel, cnt = qe.qe_filter(ctx, [cuda(date)], [(0, qe.LT, 1278)])
    ref = O.filter([date], [O.Pred(0, O.LT, 1278)])
    assert int(cnt.item()) == len(ref)
    assert np.array_equal(sel[:len(ref)].cpu().numpy(), ref)


@pytest.mark.parametrize("op", list(OPMAP))
def test_filter_ops_and_types(ctx, op):
    rng = np.random.default_rng(op)
    n = 70_001
    cols = [rng.integers(-100, 100, n).astype(np.int32), rng.integers(-128, 127, n).astype(np.int8),
            rng.integers(-2 ** 40, 2 ** 40, n, dtype=np.int64)]
    preds = [(0, op, -7, 40), (1, qe.GE, -60), (2, qe.NE, int(cols[2][5]))]
    sel, cnt = qe.qe_filter(ctx, [cuda(c) for c in cols], preds)
    ref = O.filter(cols, [O.Pred(c, OPMAP[o], lo, hi[0] if hi else 0) for c, o, lo, *hi in preds])
    assert int(cnt.item()) == len(ref)
    assert np.array_equal(sel[:len(ref)].cpu().numpy(), ref)


def test_filter_selectivity_extremes_and_views(ctx):
    n = 50_000
    date = datagen.star_fact(n, 10, seed=3)["date"].numpy()
    d = cuda(date)
    for c, expect in ((0, 0), (datagen.DATE_SPAN, n)):
        sel, cnt = qe.qe_filter(ctx, [d], [(0, qe.LT, c)])
        assert int(cnt.item()) == expect
    sel, cnt = qe.qe_filter(ctx, [d], [(0, qe.LT, c)])
    assert np.array_equal(sel.cpu().numpy(), np.arange(n))
    # views starting at odd element offsets (not 16-byte aligned)
    for off in (1, 3):
        v = d[off:]
        sel, cnt = qe.qe_filter(ctx, [v], [(0, qe.LT, 999)])
        ref = O.filter([date[off:]], [O.Pred(0, O.LT, 999)])
        assert np.array_equal(sel[:int(cnt.item())].cpu().numpy(), ref)


# large inputs take the two-pass filter (4-row vector loads of the first
# predicate's column); unaligned first columns fall back to the one-pass scan
TWO_PASS_N = 5_000_011


@pytest.mark.parametrize("first", ["i32", "i8", "i64"])
@pytest.mark.parametrize("op", list(OPMAP))
def test_filter_two_pass(ctx, first, op):
    rng = np.random.default_rng(op * 7 + len(first))
    n = TWO_PASS_N
    c32 = rng.integers(-100, 100, n).astype(np.int32)
    c8 = rng.integers(-128, 127, n).astype(np.int8)
    c64 = rng.integers(-2 ** 40, 2 ** 40, n, dtype=np.int64)
    cols = {"i32": [c32, c8, c64], "i8": [c8, c32, c64], "i64": [c64, c32, c8]}[first]
    lo = {"i32": (-7, 40), "i8": (-60, 11), "i64": (-2 ** 39, 2 ** 38)}[first]
    preds = [(0, op, lo[0], lo[1]), (1, qe.GE, -50)]
    sel, cnt = qe.qe_filter(ctx, [cuda(c) for c in cols], preds)
    ref = O.filter(cols, [O.Pred(c, OPMAP[o], a, b[0] if b else 0) for c, o, a, *b in preds])
    assert int(cnt.item()) == len(ref)
    assert np.array_equal(sel[:len(ref)].cpu().numpy(), ref)


def test_filter_two_pass_bounds_and_views(ctx):
    n = TWO_PASS_N
    date = datagen.star_fact(n, 10, seed=9)["date"].numpy()
    d = cuda(date)
    # a range that clamps to the column's width, and the empty ranges
    for pred, o_pred in (((0, qe.LT, 2 ** 40), O.Pred(0, O.LT, 2 ** 40)),
                         ((0, qe.GT, 2 ** 40), O.Pred(0, O.GT, 2 ** 40)),
                         ((0, qe.NE, -(2 ** 40)), O.Pred(0, O.NE, -(2 ** 40))),
                         ((0, qe.BETWEEN, 900, 100), O.Pred(0, O.BETWEEN, 900, 100))):
        sel, cnt = qe.qe_filter(ctx, [d], [pred])
        ref = O.filter([date], [o_pred])
        assert int(cnt.item()) == len(ref)
        assert np.array_equal(sel[:len(ref)].cpu().numpy(), ref)
    for off in (1, 2):
        sel, cnt = qe.qe_filter(ctx, [d[off:]], [(0, qe.LT, 999)])
        ref = O.filter([date[off:]], [O.Pred(0, O.LT, 999)])
        assert np.array_equal(sel[:int(cnt.item())].cpu().numpy(), ref)
    # capacity: the first rows are written, the required size reported
    out = torch.full((1000,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(qe.QeError) as e:
        qe.qe_filter(ctx, [d], [(0, qe.LT, 1278)], out_sel=out)
    ref = O.filter([date], [O.Pred(0, O.LT, 1278)])
    assert e.value.status == qe.ERR_CAPACITY and e.value.required == len(ref)
    assert np.array_equal(out.cpu().numpy(), ref[:1000])


def test_filter_capacity_error(ctx):
    date = cuda(np.arange(10_000, dtype=np.int32))
    out = torch.full((100,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(qe.QeError) as e:
        qe.qe_filter(ctx, [date], [(0, qe.LT, 5000)], out_sel=out)
    assert e.value.status == qe.ERR_CAPACITY and e.value.required == 5000
    assert np.array_equal(out.cpu().numpy(), np.arange(100))   # the first rows are written


# ---------------------------------------------------------------- partition
def _check_partition(ctx, keys, pays, log2f, mode=qe.PART_HASH, shift=0):
    ok, op, offs = qe.qe_partition(ctx, cuda(keys), [cuda(p) for p in pays], log2f, mode, shift)
    rk, rp, roffs = O.partition(keys, pays, log2f, mode, shift)
    assert np.array_equal(offs.cpu().numpy(), roffs)
    assert np.array_equal(ok.cpu().numpy(), rk)
    for a, b in zip(op, rp):
        assert np.array_equal(a.cpu().numpy(), b)


@pytest.mark.parametrize("log2f", [0, 1, 5, 8, 9, 10, 11, 12])
@pytest.mark.parametrize("n", [1, 33, 4097, 123_457])
def test_partition_hash_fast_path(ctx, n, log2f):
    k, p = datagen.key_payload_pairs(n, seed=log2f)
    _check_partition(ctx, k.numpy(), [p.numpy()], log2f)


@pytest.mark.parametrize("log2f,shift", [(4, 0), (8, 3), (12, 52)])
def test_partition_radix_generic_payloads(ctx, log2f, shift):
    rng = np.random.default_rng(log2f)
    n = 50_001
    keys = rng.integers(-2 ** 63, 2 ** 63 - 1, n, dtype=np.int64)
    pays = [rng.integers(-2 ** 31, 2 ** 31 - 1, n).astype(np.int32), rng.integers(-128, 127, n).astype(np.int8),
            np.arange(n, dtype=np.int64)]
    _check_partition(ctx, keys, pays, log2f, qe.PART_RADIX, shift)
    _check_partition(ctx, keys, [], log2f, qe.PART_RADIX, shift)


@pytest.mark.parametrize("log2f", [3, 10, 11, 12])
def test_partition_many_chunks_per_block(ctx, log2f):
    """Several chunks per block, so the rows a block holds back for an
    incomplete output sector are carried across chunks; keys only and with
    one payload.  Fan-outs above 64 take two passes."""
    n = 3_000_001
    k, p = datagen.key_payload_pairs(n, seed=77)
    _check_partition(ctx, k.numpy(), [p.numpy()], log2f)
    _check_partition(ctx, k.numpy(), [], log2f)


@pytest.mark.parametrize("koff,poff", [(1, 0), (2, 3), (3, 1)])
def test_partition_unaligned_outputs(ctx, koff, poff):
    """Output columns that start mid-sector (8-byte but not 32-byte aligned)."""
    n = 1_000_003
    k, p = datagen.key_payload_pairs(n, seed=koff * 4 + poff)
    kb = torch.empty(n + 4, dtype=torch.int64, device="cuda")
    pb = torch.empty(n + 4, dtype=torch.int64, device="cuda")
    ok, op = kb[koff:koff + n], pb[poff:poff + n]
    offs = torch.empty(1025, dtype=torch.int64, device="cuda")
    qe.qe_partition(ctx, cuda(k.numpy()), [cuda(p.numpy())], 10, qe.PART_HASH, 0, ok, [op], offs)
    rk, rp, roffs = O.partition(k.numpy(), [p.numpy()], 10, qe.PART_HASH, 0)
    assert np.array_equal(offs.cpu().numpy(), roffs)
    assert np.array_equal(ok.cpu().numpy(), rk)
    assert np.array_equal(op.cpu().numpy(), rp[0])


@pytest.mark.parametrize("log2f", [5, 10])
def test_partition_general_kernel(ctx, log2f):
    """The general scatter (two-pass chunk ranking) on the inputs the
    write-combining scatter normally takes."""
    n = 1_500_007
    k, p = datagen.key_payload_pairs(n, seed=log2f + 100)
    ctx.set_tuning("part_general", 1)
    try:
        _check_partition(ctx, k.numpy(), [p.numpy()], log2f)
        _check_partition(ctx, k.numpy(), [], log2f)
    finally:
        ctx.set_tuning("part_general", 0)


def test_partition_skew_and_empty(ctx):
    n = 70_000
    keys = np.full(n, 42, np.int64)           # every row to one destination
    keys[::1000] = 7
    _check_partition(ctx, keys, [np.arange(n, dtype=np.int64)], 12)
    ok, op, offs = qe.qe_partition(ctx, torch.empty(0, dtype=torch.int64, device="cuda"),
                                   [torch.empty(0, dtype=torch.int64, device="cuda")], 8)
    assert offs.cpu().numpy().tolist() == [0] * 257


# ---------------------------------------------------------------- join
@pytest.mark.parametrize("layout", [qe.HT_DENSE, qe.HT_OPEN, qe.HT_AUTO])
@pytest.mark.parametrize("with_sel", [False, True])
def test_join_probe(ctx, layout, with_sel):
    rng = np.random.default_rng(layout * 2 + with_sel)
    nb, npr = 30_000, 200_001
    bk = rng.choice(np.arange(-50_000, 50_000), nb, replace=False).astype(np.int32)
    bp = rng.integers(-2 ** 31, 2 ** 31 - 1, nb).astype(np.int32)
    pk = rng.integers(-60_000, 60_000, npr).astype(np.int32)
    sel = np.sort(rng.choice(npr, 77_777, replace=False)).astype(np.int32) if with_sel else None
    ht = qe.qe_join_build(ctx, cuda(bk), cuda(bp), layout=layout)
    info = ht.info()
    assert info.layout == (qe.HT_DENSE if layout == qe.HT_AUTO else layout)
    rows, pay, cnt = qe.qe_join_probe(ctx, ht, cuda(pk), cuda(sel) if with_sel else None)
    rr, rp = O.join(bk, bp, pk, sel)
    c = int(cnt.item())
    assert c == len(rr)
    assert np.array_equal(rows[:c].cpu().numpy(), rr)
    assert np.array_equal(pay[:c].cpu().numpy(), rp)
    ht.destroy()


@pytest.mark.parametrize("layout", [qe.HT_DENSE, qe.HT_OPEN])
@pytest.mark.parametrize("with_sel", [False, True])
def test_join_probe_two_pass(ctx, layout, with_sel):
    """Large probes take the two-pass compaction."""
    rng = np.random.default_rng(layout * 2 + with_sel + 10)
    nb, npr = 300_000, 9_000_007
    bk = rng.choice(np.arange(-500_000, 500_000), nb, replace=False).astype(np.int32)
    bp = rng.integers(-2 ** 31, 2 ** 31 - 1, nb).astype(np.int32)
    pk = rng.integers(-600_000, 600_000, npr).astype(np.int32)
    sel = np.sort(rng.choice(npr, 5_000_000, replace=False)).astype(np.int32) if with_sel else None
    ht = qe.qe_join_build(ctx, cuda(bk), cuda(bp), layout=layout)
    rows, pay, cnt = qe.qe_join_probe(ctx, ht, cuda(pk), cuda(sel) if with_sel else None)
    rr, rp = O.join(bk, bp, pk, sel)
    c = int(cnt.item())
    assert c == len(rr)
    assert np.array_equal(rows[:c].cpu().numpy(), rr)
    assert np.array_equal(pay[:c].cpu().numpy(), rp)
    ht.destroy()


def test_join_dense_full_and_star(ctx):
    dim = datagen.star_dim(100_000, 25, seed=0)
    fact = datagen.star_fact(1_000_000, 100_000, seed=0)
    ht = qe.qe_join_build(ctx, dim["key"].cuda(), dim["attr"].cuda())
    assert ht.info().full == 1
    sel = O.filter([fact["date"].numpy()], [O.Pred(0, O.LT, 1278)])
    rows, pay, cnt = qe.qe_join_probe(ctx, ht, fact["fk"].cuda(), cuda(sel))
    rr, rp = O.join(dim["key"].numpy(), dim["attr"].numpy(), fact["fk"].numpy(), sel)
    assert int(cnt.item()) == len(sel) == len(rr)          # one match per row (FK)
    assert np.array_equal(rows.cpu().numpy()[:len(rr)], rr)
    assert np.array_equal(pay.cpu().numpy()[:len(rr)], rp)
    ht.destroy()


def test_join_errors(ctx):
    for layout in (qe.HT_DENSE, qe.HT_OPEN):
        with pytest.raises(qe.QeError) as e:
            qe.qe_join_build(ctx, cuda(np.array([5, 9, 5], np.int32)), cuda(np.zeros(3, np.int32)), layout=layout)
        assert e.value.status == qe.ERR_DUPLICATE_KEY
    with pytest.raises(qe.QeError) as e:
        qe.qe_join_build(ctx, cuda(np.array([1, -2 ** 31], np.int32)), cuda(np.zeros(2, np.int32)),
                         layout=qe.HT_OPEN)
    assert e.value.status == qe.ERR_RESERVED_KEY
    # INT32_MIN is an ordinary key in the dense layout
    ht = qe.qe_join_build(ctx, cuda(np.array([-2 ** 31, -2 ** 31 + 1], np.int32)),
                          cuda(np.array([3, 4], np.int32)), layout=qe.HT_DENSE)
    rows, pay, cnt = qe.qe_join_probe(ctx, ht, cuda(np.array([-2 ** 31 + 1, 0, -2 ** 31], np.int32)))
    assert rows[:2].cpu().tolist() == [0, 2] and pay[:2].cpu().tolist() == [4, 3]
    ht.destroy()
    # empty build side and empty probe side
    ht = qe.qe_join_build(ctx, torch.empty(0, dtype=torch.int32, device="cuda"),
                          torch.empty(0, dtype=torch.int32, device="cuda"))
    rows, pay, cnt = qe.qe_join_probe(ctx, ht, cuda(np.array([1, 2], np.int32)))
    assert int(cnt.item()) == 0
    rows, pay, cnt = qe.qe_join_probe(ctx, ht, torch.empty(0, dtype=torch.int32, device="cuda"))
    assert int(cnt.item()) == 0
    ht.destroy()


# ---------------------------------------------------------------- group-by
def _sorted_groups(g):
    k, a = g.to_host()
    o = np.argsort(k.numpy(), kind="stable")
    return k.numpy()[o], [x.numpy()[o] for x in a]


@pytest.mark.parametrize("placement", [qe.GB_AUTO, qe.GB_SMEM, qe.GB_HBM])
@pytest.mark.parametrize("ngroups", [1, 75, 3000, 40_000])
def test_groupby(ctx, placement, ngroups):
    rng = np.random.default_rng(ngroups + placement)
    n = 200_003
    hi = rng.integers(0, 3, n).astype(np.int8)
    lo = rng.integers(0, max(1, ngroups // 3), n).astype(np.int32)
    price = rng.integers(-10 ** 9, 10 ** 9, n).astype(np.int64)
    qty = rng.integers(1, 50, n).astype(np.int32)
    g = qe.qe_groupby(ctx, cuda(lo), [(qe.SUM, cuda(price), cuda(qty)), (qe.COUNT, None, None),
                                      (qe.MIN, cuda(price), None), (qe.MAX, cuda(price), None)],
                      key_hi=cuda(hi), capacity=ngroups + 16, placement=placement)
    keys = (hi.astype(np.int64) << 32) | lo.astype(np.int64)
    rk, ra = O.groupby(keys, [(O.SUM, price * qty), (O.COUNT, None), (O.MIN, price), (O.MAX, price)])
    k, a = _sorted_groups(g)
    assert np.array_equal(k, rk)
    for x, y in zip(a, ra):
        assert np.array_equal(x, y)


def test_groupby_gather_and_errors(ctx):
    rng = np.random.default_rng(5)
    n = 90_000
    keys = rng.integers(-5, 5, n).astype(np.int64) * (2 ** 50)
    vals = rng.integers(-2 ** 62, 2 ** 62, n, dtype=np.int64)           # sums wrap
    rows = np.sort(rng.choice(n, 40_000, replace=False)).astype(np.int32)
    g = qe.qe_groupby(ctx, cuda(keys), [(qe.SUM, cuda(vals), None, True), (qe.COUNT, None, None)],
                      rows=cuda(rows), gather_lo=True, capacity=64)
    rk, ra = O.groupby(keys[rows], [(O.SUM, vals[rows]), (O.COUNT, None)])
    k, a = _sorted_groups(g)
    assert np.array_equal(k, rk) and np.array_equal(a[0], ra[0]) and np.array_equal(a[1], ra[1])
    with pytest.raises(qe.QeError) as e:
        qe.qe_groupby(ctx, cuda(np.arange(1000, dtype=np.int64)), [(qe.COUNT, None, None)], capacity=100)
    assert e.value.status == qe.ERR_CAPACITY and e.value.required > 100
    # a few groups too many: the exact number of groups is reported
    with pytest.raises(qe.QeError) as e:
        qe.qe_groupby(ctx, cuda(np.arange(150, dtype=np.int64).repeat(3)), [(qe.COUNT, None, None)], capacity=100)
    assert e.value.status == qe.ERR_CAPACITY and e.value.required == 150
    with pytest.raises(qe.QeError) as e:
        qe.qe_groupby(ctx, cuda(np.array([1, -2 ** 63], np.int64)), [(qe.COUNT, None, None)], capacity=8)
    assert e.value.status == qe.ERR_RESERVED_KEY
    g = qe.qe_groupby(ctx, torch.empty(0, dtype=torch.int64, device="cuda"), [(qe.COUNT, None, None)], capacity=8)
    assert int(g.ngroups.item()) == 0


# ---------------------------------------------------------------- pipeline
STAR_AGGS = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
STAR_Q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD,
                 aggs=[(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)])
COLS = ("fk", "date", "price", "qty", "flag")


def run_star(ctx, fact, dim, date_lt=1278, capacity=4096, expected=0, layout=qe.HT_AUTO, key_range=None):
    f = [fact[c].cuda() for c in COLS]
    d = qe.pipeline_desc(f, [(1, qe.LT, date_lt)], fk_col=0, dim_key=dim["key"].cuda(),
                         dim_payload=dim["attr"].cuda(), key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS,
                         expected_groups=expected, layout=layout, dim_key_range=key_range)
    return qe.qe_pipeline(ctx, d, capacity)


def oracle_star(fact, dim, date_lt=1278):
    q = O.Query(**{**STAR_Q.__dict__, "preds": [O.Pred(1, O.LT, date_lt)]})
    return O.pipeline([fact[c].numpy() for c in COLS], q, dim["key"].numpy(), dim["attr"].numpy())


def assert_groups_equal(g, ref):
    k, a = _sorted_groups(g)
    assert np.array_equal(k, ref["keys"])
    for x, y in zip(a, ref["aggs"]):
        assert np.array_equal(x, y)


def test_pipeline_golden(ctx):
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tiny_pipeline.json")))
    fact = {"fk": torch.tensor(gold["fact"]["fk"], dtype=torch.int32),
            "date": torch.tensor(gold["fact"]["date"], dtype=torch.int32),
            "price": torch.tensor(gold["fact"]["price"], dtype=torch.int64),
            "qty": torch.tensor(gold["fact"]["qty"], dtype=torch.int32),
            "flag": torch.tensor(gold["fact"]["flag"], dtype=torch.int8)}
    dim = {"key": torch.tensor(gold["dim"]["key"], dtype=torch.int32),
           "attr": torch.tensor(gold["dim"]["attr"], dtype=torch.int32)}
    g = run_star(ctx, fact, dim, gold["date_lt"], capacity=16)
    k, a = _sorted_groups(g)
    e = gold["expect"]
    assert k.tolist() == e["keys"]
    assert [x.tolist() for x in a] == [e["sum"], e["count"], e["min"], e["max"]]


@pytest.mark.parametrize("layout", [qe.HT_AUTO, qe.HT_OPEN])
def test_pipeline_config0(ctx, layout):
    """1M fact rows, 100K dim rows, 75 groups (the tiny star configuration)."""
    dim = datagen.star_dim(100_000, 25, seed=0)
    fact = datagen.star_fact(1_000_000, 100_000, seed=0)
    g = run_star(ctx, fact, dim, capacity=128, expected=75, layout=layout)
    ref = oracle_star(fact, dim)
    assert len(ref["keys"]) == 75
    assert_groups_equal(g, ref)


@pytest.mark.parametrize("date_lt", [0, 26, 1278, 2301, 2557])
def test_pipeline_selectivity_and_groups(ctx, date_lt):
    dim = datagen.star_dim(20_000, 1000, seed=1)
    fact = datagen.star_fact(300_007, 20_000, seed=1)
    g = run_star(ctx, fact, dim, date_lt, capacity=3100, expected=3000, key_range=(0, 19_999))
    assert_groups_equal(g, oracle_star(fact, dim, date_lt))


def test_pipeline_many_groups_hbm(ctx):
    """8334 attribute values x 3 flags = 25,002 groups (HBM group table)."""
    dim = datagen.star_dim(50_000, 8334, seed=2)
    fact = datagen.star_fact(400_000, 50_000, seed=2)
    g = run_star(ctx, fact, dim, capacity=30_000, expected=25_002)
    assert_groups_equal(g, oracle_star(fact, dim))


def test_pipeline_without_join_and_misses(ctx):
    rng = np.random.default_rng(8)
    n = 100_000
    code = rng.integers(0, 1000, n).astype(np.int32)
    v = rng.integers(0, 10 ** 6, n).astype(np.int64)
    d = qe.pipeline_desc([cuda(code), cuda(v)], [(1, qe.GE, 500_000)], fk_col=-1, key_lo_col=0,
                         aggs=[(qe.SUM, 1, -1), (qe.COUNT, -1, -1)])
    g = qe.qe_pipeline(ctx, d, 1024)
    q = O.Query(preds=[O.Pred(1, O.GE, 500_000)], fk_col=-1, key_lo_col=0,
                aggs=[(O.SUM, 1, -1), (O.COUNT, -1, -1)])
    assert_groups_equal(g, O.pipeline([code, v], q))
    # a join where some foreign keys have no dimension row (inner join drops them)
    dim = datagen.star_dim(5_000, 25, seed=4)
    fact = datagen.star_fact(60_000, 7_000, seed=4)
    g = run_star(ctx, fact, dim, capacity=128, expected=75)
    ref = oracle_star(fact, dim)
    assert ref["njoin"] < ref["nsel"]
    assert_groups_equal(g, ref)


@pytest.mark.parametrize("n", [1, 4097, 1_000_003])
def test_single_table_aggregation(ctx, n):
    """Filter + group-by with no join over the fact columns (a Q1-shaped
    query: SUM(price * qty), COUNT, MIN, MAX per flag), with the flag's range
    given as a column statistic, against the oracle."""
    fact = datagen.star_fact(n, 1000, seed=n % 89)
    f = [fact[c].cuda() for c in COLS[1:]]
    aggs = [(qe.SUM, 1, 2), (qe.COUNT, -1, -1), (qe.MIN, 1, -1), (qe.MAX, 1, -1)]
    d = qe.pipeline_desc(f, [(0, qe.LT, 1278)], key_hi_col=-1, key_lo_col=3, aggs=aggs, expected_groups=3,
                         est_selectivity=0.5, key_range=(None, (0, 2)))
    g = qe.qe_pipeline(ctx, d, 64)
    q = O.Query(preds=[O.Pred(0, O.LT, 1278)], fk_col=-1, key_hi_col=-1, key_lo_col=3,
                aggs=[(O.SUM, 1, 2), (O.COUNT, -1, -1), (O.MIN, 1, -1), (O.MAX, 1, -1)])
    assert_groups_equal(g, O.pipeline([fact[c].numpy() for c in COLS[1:]], q))


# ---------------------------------------------------------------- dense group layouts
def run_star_hint(ctx, fact, dim, key_range, capacity, date_lt=1278, expected=0):
    f = [fact[c].cuda() for c in COLS]
    d = qe.pipeline_desc(f, [(1, qe.LT, date_lt)], fk_col=0, dim_key=dim["key"].cuda(),
                         dim_payload=dim["attr"].cuda(), key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS,
                         expected_groups=expected, key_range=key_range)
    return qe.qe_pipeline(ctx, d, capacity)


@pytest.mark.parametrize("generic,items", [(False, 2), (False, 3), (True, 0)])
def test_pipeline_dense_smem_each_shape(ctx, generic, items):
    """The star-specialised kernel at 2 and 3 rows per thread, and the generic kernel."""
    ctx.set_tuning("force_generic", int(generic))
    ctx.set_tuning("star_items", items)
    try:
        dim = datagen.star_dim(20_000, 1000, seed=5)
        fact = datagen.star_fact(500_001, 20_000, seed=5)
        g = run_star_hint(ctx, fact, dim, ((0, 2), (0, 999)), 3100)
        assert_groups_equal(g, oracle_star(fact, dim))
    finally:
        ctx.set_tuning("force_generic", 0)
        ctx.set_tuning("star_items", 0)


@pytest.mark.parametrize("n_attr", [25, 1000])
def test_pipeline_star_wide_values(ctx, n_attr):
    """SUM(price * qty) whose products need all 64 bits (negative and large
    prices), into 75 groups (the star kernels keep SUM as 32-bit halves with
    carries) and 3,000 groups (64-bit SUM), in the single pipeline and in a
    batch (32-bit halves for both)."""
    rng = np.random.default_rng(21)
    dim = datagen.star_dim(20_000, n_attr, seed=21)
    fact = dict(datagen.star_fact(700_001, 20_000, seed=21))
    fact["price"] = torch.from_numpy(rng.integers(-2 ** 40, 2 ** 40, 700_001, dtype=np.int64))
    fact["price"][::7] = 2 ** 62 + 12345                  # products wrap modulo 2^64
    ref = oracle_star(fact, dim)
    kr = ((0, 2), (0, n_attr - 1))
    g = run_star_hint(ctx, fact, dim, kr, 3100)
    assert_groups_equal(g, ref)
    f = [fact[c].cuda() for c in COLS]
    d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=dim["key"].cuda(), dim_payload=dim["attr"].cuda(),
                         key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS, dim_key_range=(0, 19_999),
                         key_range=kr, expected_groups=3 * n_attr)
    gb, o = qe.alloc_groups(3100, 4, torch.device("cuda"))
    qe.qe_batch_run(ctx, [d], [o], opts=qe.qe_batch_opts(0, 1 << 16, 0, 0))
    assert_groups_equal(gb, ref)


@pytest.mark.parametrize("generic", [False, True])
def test_pipeline_dense_hint_too_narrow_spills(ctx, generic):
    ctx.set_tuning("force_generic", int(generic))
    try:
        dim = datagen.star_dim(20_000, 100, seed=6)
        fact = datagen.star_fact(300_000, 20_000, seed=6)
        g = run_star_hint(ctx, fact, dim, ((1, 1), (10, 49)), 400)   # most keys fall outside
        assert_groups_equal(g, oracle_star(fact, dim))
    finally:
        ctx.set_tuning("force_generic", 0)


@pytest.mark.parametrize("n", [1_000, 400_000, 3_000_001])
def test_pipeline_dense_hbm_25k(ctx, n):
    """25,002 groups: a direct array too large for one SM's shared memory,
    kept in HBM."""
    dim = datagen.star_dim(50_000, 8334, seed=7)
    fact = datagen.star_fact(n, 50_000, seed=7)
    g = run_star_hint(ctx, fact, dim, ((0, 2), (0, 8333)), 30_000)
    assert_groups_equal(g, oracle_star(fact, dim))


def test_pipeline_dense_payload_only(ctx):
    """Group by the joined attribute alone; its range comes from the build."""
    dim = datagen.star_dim(30_000, 77, seed=8)
    fact = datagen.star_fact(250_000, 30_000, seed=8)
    f = [fact[c].cuda() for c in COLS]
    d = qe.pipeline_desc(f, [(1, qe.GE, 700)], fk_col=0, dim_key=dim["key"].cuda(), dim_payload=dim["attr"].cuda(),
                         key_hi_col=-1, key_lo_col=qe.JOIN_PAYLOAD, aggs=[(qe.MAX, 3, -1), (qe.SUM, 2, -1)])
    g = qe.qe_pipeline(ctx, d, 128)
    q = O.Query(preds=[O.Pred(1, O.GE, 700)], fk_col=0, key_hi_col=-1, key_lo_col=O.JOIN_PAYLOAD,
                aggs=[(O.MAX, 3, -1), (O.SUM, 2, -1)])
    ref = O.pipeline([fact[c].numpy() for c in COLS], q, dim["key"].numpy(), dim["attr"].numpy())
    assert_groups_equal(g, ref)


# ---------------------------------------------------------------- batched form
def _batch_inputs(sizes, seed, prebuilt=None, ctx=None, hint=True):
    """Config-0-schema pipelines (attr in [0,25)); returns descs, outs, refs."""
    descs, outs, groups, refs, keep = [], [], [], [], []
    for i, n in enumerate(sizes):
        nd = max(1, n // 10)
        dim = datagen.star_dim(nd, 25, seed=seed * 1000 + i)
        fact = datagen.star_fact(n, nd, seed=seed * 1000 + i)
        f = [fact[c].cuda() for c in COLS]
        dk, da = dim["key"].cuda(), dim["attr"].cuda()
        ht = None
        if prebuilt is not None and prebuilt(i):
            ht = qe.qe_join_build(ctx, dk, da)
        d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=dk, dim_payload=da, ht=ht, key_hi_col=4,
                             key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS, dim_key_range=(0, nd - 1),
                             key_range=((0, 2), (0, 24)) if hint else None, expected_groups=75)
        g, o = qe.alloc_groups(128, 4, torch.device("cuda"))
        descs.append(d)
        outs.append(o)
        groups.append(g)
        refs.append(oracle_star(fact, dim))
        keep.append((f, dk, da, ht))
    return descs, outs, groups, refs, keep


@pytest.mark.parametrize("hint", [True, False])
def test_batch_run_matches_oracle(ctx, hint):
    sizes = [0, 1, 999, 2048, 5000, 70_001, 200_000, 33]
    descs, outs, groups, refs, keep = _batch_inputs(sizes, seed=9, hint=hint)
    qe.qe_batch_run(ctx, descs, outs, opts=qe.qe_batch_opts(0, 1 << 16, 0, 0))
    for g, r in zip(groups, refs):
        assert_groups_equal(g, r)


def test_batch_graph_relaunch_prebuilt_and_solo_equivalence(ctx):
    sizes = [4096, 123_457, 1, 60_000, 0, 300_000]
    descs, outs, groups, refs, keep = _batch_inputs(sizes, seed=10, prebuilt=lambda i: i % 2 == 0, ctx=ctx)
    b = qe.Batch(ctx, descs, outs, qe.qe_batch_opts(0, 1 << 15, 0, 1))
    for _ in range(2):                      # the graph clears its tables each launch
        for g in groups:
            g.ngroups.fill_(-1)
        b.launch()
        ctx.sync_status()
        for g, r in zip(groups, refs):
            assert_groups_equal(g, r)
    b.destroy()
    # each pipeline alone gives the same result as in the batch
    for d, g in zip(descs, groups):
        solo = qe.qe_pipeline(ctx, d, 128)
        a, bb = _sorted_groups(solo), _sorted_groups(g)
        assert np.array_equal(a[0], bb[0]) and all(np.array_equal(x, y) for x, y in zip(a[1], bb[1]))
    for k in keep:
        if k[3] is not None:
            k[3].destroy()


def test_batch_hbm_tables_only(ctx):
    sizes = [50_000, 7, 90_000]
    descs, outs, groups, refs, keep = _batch_inputs(sizes, seed=11)
    qe.qe_batch_run(ctx, descs, outs, opts=qe.qe_batch_opts(0, 1 << 16, -1, 0))
    for g, r in zip(groups, refs):
        assert_groups_equal(g, r)
