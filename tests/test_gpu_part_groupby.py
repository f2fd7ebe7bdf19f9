"""GPU parity of the partitioned group-by (partition-then-aggregate) against
the CPU oracle, bit-exact.

A pipeline whose groups only fit an HBM hash table far larger than L2 runs
as: count each row's part (top bits of the key's hash), scan, scatter the
survivors into per-part segments, split every part into sub-parts (the next
hash bits), then aggregate each sub-part in one block's shared-memory hash
table and write its groups straight into the output (Sec. 7.2 on large hash
tables; Sec. 2.2 on one partitioning function applied before the local
operator).  The knob "gb_partition" = 2 forces that path at test sizes,
"gb_part_log2p" sets the number of parts (2 .. 1024 are covered) and
"gb_part_log2q" the sub-parts, so the spill to the HBM table of keys that
find no shared slot is covered too, as are group keys from fact columns
(every row counted from its key columns) and from the join payload
(survivors counted), semi- and anti-joins, empty and ragged inputs, many
groups per part, averages, reserved keys and too-small outputs.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_09226_gb300 import datagen
from paper_2506_09226_gb300 import qe

pytestmark = pytest.mark.gpu

SKEW = ("fk", "date", "price", "qty", "flag", "code", "gkey")
AGGS = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
O_AGGS = [(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)]


@pytest.fixture(scope="module")
def ctx():
    c = qe.Context(0)
    c.set_tuning("gb_partition", 2)
    yield c
    c.set_tuning("gb_partition", 0)
    c.set_tuning("gb_part_log2p", 0)
    c.close()


def _sorted(g):
    k, a = g.to_host()
    o = np.argsort(k.numpy(), kind="stable")
    return k.numpy()[o], [x.numpy()[o] for x in a]


def _equal(g, ref):
    k, a = _sorted(g)
    assert len(k) == len(ref["keys"])
    assert np.array_equal(k, ref["keys"])
    for x, y in zip(a, ref["aggs"]):
        assert np.array_equal(x, y)


def _skew(n, nd, groups, seed):
    dim = datagen.star_dim(nd, 1000, seed=seed)
    fact = datagen.star_fact(n, nd, seed=seed, zipf_s=1.1, n_codes=100_000, n_gkeys=groups)
    return fact, dim


def _run(ctx, fact, dim, key_col, date_lt, capacity, kind=qe.INNER, key_hi=-1, avg=()):
    f = [fact[c].cuda() for c in SKEW]
    dk = dim["key"].cuda() if kind == qe.INNER else dim["key"][: len(dim["key"]) // 2].contiguous().cuda()
    d = qe.pipeline_desc(f, [(1, qe.LT, date_lt)], fk_col=0, dim_key=dk,
                         dim_payload=dim["attr"].cuda() if kind == qe.INNER else None,
                         key_hi_col=key_hi, key_lo_col=key_col, aggs=AGGS, expected_groups=capacity,
                         join_kind=kind)
    return qe.qe_pipeline(ctx, d, capacity, avg=avg)


def _oracle(fact, dim, key_col, date_lt, kind=O.INNER, key_hi=-1):
    q = O.Query(preds=[O.Pred(1, O.LT, date_lt)], fk_col=0, key_hi_col=key_hi,
                key_lo_col=O.JOIN_PAYLOAD if key_col == qe.JOIN_PAYLOAD else key_col, aggs=O_AGGS, join_kind=kind)
    dk = dim["key"].numpy() if kind == O.INNER else dim["key"][: len(dim["key"]) // 2].numpy()
    return O.pipeline([fact[c].numpy() for c in SKEW], q, dk, dim["attr"].numpy() if kind == O.INNER else None)


@pytest.mark.parametrize("log2p,generic", [(1, False), (3, False), (8, False), (10, False), (8, True)])
def test_part_groupby_int64_keys(ctx, log2p, generic):
    """~200K distinct int64 keys over 1M rows: keys from a fact column (every
    row counted from the key column), at 2 .. 1024 parts, through the
    star-shape scatter (register-prefetched) and the generic one."""
    ctx.set_tuning("gb_part_log2p", log2p)
    ctx.set_tuning("force_generic", int(generic))
    try:
        fact, dim = _skew(1_000_003, 50_000, 200_000, seed=61)
        g = _run(ctx, fact, dim, 6, 1278, 262_144)
        _equal(g, _oracle(fact, dim, 6, 1278))
    finally:
        ctx.set_tuning("gb_part_log2p", 0)
        ctx.set_tuning("force_generic", 0)


@pytest.mark.parametrize("log2q", [4, 5])
def test_part_groupby_spill(ctx, log2q):
    """Too few sub-parts for the groups (200K groups in 2 x 16 or 2 x 32
    sub-parts of a 4,096-slot shared table): a third of the keys, or a few,
    find no shared slot and spill to the HBM table; the result is still
    exact."""
    ctx.set_tuning("gb_part_log2p", 1)
    ctx.set_tuning("gb_part_log2q", log2q)
    try:
        fact, dim = _skew(800_000, 20_000, 200_000, seed=69)
        g = _run(ctx, fact, dim, 6, 2557, 1 << 20)
        _equal(g, _oracle(fact, dim, 6, 2557))
    finally:
        ctx.set_tuning("gb_part_log2p", 0)
        ctx.set_tuning("gb_part_log2q", -1)


@pytest.mark.parametrize("date_lt,fold2", [(0, 0), (26, 0), (2301, 0), (2557, 0), (26, 1), (2301, 1)])
def test_part_groupby_selectivity(ctx, date_lt, fold2):
    """0 %, 1 %, 90 % and 100 % of the rows, dictionary-code keys; the fold
    as one 1,024-thread block per SM and as two 512-thread blocks."""
    ctx.set_tuning("gb_fold2", fold2)
    try:
        fact, dim = _skew(700_001, 30_000, 100_000, seed=62)
        g = _run(ctx, fact, dim, 5, date_lt, 131_072)
        _equal(g, _oracle(fact, dim, 5, date_lt))
    finally:
        ctx.set_tuning("gb_fold2", 0)


def test_part_groupby_payload_and_hi_keys(ctx):
    """Group key (code, join payload): the survivors of filter and join are
    counted, and the key packs two parts."""
    fact, dim = _skew(600_000, 40_000, 1000, seed=63)
    g = _run(ctx, fact, dim, qe.JOIN_PAYLOAD, 2000, 1 << 20, key_hi=5)
    _equal(g, _oracle(fact, dim, qe.JOIN_PAYLOAD, 2000, key_hi=5))


@pytest.mark.parametrize("kind", [qe.SEMI, qe.ANTI])
def test_part_groupby_semi_anti(ctx, kind):
    fact, dim = _skew(500_000, 20_000, 50_000, seed=64)
    g = _run(ctx, fact, dim, 6, 1800, 65_536, kind=kind)
    _equal(g, _oracle(fact, dim, 6, 1800, kind=O.SEMI if kind == qe.SEMI else O.ANTI))


@pytest.mark.parametrize("n", [0, 1, 1023, 1025, 2049])
def test_part_groupby_tiny_and_ragged(ctx, n):
    fact, dim = _skew(n, 100, 500, seed=65 + n)
    g = _run(ctx, fact, dim, 6, 2000, 1024)
    _equal(g, _oracle(fact, dim, 6, 2000))


def test_part_groupby_averages_and_skewed_keys(ctx):
    """A key that holds a third of the rows (one part far larger than the
    others) and the derived averages."""
    fact, dim = _skew(900_000, 30_000, 80_000, seed=66)
    fact = dict(fact)
    fact["gkey"] = fact["gkey"].clone()
    fact["gkey"][::3] = 12345
    g = _run(ctx, fact, dim, 6, 1500, 131_072, avg=[0])
    ref = _oracle(fact, dim, 6, 1500)
    _equal(g, ref)
    k, _ = g.to_host()
    o = np.argsort(k.numpy(), kind="stable")
    got = g.avg_host(0).numpy()[o]
    want = O.avg(ref["aggs"][0], ref["aggs"][1])
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want))


def test_part_groupby_errors(ctx):
    """More groups than the output holds: QE_ERR_CAPACITY with the count; a
    group key equal to INT64_MIN: QE_ERR_RESERVED_KEY."""
    fact, dim = _skew(300_000, 10_000, 100_000, seed=67)
    with pytest.raises(qe.QeError) as e:
        _run(ctx, fact, dim, 6, 2557, 20_000)
    assert e.value.status == qe.ERR_CAPACITY and e.value.required > 20_000
    fact = dict(fact)
    fact["gkey"] = fact["gkey"].clone()
    fact["gkey"][777] = -2 ** 63
    fact["date"] = fact["date"].clone()
    fact["date"][777] = 0
    with pytest.raises(qe.QeError) as e:
        _run(ctx, fact, dim, 6, 2557, 200_000)
    assert e.value.status == qe.ERR_RESERVED_KEY


def test_part_groupby_matches_unpartitioned(ctx):
    """The partitioned and the direct HBM-table paths give the same groups
    (2M rows, ~400K groups)."""
    fact, dim = _skew(2_000_000, 100_000, 400_000, seed=68)
    g1 = _sorted(_run(ctx, fact, dim, 6, 1278, 524_288))
    ctx.set_tuning("gb_partition", 1)
    try:
        g2 = _sorted(_run(ctx, fact, dim, 6, 1278, 524_288))
    finally:
        ctx.set_tuning("gb_partition", 2)
    assert np.array_equal(g1[0], g2[0])
    for x, y in zip(g1[1], g2[1]):
        assert np.array_equal(x, y)


def test_autotuned_placement_matches_oracle(ctx, tmp_path):
    """The autotuner times the direct HBM table against the partitioned
    group-by at three fan-outs, with a dense and an open-addressing join
    table, applies the fastest, and the result of that choice is exact."""
    from paper_2506_09226_gb300 import tune
    fact, dim = _skew(1_500_000, 60_000, 300_000, seed=70)
    f = [fact[c].cuda() for c in SKEW]
    d = qe.pipeline_desc(f, [(1, qe.LT, 1500)], fk_col=0, dim_key=dim["key"].cuda(), dim_payload=dim["attr"].cuda(),
                         key_hi_col=-1, key_lo_col=6, aggs=AGGS, expected_groups=524_288)
    g, o = qe.alloc_groups(524_288, 4, torch.device("cuda"))
    stream = torch.cuda.current_stream()
    try:
        best = tune.tune_group_placement(ctx, d, lambda: qe.qe_pipeline(ctx, d, 524_288, check=False, out=(g, o)),
                                         stream, path=str(tmp_path / "tune.json"))
        assert best in [(p, lp, lay) for p, lp in tune.GROUP_PLACEMENT for lay in tune.JOIN_LAYOUTS]
        qe.qe_pipeline(ctx, d, 524_288, out=(g, o))
        _equal(g, _oracle(fact, dim, 6, 1500))
    finally:
        ctx.set_tuning("gb_partition", 2)
        ctx.set_tuning("gb_part_log2p", 0)
