"""GPU parity of the derived FP64 averages (Sec. 2.3 lists average among the
aggregation kinds) against the CPU oracle.

The library derives avg = (double)SUM / (double)COUNT from the exact int64
SUM and COUNT of each group when the output asks for it.  Every test calls
the C ABI and compares with oracle.avg over the oracle's own SUM and COUNT,
within 1e-12 relative (both sides take one rounding of the sum and one IEEE
division, so the results are expected to agree exactly; 1e-12 is the stated
bound).  Covered: the shared-memory and HBM hash tables of qe_groupby, the
star kernel (shared-memory direct array), the HBM direct array, the generic
pipeline kernel, a batch, a group with count 1, sums near 2^62 and negative
sums, and the argument checks.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_09226_gb300 import datagen
from paper_2506_09226_gb300 import qe

pytestmark = pytest.mark.gpu

REL = 1e-12
COLS = ("fk", "date", "price", "qty", "flag")
STAR_AGGS = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
O_STAR = [(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)]


@pytest.fixture(scope="module")
def ctx():
    c = qe.Context(0)
    yield c
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(g, a, ref_keys, ref_sum, ref_cnt):
    """Group keys, SUM and COUNT exactly; the average of aggregate a within REL."""
    k, aggs = g.to_host()
    avg = g.avg_host(a).numpy()
    o = np.argsort(k.numpy(), kind="stable")
    assert np.array_equal(k.numpy()[o], ref_keys)
    want = O.avg(ref_sum, ref_cnt)
    got = avg[o]
    assert np.all(np.isfinite(got))
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-300)
    assert np.all((got == want) | (err <= REL)), float(err.max())
    return got, want


@pytest.mark.parametrize("placement", [qe.GB_AUTO, qe.GB_HBM])
def test_groupby_avg_edge_values(ctx, placement):
    """Groups of one row with sums near 2^62 and -2^63, negative sums,
    thirds, and a large group, through both group-table placements."""
    rng = np.random.default_rng(3)
    n = 200_003
    keys = rng.integers(0, 5000, n).astype(np.int64)
    vals = rng.integers(-10 ** 9, 10 ** 9, n).astype(np.int64)
    keys[:4] = [10_001, 10_002, 10_003, 10_004]              # count-1 groups
    vals[:4] = [2 ** 62 + 1, -(2 ** 63 - 1), 2 ** 53 + 3, -7]
    keys[4:7] = 10_005                                      # 1/3 and 2/3 of small sums
    vals[4:7] = [1, 0, 0]
    g = qe.qe_groupby(ctx, cuda(keys), [(qe.SUM, cuda(vals), None), (qe.COUNT, None, None)], capacity=8192,
                      placement=placement, avg=[0])
    rk, (rs, rc) = O.groupby(keys, [(O.SUM, vals), (O.COUNT, None)])
    got, want = _check(g, 0, rk, rs, rc)
    i = int(np.searchsorted(rk, 10_001))
    assert rc[i] == 1 and got[i] == 2.0 ** 62
    assert got[int(np.searchsorted(rk, 10_002))] == -(2.0 ** 63)
    assert got[int(np.searchsorted(rk, 10_005))] == 1 / 3


def test_pipeline_star_avg(ctx):
    """The star kernel (3,000 groups in a shared-memory direct array): the
    average of SUM(price*qty) over COUNT."""
    dim = datagen.star_dim(20_000, 1000, seed=5)
    fact = datagen.star_fact(500_001, 20_000, seed=5)
    f = [fact[c].cuda() for c in COLS]
    d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=dim["key"].cuda(), dim_payload=dim["attr"].cuda(),
                         key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS, key_range=((0, 2), (0, 999)))
    g = qe.qe_pipeline(ctx, d, 3100, avg=[0])
    q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD, aggs=O_STAR)
    r = O.pipeline([fact[c].numpy() for c in COLS], q, dim["key"].numpy(), dim["attr"].numpy())
    _check(g, 0, r["keys"], r["aggs"][0], r["aggs"][1])


@pytest.mark.parametrize("mode", ["hbm_dense", "generic_hash"])
def test_pipeline_avg_other_tables(ctx, mode):
    """AVG(price) with 25,002 groups in the HBM direct array, and through the
    generic kernel's hash tables (no key range)."""
    dim = datagen.star_dim(50_000, 8334, seed=7)
    fact = datagen.star_fact(400_000, 50_000, seed=7)
    f = [fact[c].cuda() for c in COLS]
    aggs = [(qe.SUM, 2, -1), (qe.COUNT, -1, -1), (qe.MAX, 3, -1)]
    kr = ((0, 2), (0, 8333)) if mode == "hbm_dense" else None
    d = qe.pipeline_desc(f, [(1, qe.GE, 1000)], fk_col=0, dim_key=dim["key"].cuda(), dim_payload=dim["attr"].cuda(),
                         key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD, aggs=aggs, key_range=kr, expected_groups=25_002)
    g = qe.qe_pipeline(ctx, d, 30_000, avg=[0])
    q = O.Query(preds=[O.Pred(1, O.GE, 1000)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD,
                aggs=[(O.SUM, 2, -1), (O.COUNT, -1, -1), (O.MAX, 3, -1)])
    r = O.pipeline([fact[c].numpy() for c in COLS], q, dim["key"].numpy(), dim["attr"].numpy())
    _check(g, 0, r["keys"], r["aggs"][0], r["aggs"][1])


def test_batch_avg(ctx):
    """Averages written by the batch kernel's own compaction, for a pipeline
    whose direct array is in shared memory and one without a key range."""
    descs, outs, groups, refs, keep = [], [], [], [], []
    for i, (n, hint) in enumerate([(150_000, True), (90_001, False), (1, True)]):
        nd = max(1, n // 10)
        dim = datagen.star_dim(nd, 25, seed=40 + i)
        fact = datagen.star_fact(n, nd, seed=40 + i)
        f = [fact[c].cuda() for c in COLS]
        dk, da = dim["key"].cuda(), dim["attr"].cuda()
        d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=dk, dim_payload=da, key_hi_col=4,
                             key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS, dim_key_range=(0, nd - 1),
                             key_range=((0, 2), (0, 24)) if hint else None, expected_groups=75)
        g, o = qe.alloc_groups(128, 4, torch.device("cuda"), avg=[0])
        descs.append(d)
        outs.append(o)
        groups.append(g)
        q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD, aggs=O_STAR)
        refs.append(O.pipeline([fact[c].numpy() for c in COLS], q, dim["key"].numpy(), dim["attr"].numpy()))
        keep.append((f, dk, da))
    qe.qe_batch_run(ctx, descs, outs, opts=qe.qe_batch_opts(0, 1 << 16, 0, 0))
    for g, r in zip(groups, refs):
        _check(g, 0, r["keys"], r["aggs"][0], r["aggs"][1])


def test_avg_argument_checks(ctx):
    """An average over a non-SUM aggregate, or without a COUNT, is rejected
    before anything runs."""
    keys = cuda(np.arange(100, dtype=np.int64) % 7)
    vals = cuda(np.arange(100, dtype=np.int64))
    with pytest.raises(qe.QeError) as e:
        qe.qe_groupby(ctx, keys, [(qe.MIN, vals, None), (qe.COUNT, None, None)], capacity=16, avg=[0])
    assert e.value.status == qe.ERR_INVALID_ARG
    with pytest.raises(qe.QeError) as e:
        qe.qe_groupby(ctx, keys, [(qe.SUM, vals, None), (qe.MAX, vals, None)], capacity=16, avg=[0])
    assert e.value.status == qe.ERR_INVALID_ARG
    with pytest.raises(qe.QeError) as e:
        qe.qe_groupby(ctx, keys, [(qe.SUM, vals, None), (qe.COUNT, None, None)], capacity=16, avg=[2])
    assert e.value.status == qe.ERR_INVALID_ARG
