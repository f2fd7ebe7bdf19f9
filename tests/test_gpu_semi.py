"""GPU parity of the semi- and anti-join against the CPU oracle (bit-exact).

qe_join_semi over key sets (repeated keys) and over unique-key tables, both
layouts, with and without a selection vector, one- and two-pass; pipelines
whose join is a semi- or anti-join (built in the call, or against a
prebuilt key set; dense and open layouts; grouped by fact columns); and the
same pipelines inside a batch, each equal to its solo run and the oracle.
Edge cases: empty sides, repeated keys, INT32_MIN, the output capacity, and
the argument errors (a probe of a key set, a payload key of a semi-join).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_09226_gb300 import datagen
from paper_2506_09226_gb300 import qe

pytestmark = pytest.mark.gpu

COLS = ("fk", "date", "price", "qty", "flag")
AGGS = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
O_AGGS = [(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)]


@pytest.fixture(scope="module")
def ctx():
    c = qe.Context(0)
    yield c
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_semi(ctx, ht, pk, sel, bk, anti):
    rows, cnt = qe.qe_join_semi(ctx, ht, cuda(pk), cuda(sel) if sel is not None else None, anti=anti)
    ref = O.semi_join(bk, pk, sel, anti)
    c = int(cnt.item())
    assert c == len(ref)
    assert np.array_equal(rows[:c].cpu().numpy(), ref)


@pytest.mark.parametrize("layout", [qe.HT_DENSE, qe.HT_OPEN, qe.HT_AUTO])
@pytest.mark.parametrize("with_sel", [False, True])
def test_semi_anti_key_set(ctx, layout, with_sel):
    rng = np.random.default_rng(layout * 2 + with_sel + 40)
    nb, npr = 50_000, 200_001
    bk = rng.integers(-40_000, 40_000, nb).astype(np.int32)            # repeats
    pk = rng.integers(-60_000, 60_000, npr).astype(np.int32)
    sel = np.sort(rng.choice(npr, 77_777, replace=False)).astype(np.int32) if with_sel else None
    ht = qe.qe_join_build_set(ctx, cuda(bk), layout=layout)
    info = ht.info()
    assert info.key_set == 1 and info.full == 0
    assert info.layout == (qe.HT_DENSE if layout == qe.HT_AUTO else layout)
    if info.layout == qe.HT_DENSE:
        assert info.bytes == (info.slots + 31) // 32 * 4               # the bitmap alone
    for anti in (False, True):
        _check_semi(ctx, ht, pk, sel, bk, anti)
    ht.destroy()


@pytest.mark.parametrize("layout", [qe.HT_DENSE, qe.HT_OPEN])
def test_semi_anti_unique_table_and_two_pass(ctx, layout):
    """A table from qe_join_build serves the semi-join too; 9M positions take
    the two-pass compaction."""
    rng = np.random.default_rng(50 + layout)
    nb, npr = 300_000, 9_000_007
    bk = rng.choice(np.arange(-500_000, 500_000), nb, replace=False).astype(np.int32)
    pk = rng.integers(-600_000, 600_000, npr).astype(np.int32)
    sel = np.sort(rng.choice(npr, 5_000_000, replace=False)).astype(np.int32)
    ht = qe.qe_join_build(ctx, cuda(bk), cuda(np.zeros(nb, np.int32)), layout=layout)
    for s in (None, sel):
        for anti in (False, True):
            _check_semi(ctx, ht, pk, s, bk, anti)
    ht.destroy()


def test_semi_edges_and_errors(ctx):
    e32 = torch.empty(0, dtype=torch.int32, device="cuda")
    # empty key set: the semi-join keeps nothing, the anti-join everything
    ht = qe.qe_join_build_set(ctx, e32)
    pk = np.array([3, -2 ** 31, 7], np.int32)
    _check_semi(ctx, ht, pk, None, np.empty(0, np.int32), False)
    _check_semi(ctx, ht, pk, None, np.empty(0, np.int32), True)
    rows, cnt = qe.qe_join_semi(ctx, ht, e32)
    assert int(cnt.item()) == 0
    ht.destroy()
    # INT32_MIN is an ordinary key of a dense set; the open layout reserves it
    bk = np.array([-2 ** 31, -2 ** 31, -2 ** 31 + 2], np.int32)
    ht = qe.qe_join_build_set(ctx, cuda(bk), layout=qe.HT_DENSE)
    _check_semi(ctx, ht, np.array([-2 ** 31 + 2, 0, -2 ** 31, -2 ** 31 + 1], np.int32), None, bk, False)
    # a key set has no payloads to probe
    with pytest.raises(qe.QeError) as e:
        qe.qe_join_probe(ctx, ht, cuda(pk))
    assert e.value.status == qe.ERR_INVALID_ARG
    ht.destroy()
    with pytest.raises(qe.QeError) as e:
        qe.qe_join_build_set(ctx, cuda(bk), layout=qe.HT_OPEN)
    assert e.value.status == qe.ERR_RESERVED_KEY
    # too small an output: nothing past the capacity, the required count reported
    ht = qe.qe_join_build_set(ctx, cuda(np.arange(100, dtype=np.int32)))
    out = torch.full((10,), -5, dtype=torch.int32, device="cuda")
    with pytest.raises(qe.QeError) as e:
        qe.qe_join_semi(ctx, ht, cuda(np.arange(50, dtype=np.int32)), capacity=4, out_rows=out)
    assert e.value.status == qe.ERR_CAPACITY
    assert out[4:].cpu().tolist() == [-5] * 6
    ht.destroy()


# ---------------------------------------------------------------- pipelines
def _semi_case(seed, n_fact, n_dimkeys, key_span):
    """Fact rows whose foreign keys fall partly outside a multiset of dim keys."""
    rng = np.random.default_rng(seed)
    fact = datagen.star_fact(n_fact, key_span, seed=seed)
    dk = rng.integers(0, key_span, n_dimkeys).astype(np.int32)
    return fact, dk


def _run(ctx, fact, dk, kind, layout=qe.HT_AUTO, ht=None, key_lo=4, capacity=64):
    f = [fact[c].cuda() for c in COLS]
    d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=cuda(dk) if ht is None else None, ht=ht,
                         key_hi_col=-1, key_lo_col=key_lo, aggs=AGGS, layout=layout, join_kind=kind)
    return qe.qe_pipeline(ctx, d, capacity), d


def _oracle(fact, dk, kind, key_lo=4, dp=None):
    q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0, key_hi_col=-1, key_lo_col=key_lo, aggs=O_AGGS,
                join_kind=kind)
    if kind == O.INNER and dp is None:
        dp = np.zeros(len(dk), np.int32)
    return O.pipeline([fact[c].numpy() for c in COLS], q, dk, dp)


def _assert_groups(g, ref):
    k, a = g.to_host()
    o = np.argsort(k.numpy(), kind="stable")
    assert np.array_equal(k.numpy()[o], ref["keys"])
    for x, y in zip(a, ref["aggs"]):
        assert np.array_equal(x.numpy()[o], y)


@pytest.mark.parametrize("kind", [qe.SEMI, qe.ANTI])
@pytest.mark.parametrize("layout", [qe.HT_DENSE, qe.HT_OPEN])
def test_pipeline_semi_anti(ctx, kind, layout):
    fact, dk = _semi_case(60 + kind + layout, 300_007, 40_000, 60_000)
    g, _ = _run(ctx, fact, dk, kind, layout)
    ref = _oracle(fact, dk, kind)
    assert 0 < ref["njoin"] < ref["nsel"]
    _assert_groups(g, ref)
    # grouped by the int32 foreign key itself (many groups, HBM table)
    g, _ = _run(ctx, fact, dk, kind, layout, key_lo=0, capacity=70_000)
    _assert_groups(g, _oracle(fact, dk, kind, key_lo=0))


@pytest.mark.parametrize("kind", [qe.SEMI, qe.ANTI])
def test_pipeline_semi_anti_flag_groups(ctx, kind):
    """The shape bench.py times: a key set of half of a permuted key range,
    the flag's range given as a column statistic, three groups."""
    fact = datagen.star_fact(1_000_003, 200_000, seed=80 + kind)
    dk = datagen.star_dim(200_000, 1, seed=80 + kind)["key"][:100_000].numpy()
    f = [fact[c].cuda() for c in COLS]
    d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=cuda(dk), key_hi_col=-1, key_lo_col=4,
                         aggs=AGGS, expected_groups=3, est_selectivity=0.5, key_range=(None, (0, 2)),
                         join_kind=kind)
    g = qe.qe_pipeline(ctx, d, 64)
    ref = _oracle(fact, dk, kind)
    assert len(ref["keys"]) == 3
    _assert_groups(g, ref)


# Group keys of the star kinds without a join payload: (key_hi, key_lo, key
# range) -- int8 flag alone (3 slots); (flag, int32 qty) (150 slots); the
# int32 foreign key over 5,000 values (shared-memory array past the 32-bit
# SUM halves) and over 60,000 values (array in HBM); a range that leaves
# flag 2 out (those rows go to the HBM hash table).
STAR_KEYS = {
    "flag": (-1, 4, (None, (0, 2)), 5_000),
    "flag_qty": (4, 3, ((0, 2), (1, 50)), 5_000),
    "fk_5000": (-1, 0, (None, (0, 4_999)), 5_000),
    "fk_60000": (-1, 0, (None, (0, 59_999)), 60_000),
    "flag_spill": (-1, 4, (None, (0, 1)), 5_000),
}


@pytest.mark.parametrize("kind", [qe.SEMI, qe.ANTI, "none"])
@pytest.mark.parametrize("shape", list(STAR_KEYS))
def test_pipeline_star_kinds(ctx, kind, shape):
    """The star kernel for semi- / anti-joins and for no join, against the
    oracle and against the generic kernel, on 1M rows (several tiles per
    block and a ragged tail) whose foreign keys partly fall outside the key
    set's range."""
    hi, lo, rng_, span = STAR_KEYS[shape]
    seed = 90 + len(shape) + (3 if kind == "none" else kind)
    fact = datagen.star_fact(1_000_003, span, seed=seed)
    # keys below span/10 or from 9 span/10 up lie outside the key set's range
    dk = np.random.default_rng(seed).integers(span // 10, span - span // 10, span // 2).astype(np.int32)
    f = [fact[c].cuda() for c in COLS]
    join = kind != "none"
    d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0 if join else -1, dim_key=cuda(dk) if join else None,
                         key_hi_col=hi, key_lo_col=lo, aggs=AGGS, key_range=rng_,
                         join_kind=kind if join else qe.INNER)
    q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0 if join else -1, key_hi_col=hi, key_lo_col=lo, aggs=O_AGGS,
                join_kind=kind if join else O.INNER)
    ref = O.pipeline([fact[c].numpy() for c in COLS], q, dk if join else None, None)
    if join:
        assert 0 < ref["njoin"] < ref["nsel"]
    _assert_groups(qe.qe_pipeline(ctx, d, 70_000), ref)
    ctx.set_tuning("force_generic", 1)
    try:
        _assert_groups(qe.qe_pipeline(ctx, d, 70_000), ref)
    finally:
        ctx.set_tuning("force_generic", 0)


@pytest.mark.parametrize("kind", [qe.SEMI, qe.ANTI])
def test_pipeline_semi_anti_prebuilt_set(ctx, kind):
    fact, dk = _semi_case(70 + kind, 100_000, 5_000, 20_000)
    ht = qe.qe_join_build_set(ctx, cuda(dk))
    g, _ = _run(ctx, fact, dk, kind, ht=ht)
    _assert_groups(g, _oracle(fact, dk, kind))
    # an inner join cannot use a key set
    f = [fact[c].cuda() for c in COLS]
    with pytest.raises(qe.QeError) as e:
        qe.qe_pipeline(ctx, qe.pipeline_desc(f, [], fk_col=0, ht=ht, key_hi_col=-1, key_lo_col=4, aggs=AGGS), 64)
    assert e.value.status == qe.ERR_INVALID_ARG
    ht.destroy()
    # a semi- or anti-join has no payload to group by
    with pytest.raises(qe.QeError) as e:
        _run(ctx, fact, dk, kind, key_lo=qe.JOIN_PAYLOAD)
    assert e.value.status == qe.ERR_INVALID_ARG


def test_batch_semi_anti_mixed(ctx):
    """Inner, semi and anti pipelines in one batch (dimension built inside the
    kernel from a key range, or a prebuilt key set), each equal to its solo
    run and to the oracle."""
    cases = []
    for i, (kind, n) in enumerate([(qe.INNER, 70_001), (qe.SEMI, 123_457), (qe.ANTI, 5_000), (qe.SEMI, 1),
                                   (qe.ANTI, 200_000), (qe.SEMI, 0)]):
        fact, dk = _semi_case(80 + i, n, max(1, n // 4), max(2, n // 2))
        if kind == qe.INNER:
            dk = np.unique(dk)
        cases.append((kind, fact, dk))
    descs, groups, outs, keep, refs = [], [], [], [], []
    for i, (kind, fact, dk) in enumerate(cases):
        f = [fact[c].cuda() for c in COLS]
        span = (0, int(fact["fk"].max().item()) if len(fact["fk"]) else 0)
        span = (0, max(span[1], int(dk.max())))
        ht = qe.qe_join_build_set(ctx, cuda(dk)) if (kind != qe.INNER and i % 2) else None
        dkt = cuda(dk)
        dpt = cuda(np.arange(len(dk), dtype=np.int32) % 7) if kind == qe.INNER else None
        d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=dkt, dim_payload=dpt, ht=ht, key_hi_col=-1,
                             key_lo_col=4, aggs=AGGS, dim_key_range=span, join_kind=kind)
        g, o = qe.alloc_groups(64, 4, torch.device("cuda"))
        descs.append(d)
        outs.append(o)
        groups.append(g)
        keep.append((f, dkt, dpt, ht))
        refs.append(_oracle(fact, dk, kind))
    qe.qe_batch_run(ctx, descs, outs, opts=qe.qe_batch_opts(0, 1 << 15, 0, 0))
    for d, g, r in zip(descs, groups, refs):
        _assert_groups(g, r)
        solo = qe.qe_pipeline(ctx, d, 64)
        _assert_groups(solo, r)
    for k in keep:
        if k[3] is not None:
            k[3].destroy()


@pytest.mark.parametrize("smem_slots", [0, -1])
def test_batch_star_kinds(ctx, smem_slots):
    """Semi- and anti-join pipelines and pipelines with no join run the star
    row loop inside a batch as well, beside inner-join star pipelines: group
    keys of three shapes, the direct arrays in shared memory (smem_slots 0) or
    in HBM (-1), key sets built inside the kernel, pipelines of several
    32,768-row items with ragged tails.  Every result equals the oracle's and
    the pipeline's solo run."""
    descs, groups, outs, refs, keep = [], [], [], [], []

    def add(d, ref, cap):
        g, o = qe.alloc_groups(cap, 4, torch.device("cuda"))
        descs.append(d)
        groups.append(g)
        outs.append(o)
        refs.append((ref, cap))

    i = 0
    for shape in ("flag", "flag_qty", "fk_5000"):
        hi, lo, rng_, span = STAR_KEYS[shape]
        for kind in (qe.SEMI, qe.ANTI, "none"):
            seed = 300 + i
            n = 200_003 + 4_099 * i
            i += 1
            fact = datagen.star_fact(n, span, seed=seed)
            dk = np.random.default_rng(seed).integers(span // 10, span - span // 10, span // 2).astype(np.int32)
            f = [fact[c].cuda() for c in COLS]
            join = kind != "none"
            dkt = cuda(dk) if join else None
            keep.append((f, dkt))
            d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0 if join else -1, dim_key=dkt, key_hi_col=hi,
                                 key_lo_col=lo, aggs=AGGS, key_range=rng_,
                                 dim_key_range=(0, span - 1) if join else None,
                                 join_kind=kind if join else qe.INNER)
            q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0 if join else -1, key_hi_col=hi, key_lo_col=lo,
                        aggs=O_AGGS, join_kind=kind if join else O.INNER)
            add(d, O.pipeline([fact[c].numpy() for c in COLS], q, dk if join else None, None), 8192)
    for j in range(2):
        n, nd = 150_001 + 33 * j, 20_000
        dim = datagen.star_dim(nd, 25, seed=400 + j)
        fact = datagen.star_fact(n, nd, seed=400 + j)
        f = [fact[c].cuda() for c in COLS]
        dkt, dpt = cuda(dim["key"].numpy()), cuda(dim["attr"].numpy())
        keep.append((f, dkt, dpt))
        d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=dkt, dim_payload=dpt, key_hi_col=4,
                             key_lo_col=qe.JOIN_PAYLOAD, aggs=AGGS, key_range=((0, 2), (0, 24)),
                             dim_key_range=(0, nd - 1))
        q = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD, aggs=O_AGGS)
        add(d, O.pipeline([fact[c].numpy() for c in COLS], q, dim["key"].numpy(), dim["attr"].numpy()), 128)
    qe.qe_batch_run(ctx, descs, outs, opts=qe.qe_batch_opts(0, 1 << 15, smem_slots, 0))
    for d, g, (ref, cap) in zip(descs, groups, refs):
        _assert_groups(g, ref)
        _assert_groups(qe.qe_pipeline(ctx, d, cap), ref)
