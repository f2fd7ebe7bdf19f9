"""GPU parity at the full sizes of the at-scale and skewed workloads.

The oracle cannot process these inputs whole in a test's time, so each test
checks (1) sampled outputs that the oracle computes one by one and (2)
properties that hold at any size, with checks done by plain torch reductions
on the device:

* star pipeline at scale (fact 600M rows, dimension 20M rows, 3,000 groups),
  in the launch configuration bench.py times: every group's four aggregates
  against a plain torch group-by of the same rows on the device, and three
  groups against the oracle run over the full input; the same for the
  25,002-group variant (attr in [0, 8334): the direct array in HBM);
* the batched form in the launch shape bench.py times (262,144-row work
  items, shared-memory group tables, a CUDA graph): several hundred small
  pipelines and two of 5M+ rows, every output against the oracle;
* partition of 600M (int64 key, int64 payload) pairs at fan-out 256 / 1024 /
  4096: offsets, payloads a permutation of the row ids, key/payload pairs
  intact, input order inside every destination, and the destination of
  sampled rows against the oracle's partition function;
* skewed, high-cardinality pipeline (fact 300M rows, Zipf(1.1) foreign keys
  over 50M dimension keys, group-by on ~40M distinct int64 keys in HBM,
  selectivity 1 % / 50 % / 90 %; group-by on 10^6 dictionary codes):
  every group of 1000 sampled keys against the oracle run over exactly the
  rows of those keys; the number of groups; sums of COUNT and SUM;
* the join variants on the 600M-row fact table, in the launch configuration
  bench.py times: the semi- / anti-join pipelines and the single-table
  aggregation group by group against torch reductions over the rows they
  keep (so semi + anti = single-table as well); the stand-alone semi- and
  anti-join, the many-to-many join (4 build rows per key, 1.2 billion output
  pairs) and the pair-key join against their full expected outputs built
  with torch indexing, and sampled probe positions against the oracle run
  over the build rows of their keys.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_09226_gb300 import datagen
from paper_2506_09226_gb300 import qe

pytestmark = pytest.mark.gpu

COLS = ("fk", "date", "price", "qty", "flag")
STAR_AGGS = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
O_AGGS = [(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)]
DATE_LT = 1278


@pytest.fixture(scope="module")
def ctx():
    c = qe.Context(0)
    yield c
    c.close()


class _Groups:
    """Groups sorted by key, with lookup of single keys."""

    def __init__(self, g):
        k, a = g.to_host()
        o = np.argsort(k.numpy(), kind="stable")
        self.keys = k.numpy()[o]
        self.aggs = [x.numpy()[o] for x in a]

    def __len__(self):
        return len(self.keys)

    def __getitem__(self, key):
        i = int(np.searchsorted(self.keys, key))
        assert i < len(self.keys) and self.keys[i] == key, key
        return tuple(int(a[i]) for a in self.aggs)

    def total(self, j):
        return int(self.aggs[j].sum(dtype=np.int64))


def _filtered_totals(fact, mask):
    """(rows, sum price*qty, min price, max price) over the rows in mask."""
    price = fact["price"][mask]
    qty = fact["qty"][mask].to(torch.int64)
    return (int(mask.sum().item()), int((price * qty).sum().item()), int(price.min().item()),
            int(price.max().item()))


# ---------------------------------------------------------------- star pipeline at scale
@pytest.fixture(scope="module")
def star600():
    dev = torch.device("cuda", 0)
    dim = datagen.star_dim(20_000_000, 1000, seed=1, device=dev)
    fact = datagen.star_fact(600_000_000, 20_000_000, seed=1, device=dev)
    half = dim["key"][: 10_000_000].contiguous()
    member = torch.zeros(20_000_000, dtype=torch.bool, device=dev)
    member[half.long()] = True
    yield fact, dim, half, member
    del fact, dim, half, member
    torch.cuda.empty_cache()


def _torch_star_groups(fact, dim, n_attr, date_lt=DATE_LT, chunk=100_000_000):
    """Every group of group-by(flag, attr)(join(filter(fact), dim)) with
    SUM(price*qty), COUNT, MIN(price), MAX(price), by plain torch reductions
    on the device (index_add_, bincount, scatter_reduce), in ascending key
    order.  The dimension's keys are a permutation of 0..n-1 (checked), so
    attr of a foreign key is one gather."""
    dev = fact["fk"].device
    nd = dim["key"].numel()
    assert torch.equal(torch.sort(dim["key"]).values, torch.arange(nd, dtype=torch.int32, device=dev))
    attr_of = torch.empty(nd, dtype=torch.int64, device=dev)
    attr_of[dim["key"].long()] = dim["attr"].long()
    G = 3 * n_attr
    s = torch.zeros(G, dtype=torch.int64, device=dev)
    c = torch.zeros(G, dtype=torch.int64, device=dev)
    mn = torch.full((G,), 2 ** 63 - 1, dtype=torch.int64, device=dev)
    mx = torch.full((G,), -2 ** 63, dtype=torch.int64, device=dev)
    n = fact["fk"].numel()
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        m = fact["date"][a:b] < date_lt
        gid = fact["flag"][a:b][m].long() * n_attr + attr_of[fact["fk"][a:b][m].long()]
        price = fact["price"][a:b][m]
        s.index_add_(0, gid, price * fact["qty"][a:b][m].long())
        c += torch.bincount(gid, minlength=G)
        mn.scatter_reduce_(0, gid, price, "amin")
        mx.scatter_reduce_(0, gid, price, "amax")
        del m, gid, price
    live = torch.nonzero(c).flatten()
    keys = ((live // n_attr) << 32) | (live % n_attr)
    return keys.cpu().numpy(), [x[live].cpu().numpy() for x in (s, c, mn, mx)]


def _run_star600(ctx, fact, dim, expected):
    d = qe.pipeline_desc([fact[c] for c in COLS], [(1, qe.LT, DATE_LT)], fk_col=0, dim_key=dim["key"],
                         dim_payload=dim["attr"], key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS,
                         expected_groups=expected, est_selectivity=DATE_LT / 2557, key_range=((0, 2), None))
    return _Groups(qe.qe_pipeline(ctx, d, 4096 if expected <= 4096 else 32768))


def _assert_all_groups(got, keys, aggs):
    assert len(got) == len(keys)
    assert np.array_equal(got.keys, keys)
    for a, (x, y) in enumerate(zip(got.aggs, aggs)):
        assert np.array_equal(x, y), a


def test_star_pipeline_600M(ctx, star600):
    """The step's pipeline (bench.py's launch configuration): all 3,000
    groups exactly, and three against the oracle over the full input."""
    fact, dim, _, _ = star600
    got = _run_star600(ctx, fact, dim, 3000)
    keys, aggs = _torch_star_groups(fact, dim, 1000)
    assert len(keys) == 3000
    _assert_all_groups(got, keys, aggs)
    # sampled groups against the oracle over the full input
    host = [fact[c].cpu().numpy() for c in COLS]
    dk, da = dim["key"].cpu().numpy(), dim["attr"].cpu().numpy()
    q = O.Query(preds=[O.Pred(1, O.LT, DATE_LT)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD, aggs=O_AGGS)
    rng = np.random.default_rng(11)
    for gk in [int(keys[0]), int(keys[-1]), int(keys[rng.integers(1, len(keys) - 1)])]:
        cnt, ref = O.pipeline_group(host, q, gk, dk, da)
        assert cnt == got[gk][1]
        assert tuple(int(x) for x in ref) == got[gk], gk


def test_star_pipeline_600M_25k_groups(ctx, star600):
    """bench.py's 25K-group variant: the same fact table against a 20M-row
    dimension whose attr is in [0, 8334), 25,002 groups in an HBM direct
    array; every group exactly."""
    fact, _, _, _ = star600
    dim25 = datagen.star_dim(20_000_000, 8334, seed=1, device=fact["fk"].device)
    got = _run_star600(ctx, fact, dim25, 25002)
    keys, aggs = _torch_star_groups(fact, dim25, 8334)
    assert len(keys) == 25002
    _assert_all_groups(got, keys, aggs)
    del dim25


# ---------------------------------------------------------------- batched form in the bench's shape
def test_batch_bench_launch_shape(ctx):
    """The batched form as bench.py launches it: 262,144-row work items,
    shared-memory group tables, one CUDA graph; 400 pipelines of 1K-100K
    fact rows (log-uniform) with a 5M- and a 7M-row pipeline among them,
    dimension rows = fact rows / 10; every output against the oracle."""
    from paper_2506_09226_gb300 import batch as B
    sizes = datagen.log_uniform_sizes(400, 1e3, 1e5, seed=44)
    sizes[37], sizes[251] = 5_000_000, 7_000_003
    w = datagen.batch_star(sizes, B.N_ATTR, seed=44)
    wd = {"fact": {c: t.cuda() for c, t in w["fact"].items()}, "dim": {c: t.cuda() for c, t in w["dim"].items()},
          **{k: w[k] for k in ("fact_off", "dim_off", "sizes", "dim_sizes")}}
    outs = B.BatchOutputs(len(sizes), B.CAPACITY, torch.device("cuda"))
    descs = B.star_descs(wd)
    b = qe.Batch(ctx, descs, outs.structs, qe.qe_batch_opts(0, 1 << 18, 0, 1))
    b.launch()
    ctx.sync_status()
    b.destroy()
    q = O.Query(preds=[O.Pred(1, O.LT, B.DATE_LT)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD, aggs=O_AGGS)
    f, d = w["fact"], w["dim"]
    for i, n in enumerate(sizes):
        a, nd, bo = int(w["fact_off"][i]), int(w["dim_sizes"][i]), int(w["dim_off"][i])
        ref = O.pipeline([f[c][a:a + int(n)].numpy() for c in COLS], q, d["key"][bo:bo + nd].numpy(),
                         d["attr"][bo:bo + nd].numpy())
        k, aggs = outs.groups(i)
        assert np.array_equal(k, ref["keys"]), i
        for x, y in zip(aggs, ref["aggs"]):
            assert np.array_equal(x, y), i


# ---------------------------------------------------------------- partition at scale
@pytest.fixture(scope="module")
def pairs():
    dev = torch.device("cuda", 0)
    key, pay = datagen.key_payload_pairs(600_000_000, seed=2, device=dev)
    yield key, pay
    del key, pay
    torch.cuda.empty_cache()


@pytest.mark.parametrize("log2f", [8, 10, 12])
def test_partition_600M(ctx, pairs, log2f):
    key, pay = pairs
    n, F = key.numel(), 1 << log2f
    ok, op = torch.empty_like(key), torch.empty_like(pay)
    offs = torch.empty(F + 1, dtype=torch.int64, device=key.device)
    qe.qe_partition(ctx, key, [pay], log2f, qe.PART_HASH, 0, ok, [op], offs)

    o = offs.cpu().numpy()
    assert o[0] == 0 and o[-1] == n and np.all(np.diff(o) >= 0)
    # payloads are the row ids: a permutation, with each key still beside its payload
    assert int(op.min().item()) == 0 and int(op.max().item()) == n - 1
    seen = torch.zeros(n, dtype=torch.bool, device=key.device)
    seen[op] = True
    assert bool(seen.all().item())
    del seen
    assert bool(torch.equal(ok, key[op]))
    # input order inside every destination: row ids increase except where a destination starts
    step_up = op[1:] > op[:-1]
    starts = torch.from_numpy(o[1:-1]).to(key.device)
    starts = starts[(starts > 0) & (starts < n)] - 1
    step_up[starts] = True
    assert bool(step_up.all().item())
    del step_up
    # destination of sampled output rows against the oracle's partition function
    rng = np.random.default_rng(log2f)
    pos = np.sort(rng.choice(n, 20_000, replace=False))
    ks = ok[torch.from_numpy(pos).to(key.device)].cpu().numpy()
    seg = np.searchsorted(o, pos, side="right") - 1
    for p, k in zip(seg, ks):
        assert O.partition_of(int(k), log2f) == p
    # each destination's size against the oracle's function on a sample of input rows
    samp = key[torch.from_numpy(rng.choice(n, 200_000, replace=False)).to(key.device)].cpu().numpy()
    hist = np.bincount([O.partition_of(int(k), log2f) for k in samp], minlength=F) * (n / len(samp))
    sizes = np.diff(o)
    sigma = np.sqrt(hist.clip(min=1) * (n / len(samp)))
    assert np.all(np.abs(sizes - hist) < 6 * sigma + 5)


# ---------------------------------------------------------------- skew and high cardinality
@pytest.fixture(scope="module")
def skew():
    dev = torch.device("cuda", 0)
    dim = datagen.star_dim(50_000_000, 1000, seed=3, device=dev)
    fact = datagen.star_fact(300_000_000, 50_000_000, seed=3, device=dev, zipf_s=1.1, n_codes=1_000_000,
                             n_gkeys=40_000_000)
    yield fact, dim
    del fact, dim
    torch.cuda.empty_cache()


SKEW_COLS = ("fk", "date", "price", "qty", "flag", "code", "gkey")


def _check_sampled_groups(fact, dim, got, key_col, preds_qe, preds_o, rng, nsample=1000):
    """Every group of nsample sampled keys against the oracle, run over the
    rows holding those keys (and the dimension rows they reference)."""
    pick = torch.from_numpy(rng.choice(got.keys, min(nsample, len(got)), replace=False)).to(fact["fk"].device)
    col = fact[key_col]
    rows = torch.isin(col.to(torch.int64), pick)
    sub = [fact[c][rows].cpu().numpy() for c in SKEW_COLS]
    fks = fact["fk"][rows]
    drows = torch.isin(dim["key"], fks)
    dk, da = dim["key"][drows].cpu().numpy(), dim["attr"][drows].cpu().numpy()
    q = O.Query(preds=preds_o, fk_col=0, key_hi_col=-1, key_lo_col=SKEW_COLS.index(key_col), aggs=O_AGGS)
    ref = O.pipeline(sub, q, dk, da)
    picked = set(int(x) for x in pick.cpu().numpy())
    seen = 0
    for i, k in enumerate(ref["keys"]):
        k = int(k)
        if k in picked:
            assert got[k] == tuple(int(a[i]) for a in ref["aggs"]), k
            seen += 1
    assert seen == len(picked)


def _torch_groups_by(col, fact, mask):
    """Every group of (col, SUM(price*qty), COUNT, MIN(price), MAX(price))
    over the rows in mask, by torch.unique and plain reductions on the
    device, in ascending key order."""
    keys, inv = torch.unique(col[mask].to(torch.int64), return_inverse=True)
    G = keys.numel()
    price = fact["price"][mask]
    s = torch.zeros(G, dtype=torch.int64, device=col.device).index_add_(0, inv, price * fact["qty"][mask].long())
    c = torch.bincount(inv, minlength=G)
    mn = torch.full((G,), 2 ** 63 - 1, dtype=torch.int64, device=col.device).scatter_reduce_(0, inv, price, "amin")
    mx = torch.full((G,), -2 ** 63, dtype=torch.int64, device=col.device).scatter_reduce_(0, inv, price, "amax")
    return keys, [s, c, mn, mx]


def _assert_device_groups(g, keys, aggs):
    """The library's groups (unspecified order) equal the expected ones, all
    compared on the device."""
    n = int(g.ngroups.item())
    assert n == keys.numel()
    order = torch.argsort(g.keys[:n])
    assert torch.equal(g.keys[:n][order], keys)
    for a, e in zip(g.aggs, aggs):
        assert torch.equal(a[:n][order], e)


@pytest.mark.parametrize("sel", [0.01, 0.50, 0.90])
def test_skew_pipeline_40M_groups(ctx, skew, sel):
    """The launch bench.py times (the partitioned group-by: ~40M groups far
    beyond L2): every group against torch reductions on the device, and
    every group of 1000 sampled keys against the oracle."""
    fact, dim = skew
    c = int(round(sel * datagen.DATE_SPAN))
    f = [fact[x] for x in SKEW_COLS]
    d = qe.pipeline_desc(f, [(1, qe.LT, c)], fk_col=0, dim_key=dim["key"], dim_payload=dim["attr"],
                         key_hi_col=-1, key_lo_col=SKEW_COLS.index("gkey"), aggs=STAR_AGGS,
                         expected_groups=40_000_000, est_selectivity=sel)
    g = qe.qe_pipeline(ctx, d, 40_000_000)
    mask = fact["date"] < c
    keys, aggs = _torch_groups_by(fact["gkey"], fact, mask)
    del mask
    _assert_device_groups(g, keys, aggs)
    del keys, aggs
    got = _Groups(g)
    _check_sampled_groups(fact, dim, got, "gkey", None, [O.Pred(1, O.LT, c)], np.random.default_rng(c))


def test_skew_pipeline_dictionary_codes(ctx, skew):
    """Group by the int32 dictionary codes (10^6 values) under a code-range predicate."""
    fact, dim = skew
    k = 250_000
    f = [fact[x] for x in SKEW_COLS]
    d = qe.pipeline_desc(f, [(5, qe.LT, k)], fk_col=0, dim_key=dim["key"], dim_payload=dim["attr"],
                         key_hi_col=-1, key_lo_col=SKEW_COLS.index("code"), aggs=STAR_AGGS,
                         expected_groups=k)
    g = qe.qe_pipeline(ctx, d, 1_000_000)
    mask = fact["code"] < k
    nkeys = int(torch.unique(fact["code"][mask]).numel())
    rows, s, _, _ = _filtered_totals(fact, mask)
    del mask
    assert int(g.ngroups.item()) == nkeys
    got = _Groups(g)
    assert got.total(1) == rows
    assert got.total(0) == s
    _check_sampled_groups(fact, dim, got, "code", None, [O.Pred(5, O.LT, k)], np.random.default_rng(5))


# ---------------------------------------------------------------- join variants at scale
def test_semi_anti_single_table_600M(ctx, star600):
    """Filter + semi- / anti-join against half the dimension's keys + group-by
    flag, and the same filter + group-by with no join: every group's four
    aggregates against torch reductions over exactly the rows kept."""
    fact, dim, half, member = star600
    cols = [fact[c] for c in COLS]
    got = {}
    for name, kind in (("semi", qe.SEMI), ("anti", qe.ANTI)):
        d = qe.pipeline_desc(cols, [(1, qe.LT, DATE_LT)], fk_col=0, dim_key=half, key_hi_col=-1, key_lo_col=4,
                             aggs=STAR_AGGS, expected_groups=3, est_selectivity=DATE_LT / 2557,
                             key_range=(None, (0, 2)), join_kind=kind)
        got[name] = _Groups(qe.qe_pipeline(ctx, d, 64))
    d = qe.pipeline_desc(cols[1:], [(0, qe.LT, DATE_LT)], key_hi_col=-1, key_lo_col=3,
                         aggs=[(qe.SUM, 1, 2), (qe.COUNT, -1, -1), (qe.MIN, 1, -1), (qe.MAX, 1, -1)],
                         expected_groups=3, est_selectivity=DATE_LT / 2557, key_range=(None, (0, 2)))
    got["single"] = _Groups(qe.qe_pipeline(ctx, d, 64))
    keep = fact["date"] < DATE_LT
    inset = member[fact["fk"].long()]
    masks = {"single": keep, "semi": keep & inset, "anti": keep & ~inset}
    for name, m in masks.items():
        assert got[name].keys.tolist() == [0, 1, 2], name
        for f in range(3):
            ref = _filtered_totals(fact, m & (fact["flag"] == f))
            g = got[name][f]
            assert (g[1], g[0], g[2], g[3]) == ref, (name, f)
    for f in range(3):
        a, b, c = got["semi"][f], got["anti"][f], got["single"][f]
        assert a[0] + b[0] == c[0] and a[1] + b[1] == c[1]
        assert min(a[2], b[2]) == c[2] and max(a[3], b[3]) == c[3]


def test_semi_multi_pair_joins_600M(ctx, star600):
    """The stand-alone joins over the filter's 300M-position selection vector,
    each against its complete expected output, and sampled positions of the
    many-to-many and pair-key joins against the oracle."""
    fact, dim, half, member = star600
    dev = fact["fk"].device
    n, nd = fact["fk"].numel(), 20_000_000
    sel = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    qe.qe_filter(ctx, [fact["date"]], [(0, qe.LT, DATE_LT)], sel, cnt)
    nsel = int(cnt.item())
    sel = sel[:nsel]
    assert torch.equal(sel, torch.nonzero(fact["date"] < DATE_LT).flatten().to(torch.int32))
    fks = fact["fk"][sel.long()]
    rng = np.random.default_rng(29)
    sample = np.sort(rng.choice(nsel, 1000, replace=False))

    # semi- and anti-join: the selected positions whose key is (not) in the set, in order
    hs = qe.qe_join_build_set(ctx, half)
    inset = member[fks.long()]
    for anti, want in ((False, sel[inset]), (True, sel[~inset])):
        rows, c = qe.qe_join_semi(ctx, hs, fact["fk"], sel, n=nsel, anti=anti, capacity=nsel)
        assert int(c.item()) == want.numel()
        assert torch.equal(rows[: want.numel()], want)
    hs.destroy()
    del inset

    # many-to-many: every position meets the 4 build rows of its key
    md = datagen.multi_dim(nd, 4, 1000, seed=4, device=dev)
    hm = qe.qe_join_build_multi(ctx, md["key"], md["attr"])
    rows, pay, c = qe.qe_join_probe_multi(ctx, hm, fact["fk"], sel, n=nsel, capacity=4 * nsel + 1)
    assert int(c.item()) == 4 * nsel
    assert torch.equal(rows[: 4 * nsel], sel.repeat_interleave(4))
    o1 = torch.argsort(md["attr"], stable=True)
    o2 = torch.argsort(md["key"][o1], stable=True)
    by_key = md["attr"][o1][o2].view(nd, 4)
    del o1, o2
    got = pay[: 4 * nsel].view(nsel, 4).sort(dim=1).values
    assert torch.equal(got, by_key[fks.long()])
    del got, by_key
    # sampled positions against the oracle, over the build rows of their keys
    ts = torch.from_numpy(sample).to(dev)
    pk = fks[ts]
    brows = torch.isin(md["key"], pk)
    rr, rp = O.join_multi(md["key"][brows].cpu().numpy(), md["attr"][brows].cpu().numpy(), pk.cpu().numpy())
    assert np.array_equal(rr, np.repeat(np.arange(len(sample), dtype=np.int32), 4))
    idx = torch.from_numpy(np.repeat(sample * 4, 4) + np.tile(np.arange(4), len(sample))).to(dev)
    assert np.array_equal(rows[idx].cpu().numpy(), np.repeat(sel[ts].cpu().numpy(), 4))
    gp = pay[idx].cpu().numpy()
    assert np.array_equal(np.sort(gp.reshape(-1, 4), axis=1), np.sort(rp.reshape(-1, 4), axis=1))
    hm.destroy()
    del md, rows, pay

    # pair keys: a position matches iff its second key is one of its first key's 4 partners
    pd = datagen.pair_dim(nd, 4, seed=5, device=dev)
    plo = datagen.pair_probe_lo(fact["fk"], pd["off"], 5, seed=5)
    hp = qe.qe_join_build_pair(ctx, pd["hi"], pd["lo"], pd["payload"])
    rows, pay, c = qe.qe_join_probe_pair(ctx, hp, fact["fk"], plo, sel, n=nsel, capacity=nsel)
    j = plo[sel.long()] - pd["off"][fks.long()]
    hit = j < 4
    by_pair = torch.empty(4 * nd, dtype=torch.int32, device=dev)
    by_pair[pd["hi"].long() * 4 + (pd["lo"] - pd["off"][pd["hi"].long()]).long()] = pd["payload"]
    k = int(hit.sum().item())
    assert int(c.item()) == k
    assert torch.equal(rows[:k], sel[hit])
    assert torch.equal(pay[:k], by_pair[fks[hit].long() * 4 + j[hit].long()])
    del by_pair, j, hit
    # sampled positions against the oracle, over the build rows of their first keys
    pos = sel[torch.from_numpy(sample).to(dev)]
    ph, pl = fact["fk"][pos.long()], plo[pos.long()]
    brows = torch.isin(pd["hi"], ph)
    rr, rp = O.join_pair(pd["hi"][brows].cpu().numpy(), pd["lo"][brows].cpu().numpy(),
                         pd["payload"][brows].cpu().numpy(), ph.cpu().numpy(), pl.cpu().numpy())
    assert 700 < len(rr) < 900
    at = torch.searchsorted(rows[:k], pos)
    found = (at < k) & (rows[:k][at.clamp(max=k - 1)] == pos)
    f = found.cpu().numpy()
    assert np.array_equal(np.nonzero(f)[0].astype(np.int32), rr)
    assert np.array_equal(pay[:k][at[found]].cpu().numpy(), rp)
    hp.destroy()
