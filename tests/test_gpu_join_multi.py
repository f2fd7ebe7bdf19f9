"""GPU parity of the many-to-many join and the pair-key join against the CPU oracle.

The outputs of one probe position come out in unspecified order, so each
position's (row, payload) pairs are compared as sorted lists; everything
else (positions in ascending order, the pairs themselves, the count) is
compared exactly.  Cases: both layouts, with and without a selection vector,
heavy and light repetition, a hot key with thousands of rows, unique keys
(the inner join), a probe large enough for many scan blocks, empty sides,
INT32_MIN, the output capacity, and the tables the other calls reject.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_09226_gb300 import qe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = qe.Context(0)
    yield c
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def canon(rows, pay):
    """(row, payload) pairs sorted by row, then payload: the order within a
    probe position is free, the order of positions is not."""
    o = np.lexsort((pay, rows))
    return rows[o], pay[o]


def check(ctx, ht, bk, bp, pk, sel=None):
    rows, pay, cnt = qe.qe_join_probe_multi(ctx, ht, cuda(pk), cuda(sel) if sel is not None else None,
                                            capacity=max(1, 4 * len(pk) + 1000))
    rr, rp = O.join_multi(bk, bp, pk, sel)
    c = int(cnt.item())
    assert c == len(rr)
    r, p = rows[:c].cpu().numpy(), pay[:c].cpu().numpy()
    # positions in ascending order: the row sequence itself matches
    assert np.array_equal(r, rr)
    a, b = canon(r, p), canon(rr, rp)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("layout", [qe.HT_DENSE, qe.HT_OPEN, qe.HT_AUTO])
@pytest.mark.parametrize("with_sel", [False, True])
def test_join_multi(ctx, layout, with_sel):
    rng = np.random.default_rng(layout * 2 + with_sel + 300)
    nb, npr = 60_000, 150_001
    bk = rng.integers(-20_000, 20_000, nb).astype(np.int32)          # about 1.5 rows per key
    bp = np.arange(nb, dtype=np.int32) * 7 - 11
    pk = rng.integers(-25_000, 25_000, npr).astype(np.int32)
    sel = np.sort(rng.choice(npr, 50_000, replace=False)).astype(np.int32) if with_sel else None
    ht = qe.qe_join_build_multi(ctx, cuda(bk), cuda(bp), layout=layout)
    info = ht.info()
    assert info.key_set == 2
    assert info.layout == (qe.HT_DENSE if layout == qe.HT_AUTO else layout)
    check(ctx, ht, bk, bp, pk, sel)
    ht.destroy()


@pytest.mark.parametrize("layout", [qe.HT_DENSE, qe.HT_OPEN])
def test_join_multi_hot_key_and_unique(ctx, layout):
    rng = np.random.default_rng(310 + layout)
    # one key with 5,000 rows, the rest light
    bk = np.concatenate([np.full(5_000, 77, np.int32), rng.integers(0, 3_000, 10_000).astype(np.int32)])
    bp = rng.integers(-2 ** 31, 2 ** 31 - 1, len(bk)).astype(np.int32)
    pk = rng.integers(0, 3_200, 9_000).astype(np.int32)
    pk[::100] = 77
    ht = qe.qe_join_build_multi(ctx, cuda(bk), cuda(bp), layout=layout)
    rows, pay, cnt = qe.qe_join_probe_multi(ctx, ht, cuda(pk), capacity=1_000_000)
    rr, rp = O.join_multi(bk, bp, pk)
    c = int(cnt.item())
    assert c == len(rr)
    a, b = canon(rows[:c].cpu().numpy(), pay[:c].cpu().numpy()), canon(rr, rp)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ht.destroy()
    # unique keys: the inner join, order included
    ub = rng.choice(np.arange(-50_000, 50_000), 20_000, replace=False).astype(np.int32)
    up = rng.integers(-1000, 1000, len(ub)).astype(np.int32)
    pk = rng.integers(-60_000, 60_000, 100_000).astype(np.int32)
    ht = qe.qe_join_build_multi(ctx, cuda(ub), cuda(up), layout=layout)
    rows, pay, cnt = qe.qe_join_probe_multi(ctx, ht, cuda(pk))
    rr, rp = O.join(ub, up, pk)
    c = int(cnt.item())
    assert c == len(rr)
    assert np.array_equal(rows[:c].cpu().numpy(), rr) and np.array_equal(pay[:c].cpu().numpy(), rp)
    ht.destroy()


def test_join_multi_large_probe(ctx):
    """Millions of positions: many segments and scan blocks."""
    rng = np.random.default_rng(320)
    bk = rng.integers(0, 1_000_000, 2_000_000).astype(np.int32)
    bp = rng.integers(0, 2 ** 31 - 1, len(bk)).astype(np.int32)
    pk = rng.integers(0, 1_200_000, 6_000_003).astype(np.int32)
    ht = qe.qe_join_build_multi(ctx, cuda(bk), cuda(bp))
    rows, pay, cnt = qe.qe_join_probe_multi(ctx, ht, cuda(pk), capacity=20_000_000)
    rr, rp = O.join_multi(bk, bp, pk)
    c = int(cnt.item())
    assert c == len(rr)
    r, p = rows[:c].cpu().numpy(), pay[:c].cpu().numpy()
    assert np.array_equal(r, rr)
    a, b = canon(r, p), canon(rr, rp)
    assert np.array_equal(a[1], b[1])
    ht.destroy()


def test_join_multi_edges_and_errors(ctx):
    e32 = torch.empty(0, dtype=torch.int32, device="cuda")
    ht = qe.qe_join_build_multi(ctx, e32, e32)
    rows, pay, cnt = qe.qe_join_probe_multi(ctx, ht, cuda(np.array([1, 2], np.int32)))
    assert int(cnt.item()) == 0
    rows, pay, cnt = qe.qe_join_probe_multi(ctx, ht, e32)
    assert int(cnt.item()) == 0
    ht.destroy()
    # INT32_MIN: an ordinary key of a dense multimap, reserved by the open one
    m = -2 ** 31
    bk = np.array([m, m + 5, m], np.int32)
    bp = np.array([1, 2, 3], np.int32)
    ht = qe.qe_join_build_multi(ctx, cuda(bk), cuda(bp), layout=qe.HT_DENSE)
    check(ctx, ht, bk, bp, np.array([m, m + 4, m + 5, m, 7], np.int32))
    # a multimap is for qe_join_probe_multi only
    for call in (lambda: qe.qe_join_probe(ctx, ht, cuda(bk)), lambda: qe.qe_join_semi(ctx, ht, cuda(bk))):
        with pytest.raises(qe.QeError) as e:
            call()
        assert e.value.status == qe.ERR_INVALID_ARG
    ht.destroy()
    with pytest.raises(qe.QeError) as e:
        qe.qe_join_build_multi(ctx, cuda(bk), cuda(bp), layout=qe.HT_OPEN)
    assert e.value.status == qe.ERR_RESERVED_KEY
    # a unique-key table is not a multimap
    ht = qe.qe_join_build(ctx, cuda(np.array([1, 2], np.int32)), cuda(np.array([3, 4], np.int32)))
    with pytest.raises(qe.QeError) as e:
        qe.qe_join_probe_multi(ctx, ht, cuda(np.array([1], np.int32)))
    assert e.value.status == qe.ERR_INVALID_ARG
    ht.destroy()
    # too small an output: nothing past the capacity, the full count reported
    bk = np.full(10, 3, np.int32)
    ht = qe.qe_join_build_multi(ctx, cuda(bk), cuda(np.arange(10, dtype=np.int32)))
    out_r = torch.full((8,), -5, dtype=torch.int32, device="cuda")
    out_p = torch.full((8,), -5, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(qe.QeError) as e:
        qe.qe_join_probe_multi(ctx, ht, cuda(np.array([3, 3], np.int32)), capacity=5, out_rows=out_r,
                               out_payload=out_p, out_count=cnt)
    assert e.value.status == qe.ERR_CAPACITY and e.value.required == 20
    assert out_r[5:].cpu().tolist() == [-5] * 3 and out_p[5:].cpu().tolist() == [-5] * 3
    assert out_r[:5].cpu().tolist() == [0] * 5
    ht.destroy()


# ---------------------------------------------------------------- pair keys
@pytest.mark.parametrize("n_probe", [1, 4097, 300_001, 5_000_003])
@pytest.mark.parametrize("with_sel", [False, True])
def test_join_pair(ctx, n_probe, with_sel):
    """Join on two key columns: unique build pairs whose halves repeat,
    one- and two-pass probes, with and without a selection vector."""
    rng = np.random.default_rng(n_probe % 997 + with_sel)
    pairs = rng.choice(2_000 * 1_000, 400_000, replace=False)
    bhi, blo = (pairs // 1_000 - 1_000).astype(np.int32), (pairs % 1_000 * 7 - 3_000).astype(np.int32)
    bp = rng.integers(-2 ** 31, 2 ** 31 - 1, len(pairs)).astype(np.int32)
    phi = rng.integers(-1_050, 1_050, n_probe).astype(np.int32)
    plo = (rng.integers(0, 1_000, n_probe) * 7 - 3_000).astype(np.int32)
    sel = np.sort(rng.choice(n_probe, n_probe // 2 + 1, replace=False)).astype(np.int32) if with_sel else None
    ht = qe.qe_join_build_pair(ctx, cuda(bhi), cuda(blo), cuda(bp))
    info = ht.info()
    assert info.key_set == 3 and info.bytes == info.slots * 16        # {key, payload} slots
    rows, pay, cnt = qe.qe_join_probe_pair(ctx, ht, cuda(phi), cuda(plo), cuda(sel) if with_sel else None)
    rr, rp = O.join_pair(bhi, blo, bp, phi, plo, sel)
    c = int(cnt.item())
    assert c == len(rr)
    assert np.array_equal(rows[:c].cpu().numpy(), rr) and np.array_equal(pay[:c].cpu().numpy(), rp)
    ht.destroy()


def test_join_pair_edges_and_errors(ctx):
    m = -2 ** 31
    # extreme halves are ordinary; only the packed (INT32_MIN, INT32_MIN) is reserved
    bhi, blo = np.array([m, m, 2 ** 31 - 1], np.int32), np.array([7, 2 ** 31 - 1, m], np.int32)
    bp = np.array([1, 2, 3], np.int32)
    ht = qe.qe_join_build_pair(ctx, cuda(bhi), cuda(blo), cuda(bp))
    phi, plo = np.array([m, 7, m, 2 ** 31 - 1, m], np.int32), np.array([7, m, 2 ** 31 - 1, m, m], np.int32)
    rows, pay, cnt = qe.qe_join_probe_pair(ctx, ht, cuda(phi), cuda(plo))
    rr, rp = O.join_pair(bhi, blo, bp, phi, plo)
    c = int(cnt.item())
    assert rows[:c].cpu().tolist() == rr.tolist() == [0, 2, 3] and pay[:c].cpu().tolist() == rp.tolist()
    for call in (lambda: qe.qe_join_probe(ctx, ht, cuda(phi)), lambda: qe.qe_join_semi(ctx, ht, cuda(phi)),
                 lambda: qe.qe_join_probe_multi(ctx, ht, cuda(phi))):
        with pytest.raises(qe.QeError) as e:
            call()
        assert e.value.status == qe.ERR_INVALID_ARG
    ht.destroy()
    for hi, lo, code in (([3, 3], [4, 4], qe.ERR_DUPLICATE_KEY), ([m, 1], [m, 1], qe.ERR_RESERVED_KEY)):
        with pytest.raises(qe.QeError) as e:
            qe.qe_join_build_pair(ctx, cuda(np.array(hi, np.int32)), cuda(np.array(lo, np.int32)),
                                  cuda(np.zeros(2, np.int32)))
        assert e.value.status == code
    e32 = torch.empty(0, dtype=torch.int32, device="cuda")
    ht = qe.qe_join_build_pair(ctx, e32, e32, e32)
    rows, pay, cnt = qe.qe_join_probe_pair(ctx, ht, cuda(phi), cuda(plo))
    assert int(cnt.item()) == 0
    ht.destroy()
