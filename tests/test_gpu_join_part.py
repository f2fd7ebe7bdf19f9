"""GPU parity of the region-ordered join builds against the CPU oracle.

A build into a table far larger than L2 first reorders its rows region by
region (the top bits of the slot each row hashes to; for a dense multimap,
of key - key_min), then runs the ordinary insert kernels over the reordered
rows (Sec. 7.2 on hash tables too large to build efficiently; Sec. 2.2 on
one partitioning function applied before the local join).  The knob
"join_partition" = 2 forces that path at test sizes and "join_part_log2"
sets the regions (2 .. 256 are covered).  Every table is probed and the
result compared with the oracle's join exactly; the region step is checked
to have run (its profiling scope), and the build errors (repeated keys, the
reserved key, keys outside a given range) must still be reported.  Tile
edges of the reordering (4,096 rows) and empty inputs are covered.
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
    c.set_tuning("join_partition", 2)
    yield c
    c.set_tuning("join_partition", 0)
    c.set_tuning("join_part_log2", 0)
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def regions_run(ctx, build):
    """Builds with profiling on; returns (table, launches of the region step)."""
    ctx.profile(True)
    ctx.profile_reset()
    try:
        ht = build()
        n, _ = ctx.profile_read("build_partition")
    finally:
        ctx.profile(False)
    return ht, n


def unique_keys(rng, n, lo=-2 ** 31 + 1, hi=2 ** 31 - 1):
    k = np.unique(rng.integers(lo, hi, int(n * 1.1) + 16).astype(np.int32))
    rng.shuffle(k)
    return k[:n]


@pytest.mark.parametrize("log2p", [1, 3, 8])
@pytest.mark.parametrize("nb", [300_001, 4_097])
def test_region_open_build(ctx, log2p, nb):
    """Open-addressing table over sparse int32 keys, probed with half hits."""
    ctx.set_tuning("join_part_log2", log2p)
    try:
        rng = np.random.default_rng(nb + log2p)
        bk = unique_keys(rng, nb)
        bp = rng.integers(-2 ** 31, 2 ** 31 - 1, nb).astype(np.int32)
        pk = np.where(rng.random(700_003) < 0.5, rng.choice(bk, 700_003),
                      rng.integers(-2 ** 31 + 1, 2 ** 31 - 1, 700_003)).astype(np.int32)
        ht, n = regions_run(ctx, lambda: qe.qe_join_build(ctx, cuda(bk), cuda(bp), layout=qe.HT_OPEN))
        assert n == 1 and ht.info().layout == qe.HT_OPEN
        rows, pay, cnt = qe.qe_join_probe(ctx, ht, cuda(pk))
        rr, rp = O.join(bk, bp, pk)
        c = int(cnt.item())
        assert c == len(rr)
        assert np.array_equal(rows[:c].cpu().numpy(), rr) and np.array_equal(pay[:c].cpu().numpy(), rp)
        ht.destroy()
    finally:
        ctx.set_tuning("join_part_log2", 0)


@pytest.mark.parametrize("n", [1, 4_095, 4_096, 8_193])
def test_region_key_set_ragged(ctx, n):
    """A key set (repeated keys allowed) at the reordering's tile edges, as
    semi- and anti-join."""
    ctx.set_tuning("join_part_log2", 4)
    try:
        rng = np.random.default_rng(n)
        bk = rng.integers(-50_000, 50_000, n).astype(np.int32) * 7919
        bk[::3] = bk[0]
        pk = rng.integers(-60_000, 60_000, 50_001).astype(np.int32) * 7919
        ht, cnt_regions = regions_run(ctx, lambda: qe.qe_join_build_set(ctx, cuda(bk), layout=qe.HT_OPEN))
        assert cnt_regions == 1
        for anti in (False, True):
            rows, cnt = qe.qe_join_semi(ctx, ht, cuda(pk), anti=anti)
            ref = O.semi_join(bk, pk, anti=anti)
            c = int(cnt.item())
            assert c == len(ref) and np.array_equal(rows[:c].cpu().numpy(), ref)
        ht.destroy()
    finally:
        ctx.set_tuning("join_part_log2", 0)


@pytest.mark.parametrize("log2p", [2, 6])
def test_region_pair_build(ctx, log2p):
    ctx.set_tuning("join_part_log2", log2p)
    try:
        rng = np.random.default_rng(40 + log2p)
        pairs = rng.choice(3_000 * 1_000, 500_000, replace=False)
        bhi, blo = (pairs // 1_000 - 1_500).astype(np.int32), (pairs % 1_000 * 13 - 6_000).astype(np.int32)
        bp = rng.integers(-2 ** 31, 2 ** 31 - 1, len(pairs)).astype(np.int32)
        npr = 1_000_003
        phi = rng.integers(-1_550, 1_550, npr).astype(np.int32)
        plo = (rng.integers(0, 1_000, npr) * 13 - 6_000).astype(np.int32)
        sel = np.sort(rng.choice(npr, npr // 3, replace=False)).astype(np.int32)
        ht, n = regions_run(ctx, lambda: qe.qe_join_build_pair(ctx, cuda(bhi), cuda(blo), cuda(bp)))
        assert n == 1
        rows, pay, cnt = qe.qe_join_probe_pair(ctx, ht, cuda(phi), cuda(plo), cuda(sel))
        rr, rp = O.join_pair(bhi, blo, bp, phi, plo, sel)
        c = int(cnt.item())
        assert c == len(rr)
        assert np.array_equal(rows[:c].cpu().numpy(), rr) and np.array_equal(pay[:c].cpu().numpy(), rp)
        ht.destroy()
    finally:
        ctx.set_tuning("join_part_log2", 0)


@pytest.mark.parametrize("layout", [qe.HT_DENSE, qe.HT_OPEN])
@pytest.mark.parametrize("log2p", [3, 8])
def test_region_multi_build(ctx, layout, log2p):
    """Many-to-many build (about 3 rows per key, one hot key): each probe
    position's matches compared as a sorted list, positions in order."""
    ctx.set_tuning("join_part_log2", log2p)
    try:
        rng = np.random.default_rng(50 + layout * 10 + log2p)
        nb = 400_000
        bk = rng.integers(-70_000, 70_000, nb).astype(np.int32)
        bk[:2_000] = 1234
        rng.shuffle(bk)
        bp = rng.integers(-2 ** 31, 2 ** 31 - 1, nb).astype(np.int32)
        pk = rng.integers(-80_000, 80_000, 200_001).astype(np.int32)
        pk[::500] = 1234
        ht, n = regions_run(ctx, lambda: qe.qe_join_build_multi(ctx, cuda(bk), cuda(bp), layout=layout))
        assert n == 1 and ht.info().layout == layout
        rows, pay, cnt = qe.qe_join_probe_multi(ctx, ht, cuda(pk), capacity=4_000_000)
        rr, rp = O.join_multi(bk, bp, pk)
        c = int(cnt.item())
        assert c == len(rr)
        r, p = rows[:c].cpu().numpy(), pay[:c].cpu().numpy()
        assert np.array_equal(r, rr)
        o1, o2 = np.lexsort((p, r)), np.lexsort((rp, rr))
        assert np.array_equal(p[o1], rp[o2])
        ht.destroy()
    finally:
        ctx.set_tuning("join_part_log2", 0)


def test_region_build_errors_and_empty(ctx):
    """Repeated keys, the reserved key and (dense multimap) keys outside the
    given range are still reported after the reordering; empty builds work."""
    ctx.set_tuning("join_part_log2", 5)
    try:
        rng = np.random.default_rng(77)
        bk = unique_keys(rng, 100_000)
        bp = np.zeros(100_000, np.int32)
        dup = bk.copy()
        dup[99_999] = dup[17]
        with pytest.raises(qe.QeError) as e:
            qe.qe_join_build(ctx, cuda(dup), cuda(bp), layout=qe.HT_OPEN)
        assert e.value.status == qe.ERR_DUPLICATE_KEY
        res = bk.copy()
        res[5_000] = -2 ** 31
        with pytest.raises(qe.QeError) as e:
            qe.qe_join_build(ctx, cuda(res), cuda(bp), layout=qe.HT_OPEN)
        assert e.value.status == qe.ERR_RESERVED_KEY
        pairs_hi, pairs_lo = np.arange(10_000, dtype=np.int32), np.arange(10_000, dtype=np.int32)
        pairs_hi[9_000], pairs_lo[9_000] = 3, 3
        with pytest.raises(qe.QeError) as e:
            qe.qe_join_build_pair(ctx, cuda(pairs_hi), cuda(pairs_lo), cuda(np.zeros(10_000, np.int32)))
        assert e.value.status == qe.ERR_DUPLICATE_KEY
        mk = rng.integers(0, 1_000, 50_000).astype(np.int32)
        mk[49_999] = 5_000
        with pytest.raises(qe.QeError) as e:
            qe.qe_join_build_multi(ctx, cuda(mk), cuda(np.zeros(50_000, np.int32)), layout=qe.HT_DENSE,
                                   key_range=(0, 999))
        assert e.value.status == qe.ERR_INVALID_ARG
        e32 = torch.empty(0, dtype=torch.int32, device="cuda")
        for build in (lambda: qe.qe_join_build(ctx, e32, e32, layout=qe.HT_OPEN),
                      lambda: qe.qe_join_build_pair(ctx, e32, e32, e32),
                      lambda: qe.qe_join_build_multi(ctx, e32, e32, layout=qe.HT_OPEN)):
            ht = build()
            assert ht.info().nkeys == 0
            ht.destroy()
    finally:
        ctx.set_tuning("join_part_log2", 0)


def test_region_auto_rule(ctx):
    """Automatic choice: a table below 256 MB is built in input order; the
    knob's "never" keeps even a forced size in input order."""
    rng = np.random.default_rng(88)
    bk = unique_keys(rng, 200_000)
    bp = np.zeros(len(bk), np.int32)
    for knob, want in ((0, 0), (1, 0), (2, 1)):
        ctx.set_tuning("join_partition", knob)
        ht, n = regions_run(ctx, lambda: qe.qe_join_build(ctx, cuda(bk), cuda(bp), layout=qe.HT_OPEN))
        assert n == want
        ht.destroy()
    ctx.set_tuning("join_partition", 2)


def _fmix32(x):
    """MurmurHash3's 32-bit finalizer (A. Appleby, public domain), the slot
    hash of the open-addressing table, for building colliding test keys."""
    x = x.astype(np.uint32)
    x ^= x >> np.uint32(16)
    x *= np.uint32(0x85EBCA6B)
    x ^= x >> np.uint32(13)
    x *= np.uint32(0xC2B2AE35)
    x ^= x >> np.uint32(16)
    return x


def test_region_probe_overflow(ctx):
    """Keys whose probe runs past their region and the next one: 2,048 keys
    in 4,096 slots cut into 256 regions of 16 slots, 60 of them with the same
    home slot near a region's end.  Those rows finish in the overflow step;
    every key is found with its payload, and a repeat of an overflowed key is
    still reported."""
    ctx.set_tuning("join_part_log2", 8)
    try:
        rng = np.random.default_rng(91)
        cand = rng.integers(-2 ** 31 + 1, 2 ** 31 - 1, 4_000_000).astype(np.int32)
        home = _fmix32(cand.view(np.uint32)) & np.uint32(4095)
        hot = np.unique(cand[home == 4_094])[:60]
        assert len(hot) == 60
        rest = np.setdiff1d(np.unique(cand[(home % 16 < 8)]), hot)[:1_988]
        bk = np.concatenate([hot, rest]).astype(np.int32)
        rng.shuffle(bk)
        assert len(np.unique(bk)) == 2_048
        bp = rng.integers(-2 ** 31, 2 ** 31 - 1, len(bk)).astype(np.int32)
        ht, n = regions_run(ctx, lambda: qe.qe_join_build(ctx, cuda(bk), cuda(bp), layout=qe.HT_OPEN))
        assert n == 1 and ht.info().slots == 4_096
        pk = np.concatenate([bk, rng.integers(-2 ** 31 + 1, 2 ** 31 - 1, 10_000).astype(np.int32)])
        rows, pay, cnt = qe.qe_join_probe(ctx, ht, cuda(pk))
        rr, rp = O.join(bk, bp, pk)
        c = int(cnt.item())
        assert c == len(rr) and np.array_equal(rows[:c].cpu().numpy(), rr)
        assert np.array_equal(pay[:c].cpu().numpy(), rp)
        ht.destroy()
        dup = np.concatenate([bk, hot[-1:]])
        with pytest.raises(qe.QeError) as e:
            qe.qe_join_build(ctx, cuda(dup), cuda(np.zeros(len(dup), np.int32)), layout=qe.HT_OPEN)
        assert e.value.status == qe.ERR_DUPLICATE_KEY
    finally:
        ctx.set_tuning("join_part_log2", 0)
