"""Failure paths, exercised without a GPU fault.

The paper recovers from failures by re-executing work (Sec. 2.4: each GPU
runs its own program over its local data); what the library owes a caller
is that a failed call reports a status, leaves nothing behind and leaves the
context usable, so the caller can retry.  Two failure sources are tested:

* allocation failure, injected on the host (qe_debug_fail_alloc): the n-th
  library allocation of a call fails for every n the call makes, the call
  returns QE_ERR_OOM, qe_bytes_in_use returns to what it was before, and the
  same call then succeeds with the oracle's result;
* a bounded device wait that runs out: the batch kernel's probe items wait
  (bounded) for the build items of their pipeline; with the wait limit
  shortened to one iteration and a build item still running when the first
  probe item is claimed, the wait expires, the kernel records
  QE_ERR_TIMEOUT and returns, and the next run with the default limit is
  correct.

Nothing here faults, traps or hangs the GPU: every wait is bounded, and the
failures are made on the host or by a short limit.
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
O_STAR = O.Query(preds=[O.Pred(1, O.LT, 1278)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD,
                 aggs=[(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)])


@pytest.fixture(scope="module")
def ctx():
    c = qe.Context(0)
    yield c
    c.debug_fail_alloc(0)
    c.debug_set_spin_limit(0)
    c.close()


def _sorted(g):
    k, a = g.to_host()
    o = np.argsort(k.numpy(), kind="stable")
    return k.numpy()[o], [x.numpy()[o] for x in a]


def _equal(g, ref):
    k, a = _sorted(g)
    assert np.array_equal(k, ref["keys"])
    for x, y in zip(a, ref["aggs"]):
        assert np.array_equal(x, y)


def _fails_then_recovers(ctx, call, check, max_allocs=12):
    """Arm the n-th allocation to fail for n = 1, 2, ... until the call no
    longer allocates that many times; every failing call returns OOM and
    leaks nothing.  Returns the number of allocations the call makes."""
    torch.cuda.synchronize()
    base = ctx.bytes_in_use()
    for n in range(1, max_allocs + 1):
        ctx.debug_fail_alloc(n)
        try:
            out = call()
        except qe.QeError as e:
            assert e.status == qe.ERR_OOM, (n, e)
            assert "injected" in str(e)
            torch.cuda.synchronize()
            assert ctx.bytes_in_use() == base, n
            continue
        finally:
            ctx.debug_fail_alloc(0)
        torch.cuda.synchronize()
        ctx.sync_status()
        check(out)
        assert ctx.bytes_in_use() == base
        return n - 1
    raise AssertionError("the call kept allocating")


def test_oom_pipeline_every_allocation(ctx):
    """The fused pipeline with its join build inside the call and 25,002
    groups in an HBM direct array: key-range scratch, join table, direct
    array and hash table are each made to fail in turn."""
    dim = datagen.star_dim(50_000, 8334, seed=31)
    fact = datagen.star_fact(200_001, 50_000, seed=31)
    f = [fact[c].cuda() for c in COLS]
    d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=dim["key"].cuda(), dim_payload=dim["attr"].cuda(),
                         key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS, key_range=((0, 2), (0, 8333)))
    ref = O.pipeline([fact[c].numpy() for c in COLS], O_STAR, dim["key"].numpy(), dim["attr"].numpy())
    n = _fails_then_recovers(ctx, lambda: qe.qe_pipeline(ctx, d, 30_000), lambda g: _equal(g, ref))
    assert n >= 3


def test_oom_partition_and_filter(ctx):
    """The partition's scratch (two passes at fan-out 1024) and the
    two-pass filter's scratch (from 4M rows on)."""
    key, pay = datagen.key_payload_pairs(70_001, seed=32)
    okey, opay = O.partition(key.numpy(), [pay.numpy()], 10)[:2]
    kd, pd = key.cuda(), pay.cuda()

    def part():
        return qe.qe_partition(ctx, kd, [pd], 10)

    def check_part(out):
        assert np.array_equal(out[0].cpu().numpy(), okey)
        assert np.array_equal(out[1][0].cpu().numpy(), opay[0])
    assert _fails_then_recovers(ctx, part, check_part) >= 1

    date = datagen.star_fact(5_000_000, 1000, seed=33)["date"]
    ref = O.filter([date.numpy()], [O.Pred(0, O.LT, 1278)])
    dd = date.cuda()

    def filt():
        return qe.qe_filter(ctx, [dd], [(0, qe.LT, 1278)])

    def check_filt(out):
        sel, cnt = out
        assert int(cnt.item()) == len(ref)
        assert np.array_equal(sel[:len(ref)].cpu().numpy(), ref)
    assert _fails_then_recovers(ctx, filt, check_filt) >= 1


def test_budget_exhaustion_is_oom_and_recoverable():
    """A context whose HBM budget cannot hold a call's scratch returns OOM,
    holds nothing afterwards, and serves calls that fit."""
    c = qe.Context(0, hbm_budget_bytes=64 * 1024)
    try:
        key, pay = datagen.key_payload_pairs(200_000, seed=34)
        with pytest.raises(qe.QeError) as e:
            qe.qe_partition(c, key.cuda(), [pay.cuda()], 12)
        assert e.value.status == qe.ERR_OOM and "budget" in str(e.value)
        assert c.bytes_in_use() == 0
        k = torch.arange(1000, dtype=torch.int64, device="cuda") % 10
        g = qe.qe_groupby(c, k, [(qe.COUNT, None, None)], capacity=16)
        assert int(g.ngroups.item()) == 10
        assert c.bytes_in_use() == 0
    finally:
        c.close()


def test_short_spin_limit_times_out_and_context_recovers(ctx):
    """A batch whose dimension has one more build item (65,536 rows each)
    than the GPU has SMs: the block that claims the first probe item finds
    the last build item still running, and with a one-iteration wait limit
    its wait expires.  The kernel returns, QE_ERR_TIMEOUT is reported, and
    the same batch with the default limit matches the oracle."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nd = (sms + 1) * 65536
    dim = datagen.star_dim(nd, 25, seed=35)
    fact = datagen.star_fact(300_000, nd, seed=35)
    f = [fact[c].cuda() for c in COLS]
    dk, da = dim["key"].cuda(), dim["attr"].cuda()
    d = qe.pipeline_desc(f, [(1, qe.LT, 1278)], fk_col=0, dim_key=dk, dim_payload=da, key_hi_col=4,
                         key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS, dim_key_range=(0, nd - 1),
                         key_range=((0, 2), (0, 24)), expected_groups=75)
    g, o = qe.alloc_groups(128, 4, torch.device("cuda"))
    opts = qe.qe_batch_opts(0, 1 << 16, 0, 0)
    ctx.debug_set_spin_limit(1)
    try:
        with pytest.raises(qe.QeError) as e:
            qe.qe_batch_run(ctx, [d], [o], opts=opts)
        assert e.value.status == qe.ERR_TIMEOUT
    finally:
        ctx.debug_set_spin_limit(0)
    ctx.sync_status()                      # the error was cleared with the report
    g.ngroups.fill_(-1)
    qe.qe_batch_run(ctx, [d], [o], opts=opts)
    ref = O.pipeline([fact[c].numpy() for c in COLS], O_STAR, dim["key"].numpy(), dim["attr"].numpy())
    _equal(g, ref)
