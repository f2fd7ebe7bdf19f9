"""qe_filter_noalloc: the filter for callers that cannot allocate device memory.

Some hosts own all device memory through their own allocator, and some
latency-critical callers cannot afford an allocator call (which may
synchronize the device); qe_filter_noalloc serves them by keeping its scratch
in a static device array of the library instead of allocating per call.
This test calls it through the C ABI twice in a row, on different inputs,
and requires its output to equal qe_filter's bit for bit (the tolerance of
every integer result in this suite), and checks that a size beyond the
static limit is rejected on the host before anything runs.  The file name
makes pytest collect it last.
"""
import numpy as np
import pytest
import torch

from paper_2506_09226_gb300 import datagen, qe

pytestmark = pytest.mark.gpu


def _run_both(ctx, cols, preds, n):
    ref_sel, ref_cnt = qe.qe_filter(ctx, cols, preds)
    out_sel = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    out_cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    sel, cnt = qe.qe_filter_noalloc(ctx, cols, preds, out_sel, out_cnt)
    c = int(cnt.item())
    assert c == int(ref_cnt.item())
    assert np.array_equal(sel[:c].cpu().numpy(), ref_sel[:c].cpu().numpy())
    return c


def test_noalloc_matches_filter_twice():
    ctx = qe.Context(0)
    try:
        n1 = 3_000_017                                  # several tiles and a ragged tail
        f1 = datagen.star_fact(n1, 1000, seed=21)
        c1 = _run_both(ctx, [f1["date"].cuda()], [(0, qe.LT, 1278)], n1)
        assert 0 < c1 < n1
        # second call: other data, other predicate, fewer tiles; the static
        # scratch still holds the first call's state and must be cleared
        n2 = 777_777
        f2 = datagen.star_fact(n2, 1000, seed=22)
        cols = [f2["qty"].cuda(), f2["flag"].cuda()]
        c2 = _run_both(ctx, cols, [(0, qe.BETWEEN, 10, 30), (1, qe.NE, 1)], n2)
        assert 0 < c2 < n2
    finally:
        ctx.close()


def test_noalloc_rejects_oversize_on_host():
    ctx = qe.Context(0)
    try:
        small = torch.zeros(16, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        with pytest.raises(qe.QeError) as e:
            qe.qe_filter_noalloc(ctx, [small], [(0, qe.LT, 1)], small, cnt,
                                 nrows=qe.FILTER_NOALLOC_MAX_ROWS + 1, check=False)
        assert e.value.status == qe.ERR_INVALID_ARG and "static scratch limit" in str(e.value)
    finally:
        ctx.close()
