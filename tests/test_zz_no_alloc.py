"""qe_filter_noalloc: the filter for callers that cannot allocate device memory.

Some hosts own all device memory through their own allocator (a library
cudaMalloc would fail or fragment that pool), and some latency-critical
callers cannot afford an allocator call, which may synchronize the device;
qe_filter_noalloc serves them by keeping its scratch in a static device
array of the library instead of allocating per call.

The test calls it through the C ABI twice in a row, on different inputs and
predicates, and requires its selection and count to equal bit for bit (the
tolerance of every integer result in this suite) both qe_filter's and the
CPU oracle's.  The first input has 5,000,011 rows, where qe_filter runs its
two-pass kernels, so the one-pass kernel of the no-alloc call is checked
against a different code path as well as against the oracle.  While the
calls run, the context is armed to fail its next allocation and its
allocated bytes are watched, so any allocation inside the call would fail
the test.  A size beyond the static limit must be rejected on the host
before anything runs.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_09226_gb300 import datagen, qe

pytestmark = pytest.mark.gpu

OPS = {qe.LT: O.LT, qe.BETWEEN: O.BETWEEN, qe.NE: O.NE}


def _run_both(ctx, host_cols, preds):
    n = len(host_cols[0])
    cols = [torch.from_numpy(c).cuda() for c in host_cols]
    ref = O.filter(host_cols, [O.Pred(p[0], OPS[p[1]], p[2], p[3] if len(p) > 3 else 0) for p in preds])
    ex_sel, ex_cnt = qe.qe_filter(ctx, cols, preds)
    out_sel = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    out_cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    before = ctx.bytes_in_use()
    ctx.debug_fail_alloc(1)             # an allocation inside the call would fail it
    try:
        sel, cnt = qe.qe_filter_noalloc(ctx, cols, preds, out_sel, out_cnt)
    finally:
        ctx.debug_fail_alloc(0)
    assert ctx.bytes_in_use() == before
    c = int(cnt.item())
    assert c == len(ref) == int(ex_cnt.item())
    got = sel[:c].cpu().numpy()
    assert np.array_equal(got, ref)
    assert np.array_equal(got, ex_sel[:c].cpu().numpy())
    return c


def test_noalloc_matches_filter_and_oracle_twice():
    ctx = qe.Context(0)
    try:
        n1 = 5_000_011                                  # qe_filter's two-pass range; a ragged tail
        f1 = datagen.star_fact(n1, 1000, seed=21)
        c1 = _run_both(ctx, [f1["date"].numpy()], [(0, qe.LT, 1278)])
        assert 0 < c1 < n1
        # second call: other data, other predicates, fewer tiles; the static
        # scratch still holds the first call's state and must be cleared
        n2 = 777_777
        f2 = datagen.star_fact(n2, 1000, seed=22)
        c2 = _run_both(ctx, [f2["qty"].numpy(), f2["flag"].numpy()], [(0, qe.BETWEEN, 10, 30), (1, qe.NE, 1)])
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
