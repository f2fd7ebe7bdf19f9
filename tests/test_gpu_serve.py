"""Served form on the GPU: every request's result in the concurrent mix is
bit-identical to the same request run alone, and to the CPU oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2506_09226_gb300 import datagen, qe, serve

pytestmark = pytest.mark.gpu

COLS = ("fk", "date", "price", "qty", "flag")
Q = dict(fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD,
         aggs=[(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)])


def test_served_mix_equals_solo_and_oracle():
    ctx = qe.Context(0)
    dev = torch.device("cuda", 0)
    shapes = [{"n_fact": 3_000_000, "n_dim": 10_000, "n_attr": 25},
              {"n_fact": 3_000_000, "n_dim": 200_000, "n_attr": 1000},
              {"n_fact": 3_000_000, "n_dim": 500_000, "n_attr": 1000, "zipf": 1.1}]
    tables = serve.ResidentTables(ctx, shapes, dev, log=lambda *a: None)
    trace = datagen.poisson_trace(0.15, 2000.0, tables.rows, seed=1, n_lo=1e3, n_hi=2e6)
    assert len(trace) > 100
    reqs_n = [a.n for a in trace]
    outs = serve.OutputSlots(len(trace) + 8, dev)
    rounds = []
    ex = serve.BatchExecutor(ctx, tables, outs, n_streams=3, on_round=lambda rs: rounds.append([r.rid for r in rs]),
                             single_rows=1_000_000)
    adm = serve.Admission(budget_bytes=(len(trace) + 8) * serve.REQ_BYTES, slots=len(trace) + 8)
    reqs = []
    orig = ex.launch

    def launch(rs):
        reqs.extend(rs)
        return orig(rs)
    ex.launch = launch
    st = serve.serve_loop(trace, ex, adm, row_cap=3_000_000)
    ctx.sync_status()
    assert len(st.latencies_ms) == len(trace) and st.rounds == len(rounds)
    assert max(len(r) for r in rounds) > 1                 # requests were batched together
    assert any(len(r) == 1 and reqs_n[r[0]] >= 1_000_000 for r in rounds)   # and large ones ran alone
    g1, o1 = qe.alloc_groups(serve.CAPACITY, 4, dev)
    for r in reqs:
        k, a = outs.groups(r.slot)
        solo = qe.qe_pipeline(ctx, tables.desc(r), serve.CAPACITY, out=(g1, o1))
        sk, sa = solo.to_host()
        o = np.argsort(sk.numpy(), kind="stable")
        assert np.array_equal(k, sk.numpy()[o])
        assert all(np.array_equal(x, y.numpy()[o]) for x, y in zip(a, sa))
    for r in reqs[:: max(1, len(reqs) // 6)]:              # a sample against the oracle
        f = tables.fact[r.shape]
        cols = [f[c][r.offset:r.offset + r.n].cpu().numpy() for c in COLS]
        d = tables.dim[r.shape]
        ref = O.pipeline(cols, O.Query(preds=[O.Pred(1, O.LT, r.date_hi)], **Q), d["key"].cpu().numpy(),
                         d["attr"].cpu().numpy())
        k, a = outs.groups(r.slot)
        assert np.array_equal(k, ref["keys"])
        assert all(np.array_equal(x, y) for x, y in zip(a, ref["aggs"]))
    tables.close()
    ctx.close()
