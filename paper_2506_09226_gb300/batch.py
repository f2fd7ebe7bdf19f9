"""Batched form: many star pipelines in one persistent launch (qe_batch_*),
its per-operator and per-pipeline baselines, and the benchmark of both.

A batch of pipelines (each group-by(join(filter(fact), dim)) over its own
tables) runs as the work items of one kernel captured in a CUDA graph; the
baselines run the same pipelines one at a time, either as separate operator
calls (filter, build, probe, group-by, reading each intermediate size back to
the host as a tensor program does) or as one fused qe_pipeline call each.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import torch

from . import datagen, qe

STAR_COLS = ("fk", "date", "price", "qty", "flag")
STAR_AGGS = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
N_ATTR = 25            # configuration-0 schema: 3 flags x 25 attributes = 75 groups
CAPACITY = 128
DATE_LT = 1278


class BatchOutputs:
    """One output block for many pipelines: keys [n, cap], aggs [4, n, cap]."""

    def __init__(self, n: int, capacity: int, device):
        self.capacity = capacity
        self.keys = torch.empty((n, capacity), dtype=torch.int64, device=device)
        self.aggs = torch.empty((4, n, capacity), dtype=torch.int64, device=device)
        self.ngroups = torch.zeros(n, dtype=torch.int64, device=device)
        ks, as_, ns = self.keys.data_ptr(), self.aggs.data_ptr(), self.ngroups.data_ptr()
        row = capacity * 8
        plane = n * row
        self.structs = [qe.qe_groups_out(capacity, ks + i * row,
                                         (ctypes.c_void_p * qe.MAX_AGGS)(*[as_ + a * plane + i * row
                                                                           for a in range(4)]),
                                         ns + i * 8) for i in range(n)]

    def groups(self, i: int):
        """(keys, [aggs]) of pipeline i as numpy, sorted by key."""
        n = min(int(self.ngroups[i].item()), self.capacity)
        k = self.keys[i, :n].cpu().numpy()
        o = np.argsort(k, kind="stable")
        return k[o], [self.aggs[a, i, :n].cpu().numpy()[o] for a in range(4)]


def star_descs(w: dict, lo: int = 0, hi: int | None = None, hts=None):
    """Pipeline descriptors over views of a batch_star workload."""
    f, d = w["fact"], w["dim"]
    hi = len(w["sizes"]) if hi is None else hi
    descs = []
    for i in range(lo, hi):
        a, n = int(w["fact_off"][i]), int(w["sizes"][i])
        b, nd = int(w["dim_off"][i]), int(w["dim_sizes"][i])
        cols = [f[c][a:a + n] for c in STAR_COLS]
        ht = hts[i] if hts is not None else None
        descs.append(qe.pipeline_desc(cols, [(1, qe.LT, DATE_LT)], fk_col=0, dim_key=d["key"][b:b + nd],
                                      dim_payload=d["attr"][b:b + nd], ht=ht, key_hi_col=4,
                                      key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS, dim_key_range=(0, nd - 1),
                                      key_range=((0, 2), (0, N_ATTR - 1)), expected_groups=75))
    return descs


def per_operator(ctx, w: dict, i: int, scratch: dict, stream=None):
    """Pipeline i as separate operator calls, sizes read back between them."""
    f, d = w["fact"], w["dim"]
    a, n = int(w["fact_off"][i]), int(w["sizes"][i])
    b, nd = int(w["dim_off"][i]), int(w["dim_sizes"][i])
    sel, cnt, rows, attr, jc = scratch["sel"], scratch["cnt"], scratch["rows"], scratch["attr"], scratch["jc"]
    qe.qe_filter(ctx, [f["date"][a:a + n]], [(0, qe.LT, DATE_LT)], sel, cnt, check=False)
    nsel = int(cnt.item())
    ht = qe.qe_join_build(ctx, d["key"][b:b + nd], d["attr"][b:b + nd], key_range=(0, nd - 1), check=False)
    qe.qe_join_probe(ctx, ht, f["fk"][a:a + n], sel, n=nsel, capacity=sel.numel(), out_rows=rows,
                     out_payload=attr, out_count=jc, check=False)
    nj = int(jc.item())
    g = qe.qe_groupby(ctx, attr, [(qe.SUM, f["price"][a:a + n], f["qty"][a:a + n], True), (qe.COUNT, None, None),
                                  (qe.MIN, f["price"][a:a + n], None, True), (qe.MAX, f["price"][a:a + n], None, True)],
                      key_hi=f["flag"][a:a + n], gather_hi=True, rows=rows, n=nj, capacity=CAPACITY, check=False)
    ht.destroy()
    return g


def _event_ms(fn, stream):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


def plan_waves(sizes, free_bytes: int, frac: float = 0.8):
    """Split pipelines into waves whose data and tables fit `frac` of free HBM."""
    per = [21 * n + 8 * max(1, n // 10) + 5 * max(1, n // 10) + 400_000 for n in sizes]
    waves, cur, acc = [], [], 0
    for i, c in enumerate(per):
        if cur and acc + c > frac * free_bytes:
            waves.append(cur)
            cur, acc = [], 0
        cur.append(i)
        acc += c
    if cur:
        waves.append(cur)
    return waves


def bench_batch(ctx, count: int, device, stream, peak_gbs: float, log=print, steps: int = 3,
                opts: qe.qe_batch_opts | None = None, seed: int = 4) -> dict:
    """Time `count` log-uniform star pipelines in one persistent launch against
    per-operator calls and per-pipeline fused calls."""
    sizes = datagen.log_uniform_sizes(count, 1e3, 1e7, seed=seed)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    waves = plan_waves(sizes, free)
    log(f"batch: {count} pipelines, {int(sizes.sum())} fact rows, {len(waves)} wave(s)")
    t_batch = t_perop = t_solo = 0.0
    tuned = opts is None
    launches = 0
    for wi, idx in enumerate(waves):
        t0 = time.time()
        w = datagen.batch_star(sizes[idx], N_ATTR, seed=seed * 100 + wi, device=device)
        torch.cuda.synchronize()
        log(f"  wave {wi}: {len(idx)} pipelines generated in {time.time() - t0:.1f}s")
        outs = BatchOutputs(len(idx), CAPACITY, device)
        descs = star_descs(w)
        if opts is None:
            from . import tune
            opts = tune.tune_batch(ctx, sizes[idx], lambda o: qe.Batch(ctx, descs, outs.structs, o, stream), stream)
            log(f"  tuned: item rows {opts.tile_rows}, smem_slots {opts.smem_slots}")
        b = qe.Batch(ctx, descs, outs.structs, opts, stream)
        b.launch(stream)
        ctx.sync_status(stream)
        l0 = ctx.launch_count()
        t_batch += sum(_event_ms(lambda: b.launch(stream), stream) for _ in range(steps)) / steps
        launches += (ctx.launch_count() - l0) // steps
        ctx.sync_status(stream)
        b.destroy(stream)
        # per-pipeline fused calls
        out1, cout1 = qe.alloc_groups(CAPACITY, 4, device)

        def solo():
            for d in descs:
                qe.qe_pipeline(ctx, d, CAPACITY, stream=stream, check=False, out=(out1, cout1))
        t_solo += _event_ms(solo, stream)
        # per-operator calls
        mx = int(max(sizes[idx]))
        scratch = {"sel": torch.empty(mx, dtype=torch.int32, device=device),
                   "cnt": torch.empty(1, dtype=torch.int64, device=device),
                   "rows": torch.empty(mx, dtype=torch.int32, device=device),
                   "attr": torch.empty(mx, dtype=torch.int32, device=device),
                   "jc": torch.empty(1, dtype=torch.int64, device=device)}

        def perop():
            for i in range(len(idx)):
                per_operator(ctx, w, i, scratch, stream)
        t_perop += _event_ms(perop, stream)
        ctx.sync_status(stream)
        del w, outs, descs, scratch
        torch.cuda.empty_cache()
    rows = int(sizes.sum())
    alg = sum(21 * n + 8 * max(1, n // 10) for n in sizes)
    return {"pipelines": count, "fact_rows": rows, "waves": len(waves), "item_rows": int(opts.tile_rows),
            "placement": "smem" if opts.smem_slots == 0 else "hbm", "autotuned": tuned,
            "batched": {"ms": t_batch, "rows_per_s": rows / (t_batch * 1e-3),
                        "hbm_frac": round(alg / (t_batch * 1e-3) / 1e9 / peak_gbs, 4),
                        "kernel_launches_per_pass": launches, "cuda_graph": bool(opts.use_graph)},
            "per_pipeline_fused": {"ms": t_solo, "rows_per_s": rows / (t_solo * 1e-3)},
            "per_operator": {"ms": t_perop, "rows_per_s": rows / (t_perop * 1e-3)},
            "speedup_vs_per_operator": t_perop / t_batch, "speedup_vs_per_pipeline": t_solo / t_batch}


def kind_descs(w: dict, kinds) -> list:
    """Pipeline descriptors over a batch_star workload whose join kinds cycle
    through `kinds` (qe.INNER, qe.SEMI, qe.ANTI, or "none" for no join):
    inner joins group by (flag, attribute) as star_descs does; the others
    group by flag, and a semi- or anti-join tests membership in the first
    half of the pipeline's dimension keys."""
    f, d = w["fact"], w["dim"]
    descs = []
    for i in range(len(w["sizes"])):
        a, n = int(w["fact_off"][i]), int(w["sizes"][i])
        b, nd = int(w["dim_off"][i]), int(w["dim_sizes"][i])
        cols = [f[c][a:a + n] for c in STAR_COLS]
        k = kinds[i % len(kinds)]
        if k == qe.INNER:
            descs.append(qe.pipeline_desc(cols, [(1, qe.LT, DATE_LT)], fk_col=0, dim_key=d["key"][b:b + nd],
                                          dim_payload=d["attr"][b:b + nd], key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD,
                                          aggs=STAR_AGGS, dim_key_range=(0, nd - 1),
                                          key_range=((0, 2), (0, N_ATTR - 1)), expected_groups=75))
        elif k == "none":
            descs.append(qe.pipeline_desc(cols, [(1, qe.LT, DATE_LT)], fk_col=-1, key_hi_col=-1, key_lo_col=4,
                                          aggs=STAR_AGGS, key_range=(None, (0, 2)), expected_groups=3))
        else:
            descs.append(qe.pipeline_desc(cols, [(1, qe.LT, DATE_LT)], fk_col=0, dim_key=d["key"][b:b + max(1, nd // 2)],
                                          key_hi_col=-1, key_lo_col=4, aggs=STAR_AGGS, dim_key_range=(0, nd - 1),
                                          key_range=(None, (0, 2)), expected_groups=3, join_kind=k))
    return descs


def bench_batch_kinds(ctx, count: int, device, stream, peak_gbs: float, steps: int = 3, seed: int = 9) -> dict:
    """`count` log-uniform pipelines whose join kinds cycle semi, anti, none,
    inner, in one persistent launch, against per-pipeline fused calls.
    Algorithmic bytes: 21 per fact row (17 without a join) plus 4 per key
    built into a semi- / anti-join key set and 8 per dimension row of an
    inner join."""
    kinds = (qe.SEMI, qe.ANTI, "none", qe.INNER)
    sizes = datagen.log_uniform_sizes(count, 1e3, 1e7, seed=seed)
    w = datagen.batch_star(sizes, N_ATTR, seed=seed, device=device)
    descs = kind_descs(w, kinds)
    outs = BatchOutputs(count, CAPACITY, device)
    b = qe.Batch(ctx, descs, outs.structs, qe.qe_batch_opts(0, 1 << 18, 0, 1), stream)
    b.launch(stream)
    ctx.sync_status(stream)
    t_batch = min(_event_ms(lambda: b.launch(stream), stream) for _ in range(steps))
    ctx.sync_status(stream)
    b.destroy(stream)
    out1, cout1 = qe.alloc_groups(CAPACITY, 4, device)

    def solo():
        for d in descs:
            qe.qe_pipeline(ctx, d, CAPACITY, stream=stream, check=False, out=(out1, cout1))
    solo()
    ctx.sync_status(stream)
    t_solo = _event_ms(solo, stream)
    alg = 0
    for i, n in enumerate(sizes):
        k, nd = kinds[i % len(kinds)], max(1, int(n) // 10)
        alg += (17 if k == "none" else 21) * int(n) + (8 * nd if k == qe.INNER else 0) + \
            (4 * max(1, nd // 2) if k in (qe.SEMI, qe.ANTI) else 0)
    rows = int(sizes.sum())
    del w, outs, descs
    torch.cuda.empty_cache()
    return {"pipelines": count, "fact_rows": rows, "kinds": "semi, anti, none, inner (cycling)",
            "batched": {"ms": t_batch, "rows_per_s": rows / (t_batch * 1e-3),
                        "hbm_frac": round(alg / (t_batch * 1e-3) / 1e9 / peak_gbs, 4)},
            "per_pipeline_fused": {"ms": t_solo, "rows_per_s": rows / (t_solo * 1e-3)},
            "speedup_vs_per_pipeline": t_solo / t_batch}
