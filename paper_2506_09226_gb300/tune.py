"""Autotuner for launch shapes, group-table placement, partition fan-out
and join-table layout.

Candidates are timed on the device with CUDA events and the fastest is
cached in a JSON file, keyed by a bucket of the workload's shape, so the
search runs once per bucket:
  - batched form: rows per work item (16K .. 256K) and where per-block group
    tables live (shared memory, or HBM only);
  - fused pipeline: rows per thread of the star-shape kernel (2 or 3);
  - pipelines with many groups: the direct HBM hash table against the
    partitioned group-by at several fan-outs (parts of its first pass), and
    the join table's layout (dense array or open addressing).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import qe

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), ".tune_cache.json")
BATCH_ITEM_ROWS = (1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18)
BATCH_PLACEMENT = (0, -1)        # smem_slots: 0 = shared memory when it fits, -1 = HBM only
STAR_ITEMS = (2, 3)
# (gb_partition, gb_part_log2p): the direct HBM table, then the partitioned
# group-by with 64, 128 or 256 parts (0 = planned)
GROUP_PLACEMENT = ((1, 0), (2, 6), (2, 7), (2, 8))
JOIN_LAYOUTS = (qe.HT_DENSE, qe.HT_OPEN)


def batch_bucket(sizes) -> str:
    s = np.asarray(sizes, dtype=np.float64)
    return (f"batch:n{int(math.log2(max(1, len(s))))}:mean{int(math.log2(max(1.0, s.mean())))}"
            f":max{int(math.log2(max(1.0, s.max())))}")


def pipeline_bucket(n_fact: int, groups: int) -> str:
    return f"pipe:n{int(math.log2(max(1, n_fact)))}:g{int(math.log2(max(1, groups)))}"


def _load(path):
    try:
        return json.load(open(path))
    except Exception:
        return {}


def _save(path, cache):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def search(key: str, candidates, time_one, path: str = CACHE):
    """Best candidate for `key`: the cached one, or the fastest of time_one(c)."""
    cache = _load(path)
    if key in cache and cache[key]["best"] in [list(c) if isinstance(c, tuple) else c for c in candidates]:
        b = cache[key]["best"]
        return tuple(b) if isinstance(b, list) else b
    timings = {}
    for c in candidates:
        timings[json.dumps(c)] = float(time_one(c))
    best = min(candidates, key=lambda c: timings[json.dumps(c)])
    cache[key] = {"best": list(best) if isinstance(best, tuple) else best, "ms": timings}
    _save(path, cache)
    return best


def tune_batch(ctx, sizes, make_batch, stream, steps: int = 2, path: str = CACHE) -> qe.qe_batch_opts:
    """make_batch(opts) -> qe.Batch over the workload; returns the best opts."""
    import torch

    def time_one(c):
        rows, place = c
        b = make_batch(qe.qe_batch_opts(0, rows, place, 1))
        b.launch(stream)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            b.launch(stream)
        e.record(stream)
        e.synchronize()
        b.destroy(stream)
        return a.elapsed_time(e) / steps
    rows, place = search(batch_bucket(sizes), [(r, p) for r in BATCH_ITEM_ROWS for p in BATCH_PLACEMENT],
                         time_one, path)
    return qe.qe_batch_opts(0, rows, place, 1)


def tune_pipeline(ctx, n_fact: int, groups: int, run, stream, steps: int = 3, path: str = CACHE) -> int:
    """run() executes the pipeline once; returns and applies the best star_items."""
    import torch

    def time_one(items):
        ctx.set_tuning("star_items", items)
        run()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            run()
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e) / steps
    best = search(pipeline_bucket(n_fact, groups), list(STAR_ITEMS), time_one, path)
    ctx.set_tuning("star_items", best)
    return best


def placement_bucket(n_fact: int, groups: int, n_dim: int) -> str:
    return (f"group:n{int(math.log2(max(1, n_fact)))}:g{int(math.log2(max(1, groups)))}"
            f":d{int(math.log2(max(1, n_dim)))}")


def tune_group_placement(ctx, desc, run, stream, steps: int = 2, path: str = CACHE):
    """Pick, by timing run() (one pipeline call over `desc`), where a
    many-group pipeline aggregates -- the direct HBM hash table or the
    partitioned group-by, and at which fan-out -- and the layout of the join
    table its call builds (dense array or open addressing).  Applies the
    best (knobs on the context, layout in desc.build) and returns
    (gb_partition, gb_part_log2p, layout)."""
    import torch

    old_layout = desc.build.layout

    def time_one(c):
        part, log2p, layout = c
        ctx.set_tuning("gb_partition", part)
        ctx.set_tuning("gb_part_log2p", log2p)
        desc.build.layout = layout
        run()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            run()
        e.record(stream)
        e.synchronize()
        return a.elapsed_time(e) / steps
    cands = [(p, lp, lay) for p, lp in GROUP_PLACEMENT for lay in JOIN_LAYOUTS]
    try:
        best = search(placement_bucket(desc.n_fact, desc.expected_groups, desc.n_dim), cands, time_one, path)
    except Exception:
        desc.build.layout = old_layout
        ctx.set_tuning("gb_partition", 0)
        ctx.set_tuning("gb_part_log2p", 0)
        raise
    part, log2p, layout = best
    ctx.set_tuning("gb_partition", part)
    ctx.set_tuning("gb_part_log2p", log2p)
    desc.build.layout = layout
    return best
