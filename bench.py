#!/usr/bin/env python
"""Benchmark of the GB300 relational operator pipeline (arxiv 2506.09226 hot path).

One step = one pass of the plain hot path over the at-scale star workload
(fact 600M rows x 21 B, dimension 20M rows, plus 600M (int64 key, int64
payload) pairs), all resident in HBM:
    qe_pipeline   join build over the dimension, then one fused pass over the
                  fact table: date < 1278, FK join, group by (flag, attr) with
                  SUM(price*qty), COUNT, MIN(price), MAX(price)  (3,000 groups)
    qe_partition  stable hash partition of the pairs at fan-out 1024
value = (fact rows + partition rows) per second of the step.  The inputs
(12.6 GB + 9.6 GB) are larger than the 126 MB L2, so no flush is needed.

Also reported on the same JSON line: the per-kernel roofline of the dominant
kernel, the per-kernel breakdown, partition at fan-out 256 / 4096, the
per-operator path (filter -> probe -> group-by as separate launches), the
25K-group variant, an end-to-end number through the public API with the
inputs copied from pinned host memory every step, the batched form (10,000
inner-join pipelines, and 600 pipelines whose join kinds cycle semi, anti,
none, inner) and the served form, clocks sampled during the timed region,
and the CPU oracle on a bounded sample (cpu_baseline).

--impl reference times the CPU oracle (oracle/) on a bounded sample of the
same workload, per step, and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "scanned rows/s & % of HBM peak per pipeline; served p50/p99 vs plain launches"
UNIT = "rows/s"
DATE_LT = 1278
BYTES_FACT_ROW = 21          # fk 4 + date 4 + price 8 + qty 4 + flag 1
BYTES_PAIR_MOVE = 32         # read key+payload 16 B, write 16 B


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- peaks / clocks
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.dev = device
        self.proc = None
        self.path = None

    def _gpu_id(self):
        try:
            u = str(torch.cuda.get_device_properties(self.dev).uuid)
            return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            return str(self.dev)

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self._gpu_id(), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: begin the timed region only once
        # it has written its first sample (bounded wait)
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- kernel traffic record
def kernel_source_hash(sources):
    """sha256 prefix over the files a kernel is compiled from (paths relative
    to the repository root, in the order given)."""
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, units: int):
    """DRAM bytes per launch from the committed ncu record, scaled to `units`,
    or None when the record is missing or any of the kernel's sources changed
    since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
        r = d[kernel]
        if r["source_hash"] != kernel_source_hash(r["sources"]):
            return None
    except Exception:
        return None
    return r["dram_bytes_per_unit"] * units


# ---------------------------------------------------------------- workload
def make_workload(n_fact, n_dim, n_pairs, n_attr, device):
    from paper_2506_09226_gb300 import datagen
    t0 = time.time()
    dim = datagen.star_dim(n_dim, n_attr, seed=1, device=device)
    fact = datagen.star_fact(n_fact, n_dim, seed=1, device=device)
    key, pay = datagen.key_payload_pairs(n_pairs, seed=2, device=device)
    torch.cuda.synchronize()
    log(f"workload generated in {time.time() - t0:.1f}s")
    return dim, fact, key, pay


COLS = ("fk", "date", "price", "qty", "flag")


def star_desc(qe, fact, dim, expected_groups):
    # key_range: the flag column's min/max statistics (domain {0,1,2}); the
    # attribute's range is read back by the join build
    return qe.pipeline_desc([fact[c] for c in COLS], [(1, qe.LT, DATE_LT)], fk_col=0, dim_key=dim["key"],
                            dim_payload=dim["attr"], key_hi_col=4, key_lo_col=qe.JOIN_PAYLOAD,
                            aggs=[(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)],
                            expected_groups=expected_groups, est_selectivity=DATE_LT / 2557,
                            key_range=((0, 2), None))


# ---------------------------------------------------------------- CPU oracle leg
class OracleSample:
    """A bounded, proportionally scaled instance of the step's workload for
    the CPU oracle: n fact rows with n // 30 dimension rows (the 600M : 20M
    ratio of the at-scale star), the same distributions and query, and n
    (key, payload) pairs at the same fan-out.  Generated once; run() times
    the oracle alone."""

    def __init__(self, n, log2f, n_attr=1000):
        from oracle import oracle as O
        from paper_2506_09226_gb300 import datagen
        self.O, self.n, self.log2f = O, n, log2f
        self.nd = max(1, n // 30)
        dim = datagen.star_dim(self.nd, n_attr, seed=1)
        fact = datagen.star_fact(n, self.nd, seed=1)
        key, pay = datagen.key_payload_pairs(n, seed=2)
        self.fl = [fact[c].numpy() for c in COLS]
        self.q = O.Query(preds=[O.Pred(1, O.LT, DATE_LT)], fk_col=0, key_hi_col=4, key_lo_col=O.JOIN_PAYLOAD,
                         aggs=[(O.SUM, 2, 3), (O.COUNT, -1, -1), (O.MIN, 2, -1), (O.MAX, 2, -1)])
        self.dk, self.da, self.kk, self.pp = dim["key"].numpy(), dim["attr"].numpy(), key.numpy(), pay.numpy()
        O.lib()

    def run(self):
        """Seconds for one step: the pipeline over the fact sample, then the partition."""
        t0 = time.perf_counter()
        self.O.pipeline(self.fl, self.q, self.dk, self.da)
        self.O.partition(self.kk, [self.pp], self.log2f)
        return time.perf_counter() - t0

    @property
    def rows(self):
        return 2 * self.n

    @property
    def desc(self):
        return (f"oracle (single-threaded C): the star pipeline over {self.n} fact rows joined to {self.nd} "
                f"dimension rows (the 30:1 ratio of the 600M x 20M workload), plus {self.n} pairs partitioned "
                f"at fan-out {1 << self.log2f}; rows = fact + pairs")


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    W, K = args.warmup, args.steps
    sample = OracleSample(args.ref_sample, args.log2f)
    times = []
    for i in range(W + K):
        dt = sample.run()
        if i >= W:
            times.append(dt)
        log(f"reference step {i}: {dt:.2f}s")
    t = sum(times) / len(times)
    v = sample.rows / t
    desc = sample.desc
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": K, "warmup": W,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic", "impl": "reference",
            "config": workload_config(args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                             **host_cores()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def host_cores() -> dict:
    """The host's core count (os.cpu_count) and the cores this process may
    run on (its affinity mask), reported beside the single-threaded oracle."""
    try:
        aff = sorted(os.sched_getaffinity(0))
    except AttributeError:
        aff = list(range(os.cpu_count() or 1))
    return {"host_nproc": os.cpu_count(), "affinity_cores": len(aff),
            "affinity": f"{aff[0]}-{aff[-1]}" if aff and aff == list(range(aff[0], aff[-1] + 1)) else
            ",".join(map(str, aff))}


def workload_config(args):
    return {"workload": f"star pipeline at scale: fact {args.fact_rows} rows, dim {args.dim_rows} rows "
                        f"(attr in [0,1000)), date<{DATE_LT}, FK join, group by (flag,attr) 3000 groups, "
                        f"+ hash partition of {args.pairs} (int64,int64) pairs at fan-out {1 << args.log2f}",
            "fact_rows": args.fact_rows, "dim_rows": args.dim_rows, "pairs": args.pairs,
            "fanout": 1 << args.log2f, "l2": "inputs larger than L2 (12.6 GB + 9.6 GB vs 126 MB)",
            "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "1 GPU"}


# ---------------------------------------------------------------- our arm
def job_time(ms_local: float, dist=None, device=None) -> float:
    """The step time of the whole job: the maximum over ranks (replicas run
    the same step on their own GPU), by an all-reduce when distributed."""
    if dist is None:
        return ms_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the job time."""
    return units_per_rank * world / (ms * 1e-3)


def timed(fn, iters, stream):
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(iters):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / iters


def run_qe(args):
    from paper_2506_09226_gb300 import qe
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ctx = qe.Context(local)
    peak, peak_kind = hbm_peak()

    dim, fact, key, pay = make_workload(args.fact_rows, args.dim_rows, args.pairs, 1000, dev)
    F = 1 << args.log2f
    desc = star_desc(qe, fact, dim, 3000)
    groups, gout = qe.alloc_groups(4096, 4, dev)
    okeys, opay = torch.empty_like(key), torch.empty_like(pay)
    offs = torch.empty(F + 1, dtype=torch.int64, device=dev)

    def step():
        qe.qe_pipeline(ctx, desc, 4096, check=False, out=(groups, gout))
        qe.qe_partition(ctx, key, [pay], args.log2f, qe.PART_HASH, 0, okeys, [opay], offs, check=False)

    for _ in range(args.warmup):
        step()
    ctx.sync_status()
    # ---- timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_reset()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = ctx.launch_count()
    ms = timed(step, args.steps, stream)
    launches = ctx.launch_count() - l0
    clocks = sampler.stop()
    ms = job_time(ms, dist, dev)
    ctx.sync_status()
    prof = {n: ctx.profile_read(n) for n in ("build", "pipeline", "part_hist", "part_scatter")}
    ctx.profile(False)
    ngroups = int(groups.ngroups.item())
    rows_step = args.fact_rows + args.pairs
    value = job_value(rows_step, world, ms)

    # ---- per-kernel breakdown and the dominant kernel's roofline
    alg_bytes = {"pipeline": BYTES_FACT_ROW * args.fact_rows,
                 "part_scatter": BYTES_PAIR_MOVE * args.pairs,
                 "part_hist": 8 * args.pairs,
                 "build": 8 * args.dim_rows + 4 * args.dim_rows}
    units = {"pipeline": args.fact_rows, "part_scatter": args.pairs, "part_hist": args.pairs,
             "build": args.dim_rows}
    breakdown = {}
    for n, (cnt, tot) in prof.items():
        if cnt:
            avg = tot / cnt
            gbs = alg_bytes[n] / (avg * 1e-3) / 1e9
            breakdown[n] = {"ms": round(avg, 4), "launches_per_step": cnt / args.steps,
                            "alg_bytes": alg_bytes[n], "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
    dom = max(breakdown, key=lambda n: breakdown[n]["ms"])
    d = breakdown[dom]
    traffic = recorded_traffic(dom, units[dom])
    roofline = {"bound": "hbm", "kernel": dom, "achieved": d["gbs"], "peak": peak, "unit": "GB/s",
                "frac": d["frac"], "traffic": traffic, "peak_kind": peak_kind,
                "alg_bytes_per_launch": d["alg_bytes"]}
    step_bytes = alg_bytes["pipeline"] + alg_bytes["part_scatter"] + 12 * args.dim_rows
    pipelines = {"step": {"ms": ms, "rows_per_s": value / world,
                          "hbm_frac_of_step_alg_bytes": round(step_bytes / (ms * 1e-3) / 1e9 / peak, 4)},
                 "fused_pipeline_call": None, "kernels": breakdown}

    extras = {}
    if "extras" in args.forms:
        extras = run_extras(args, qe, ctx, fact, dim, key, pay, okeys, opay, dev, stream, peak)
        pipelines["fused_pipeline_call"] = extras.pop("fused_call", None)

    # ---- end to end through the public API with pinned host inputs
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, qe, ctx, fact, dim, key, pay, okeys, opay, offs, groups, gout, dev, stream)

    # ---- batched and served forms
    forms = {}
    if "batch" in args.forms or "serve" in args.forms:
        del okeys, opay, dim, fact, key, pay, desc, groups, gout
        torch.cuda.empty_cache()
        forms = run_forms(args, qe, ctx, dev, stream, None, None, peak)
    # the join variants and the skewed, high-cardinality pipeline last: their
    # multi-GB tables stay out of the way of the batch and serve forms
    if "variants" in args.forms:
        try:
            extras["variants"] = run_variants(args, qe, ctx, dev, stream, peak, max(3, args.steps // 2))
        except qe.QeError as e:   # a library error in an extra leg is reported, not fatal to the line
            extras["variants"] = {"error": str(e)}
            torch.cuda.empty_cache()
    if "extras" in args.forms or "skew" in args.forms:
        extras["skew_40m_groups"] = run_skew(args, qe, ctx, dev, stream, peak, max(9, args.steps // 2))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sample = OracleSample(args.cpu_sample, args.log2f)
        runs = [sample.run() for _ in range(2)]
        dt = sum(runs) / len(runs)
        cpu = {"value": sample.rows / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": sample.desc + f"; mean of 2 runs ({sum(runs):.1f} s of CPU work)", **host_cores()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": workload_config(args),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches, "ngroups": ngroups, "pipelines": pipelines, **extras, **forms}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_extras(args, qe, ctx, fact, dim, key, pay, okeys, opay, dev, stream, peak):
    out = {}
    it = max(3, args.steps // 2)
    # the fused pipeline call alone
    groups, gout = qe.alloc_groups(4096, 4, dev)
    desc = star_desc(qe, fact, dim, 3000)
    fn = lambda: qe.qe_pipeline(ctx, desc, 4096, check=False, out=(groups, gout))  # noqa: E731
    fn()
    ms = timed(fn, it, stream)
    b = BYTES_FACT_ROW * args.fact_rows + 12 * args.dim_rows
    out["fused_call"] = {"ms": ms, "rows_per_s": args.fact_rows / (ms * 1e-3),
                         "hbm_frac": round(b / (ms * 1e-3) / 1e9 / peak, 4)}
    # partition at each fan-out
    part = {}
    for lf in (8, 10, 12):
        offs = torch.empty((1 << lf) + 1, dtype=torch.int64, device=dev)
        fn = lambda: qe.qe_partition(ctx, key, [pay], lf, qe.PART_HASH, 0, okeys, [opay], offs,  # noqa: E731
                                     check=False)
        fn()
        ms = timed(fn, it, stream)
        part[str(1 << lf)] = {"ms": ms, "rows_per_s": args.pairs / (ms * 1e-3),
                              "hbm_frac": round(BYTES_PAIR_MOVE * args.pairs / (ms * 1e-3) / 1e9 / peak, 4)}
    out["partition"] = part
    # per-operator path: filter -> build -> probe -> group-by as separate launches
    n = args.fact_rows
    sel = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    rows = torch.empty(n, dtype=torch.int32, device=dev)
    attr = torch.empty(n, dtype=torch.int32, device=dev)
    jcnt = torch.empty(1, dtype=torch.int64, device=dev)
    qe.qe_filter(ctx, [fact["date"]], [(0, qe.LT, DATE_LT)], sel, cnt)
    nsel = int(cnt.item())

    def per_op():
        qe.qe_filter(ctx, [fact["date"]], [(0, qe.LT, DATE_LT)], sel, cnt, check=False)
        ht = qe.qe_join_build(ctx, dim["key"], dim["attr"], check=False)
        qe.qe_join_probe(ctx, ht, fact["fk"], sel, n=nsel, capacity=n, out_rows=rows, out_payload=attr,
                         out_count=jcnt, check=False)
        g = qe.qe_groupby(ctx, attr, [(qe.SUM, fact["price"], fact["qty"], True), (qe.COUNT, None, None),
                                      (qe.MIN, fact["price"], None, True), (qe.MAX, fact["price"], None, True)],
                          key_hi=fact["flag"], gather_hi=True, rows=rows, n=nsel, capacity=4096, check=False)
        ht.destroy()
        return g
    per_op()
    ctx.sync_status()
    ms = timed(per_op, it, stream)
    out["per_operator"] = {"ms": ms, "rows_per_s": n / (ms * 1e-3),
                           "note": "filter, build, probe, group-by as separate calls; selection vector and "
                                   "join output materialised in HBM; the filter count is read once beforehand"}
    # 25K-group variant: attr in [0, 8334)
    from paper_2506_09226_gb300 import datagen
    dim25 = datagen.star_dim(args.dim_rows, 8334, seed=1, device=dev)
    g25, gout25 = qe.alloc_groups(32768, 4, dev)
    desc25 = star_desc(qe, fact, dim25, 25002)
    fn = lambda: qe.qe_pipeline(ctx, desc25, 32768, check=False, out=(g25, gout25))  # noqa: E731
    fn()
    ms = timed(fn, it, stream)
    out["groups_25k"] = {"ms": ms, "rows_per_s": args.fact_rows / (ms * 1e-3), "ngroups": int(g25.ngroups.item()),
                         "hbm_frac": round((BYTES_FACT_ROW * args.fact_rows + 12 * args.dim_rows) /
                                           (ms * 1e-3) / 1e9 / peak, 4)}
    ctx.sync_status()
    del sel, rows, attr, dim25, g25, gout25
    torch.cuda.empty_cache()
    return out


SKEW_SWEEP = (0.01, 0.05, 0.10, 0.25, 0.50, 0.75, 0.90)


def run_skew(args, qe, ctx, dev, stream, peak, it):
    """Skewed, high-cardinality pipeline: 300M fact rows with Zipf(1.1) foreign
    keys over a 50M-row dimension, grouped on ~40M distinct int64 keys, with
    the selectivity swept over 1 .. 90 % through date < c and through a
    dictionary-code predicate code < K.  Groups this many take the
    partitioned group-by (count, scan, scatter of 24-byte rows into parts,
    split of every part into sub-parts, shared-memory aggregation of each
    sub-part).  hbm_frac counts the 28 bytes each fact row reads (fk, date,
    price, qty, int64 group key; code instead of date for the code sweep);
    part_bytes states the extra traffic of the partition round trips (the
    count pass reads the 8-byte key of every row; each survivor is written
    by the scatter, read and written by the split and read by the fold, 24
    bytes each time) and hbm_frac_with_partition counts them as well.  Also timed: the 50 % point through the direct HBM hash table
    (the path the partitioning replaces) and the group-by on 10^6
    dictionary codes."""
    from paper_2506_09226_gb300 import datagen
    n_fact = max(1, args.fact_rows // 2)
    n_dim = max(1, args.dim_rows * 5 // 2)
    t0 = time.time()
    dim = datagen.star_dim(n_dim, 1000, seed=3, device=dev)
    fact = datagen.star_fact(n_fact, n_dim, seed=3, device=dev, zipf_s=1.1, n_codes=1_000_000,
                             n_gkeys=max(1, n_fact * 2 // 15))
    log(f"skew workload generated in {time.time() - t0:.1f}s")
    cols = [fact[c] for c in ("fk", "date", "price", "qty", "gkey", "code")]
    aggs = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
    cap = max(1, n_fact * 2 // 15)
    groups, gout = qe.alloc_groups(cap, 4, dev)
    res = {"fact_rows": n_fact, "dim_rows": n_dim, "groups_pool": cap}
    phases = ("part_count", "part_scatter_rows", "part_split", "part_fold", "pipeline")

    def one(pred, key_col, capacity, sel_est):
        d = qe.pipeline_desc(cols, [pred], fk_col=0, dim_key=dim["key"], dim_payload=dim["attr"],
                             key_hi_col=-1, key_lo_col=key_col, aggs=aggs, expected_groups=capacity,
                             est_selectivity=sel_est)
        fn = lambda: qe.qe_pipeline(ctx, d, capacity, check=False, out=(groups, gout))  # noqa: E731
        fn()
        ctx.sync_status()
        ctx.profile(True)
        ctx.profile_reset()
        iters = max(3, it // 3)
        ms = timed(fn, iters, stream)
        kern = {}
        for ph in phases:
            c, tot = ctx.profile_read(ph)
            if c:
                kern[ph] = round(tot / c, 4)
        ctx.profile(False)
        ctx.sync_status()
        ng = int(groups.ngroups.item())
        return ms, kern, ng

    for colname, ci, span in (("date", 1, datagen.DATE_SPAN), ("code", 5, 1_000_000)):
        sweep = {}
        for sel in args.skew_sweep:
            c = int(round(sel * span))
            ms, kern, ng = one((ci, qe.LT, c), 4, cap, sel)
            nsurv = None
            if "part_count" in kern:
                nsurv = int((fact[colname] < c).sum().item())
            pb = (8 * n_fact + 96 * nsurv) if nsurv is not None else 0
            sweep[f"{int(round(sel * 100))}%"] = {
                "ms": ms, "rows_per_s": n_fact / (ms * 1e-3), "ngroups": ng,
                "hbm_frac": round(28 * n_fact / (ms * 1e-3) / 1e9 / peak, 4), "kernels_ms": kern,
                "part_bytes": pb,
                "hbm_frac_with_partition": round((28 * n_fact + pb) / (ms * 1e-3) / 1e9 / peak, 4)}
        res[f"sweep_{colname}"] = sweep
    # the autotuner's choice at 50 %: direct table or partitioned group-by
    # (fan-out 64 / 128 / 256 parts), dense or open-addressing join table
    from paper_2506_09226_gb300 import tune
    c50 = int(round(0.5 * datagen.DATE_SPAN))
    dt = qe.pipeline_desc(cols, [(1, qe.LT, c50)], fk_col=0, dim_key=dim["key"], dim_payload=dim["attr"],
                          key_hi_col=-1, key_lo_col=4, aggs=aggs, expected_groups=cap, est_selectivity=0.5)
    try:
        part, log2p, layout = tune.tune_group_placement(
            ctx, dt, lambda: qe.qe_pipeline(ctx, dt, cap, check=False, out=(groups, gout)), stream)
        qe.qe_pipeline(ctx, dt, cap, check=False, out=(groups, gout))
        ctx.sync_status()
        ms = timed(lambda: qe.qe_pipeline(ctx, dt, cap, check=False, out=(groups, gout)), max(3, it // 3), stream)
        res["autotuned_50%"] = {"ms": ms, "rows_per_s": n_fact / (ms * 1e-3), "ngroups": int(groups.ngroups.item()),
                                "hbm_frac": round(28 * n_fact / (ms * 1e-3) / 1e9 / peak, 4),
                                "choice": {"partitioned": part == 2, "parts_log2": log2p,
                                           "join_layout": "dense" if layout == qe.HT_DENSE else "open"}}
    finally:
        ctx.set_tuning("gb_partition", 0)
        ctx.set_tuning("gb_part_log2p", 0)
    # the direct HBM hash table at 50 %, for comparison
    ctx.set_tuning("gb_partition", 1)
    try:
        ms, kern, ng = one((1, qe.LT, int(round(0.5 * datagen.DATE_SPAN))), 4, cap, 0.5)
        res["direct_hbm_table_50%"] = {"ms": ms, "rows_per_s": n_fact / (ms * 1e-3), "ngroups": ng,
                                       "hbm_frac": round(28 * n_fact / (ms * 1e-3) / 1e9 / peak, 4)}
    finally:
        ctx.set_tuning("gb_partition", 0)
    # group-by on the 10^6 dictionary codes at 50 % (a hash table of ~84 MB)
    ms, kern, ng = one((1, qe.LT, int(round(0.5 * datagen.DATE_SPAN))), 5, 1_000_000, 0.5)
    res["codes_1m_groups_50%"] = {"ms": ms, "rows_per_s": n_fact / (ms * 1e-3), "ngroups": ng,
                                  "hbm_frac": round(24 * n_fact / (ms * 1e-3) / 1e9 / peak, 4), "kernels_ms": kern}
    ctx.sync_status()
    del dim, fact, cols, groups, gout
    torch.cuda.empty_cache()
    return res


def run_variants(args, qe, ctx, dev, stream, peak, it):
    """The operator variants beside the inner join, on the step's fact table
    (regenerated from its seed) and its filter date < DATE_LT (about half the
    rows).  Each entry gives the whole call's time and its algorithmic bytes
    over that time as a fraction of the HBM peak:
      pipeline_semi / pipeline_anti: filter + semi- / anti-join against a key
        set of half the dimension's keys + group-by flag (the set is built in
        the call): 21 B per fact row + 4 B per set key;
      single_table: filter + group-by flag, no join (fk_col = -1): 17 B per row;
      inner_probe: stand-alone probe of the dimension's dense table over the
        filter's selection vector: 4 B selection + 4 B key + 8 B per output;
      open_20m_* / open_50m_*: the same build and probe with the table in the
        open-addressing layout, for the 20M-row dimension and for a 50M-row
        one probed by a foreign key uniform over its keys: build 8 B in per
        row + 8 B per slot written; probe as inner_probe;
      semi_join / anti_join: stand-alone, over the filter's selection vector:
        4 B selection + 4 B key + 4 B per output position;
      multi_build / multi_probe: many-to-many join against a partsupp-shaped
        build side (4 rows per key, 4x the dimension's rows): build 12 B per
        row (key and payload in, payload placed); probe over the selection,
        every position matching 4 rows: 4 B selection + 4 B key + 8 B per pair;
      pair_build / pair_probe: join on (fk, a second key column) against unique
        pairs (4 per first key, 4x the dimension's rows): build 12 B in + 12 B
        out per row; probe 4 B selection + 8 B keys + 8 B per output, about
        4 positions in 5 matching."""
    from paper_2506_09226_gb300 import datagen
    nd, n = args.dim_rows, args.fact_rows
    t0 = time.time()
    dim = datagen.star_dim(nd, 1000, seed=1, device=dev)
    fact = datagen.star_fact(n, nd, seed=1, device=dev)
    log(f"variant workload generated in {time.time() - t0:.1f}s")
    cols = [fact[c] for c in COLS]
    aggs = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
    groups, gout = qe.alloc_groups(64, 4, dev)
    res = {}

    def entry(ms, units, nbytes, **kw):
        return {"ms": ms, "rows_per_s": units / (ms * 1e-3),
                "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4), **kw}

    def kernel_ms(fn, name):
        ctx.profile(True)
        ctx.profile_reset()
        ms = timed(fn, it, stream)
        c, tot = ctx.profile_read(name)
        ctx.profile(False)
        return ms, (tot / c if c else None)

    # semi- and anti-join pipelines, and the single-table aggregation
    half = dim["key"][: nd // 2].contiguous()
    for name, kind in (("pipeline_semi", qe.SEMI), ("pipeline_anti", qe.ANTI)):
        d = qe.pipeline_desc(cols, [(1, qe.LT, DATE_LT)], fk_col=0, dim_key=half, key_hi_col=-1, key_lo_col=4,
                             aggs=aggs, expected_groups=3, est_selectivity=DATE_LT / datagen.DATE_SPAN,
                             key_range=(None, (0, 2)), join_kind=kind)
        fn = lambda: qe.qe_pipeline(ctx, d, 64, check=False, out=(groups, gout))  # noqa: E731
        fn()
        ctx.sync_status()
        ms, kms = kernel_ms(fn, "pipeline")
        res[name] = entry(ms, n, BYTES_FACT_ROW * n + 4 * half.numel(), kernel_ms=kms,
                          kernel_hbm_frac=round(BYTES_FACT_ROW * n / (kms * 1e-3) / 1e9 / peak, 4) if kms else None,
                          ngroups=int(groups.ngroups.item()))
    d = qe.pipeline_desc(cols[1:], [(0, qe.LT, DATE_LT)], key_hi_col=-1, key_lo_col=3, aggs=[
        (qe.SUM, 1, 2), (qe.COUNT, -1, -1), (qe.MIN, 1, -1), (qe.MAX, 1, -1)], expected_groups=3,
        est_selectivity=DATE_LT / datagen.DATE_SPAN, key_range=(None, (0, 2)))
    fn = lambda: qe.qe_pipeline(ctx, d, 64, check=False, out=(groups, gout))  # noqa: E731
    fn()
    ctx.sync_status()
    ms, kms = kernel_ms(fn, "pipeline")
    res["single_table"] = entry(ms, n, 17 * n, kernel_ms=kms, ngroups=int(groups.ngroups.item()))
    del d

    # the filter's selection vector, shared by the stand-alone joins
    sel = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    qe.qe_filter(ctx, [fact["date"]], [(0, qe.LT, DATE_LT)], sel, cnt)
    nsel = int(cnt.item())
    out_rows = torch.empty(4 * nsel + 1, dtype=torch.int32, device=dev)
    out_pay = torch.empty(4 * nsel + 1, dtype=torch.int32, device=dev)
    ocnt = torch.empty(1, dtype=torch.int64, device=dev)

    # stand-alone inner probe against the dimension (unique keys)
    hd = qe.qe_join_build(ctx, dim["key"], dim["attr"])
    fn = lambda: qe.qe_join_probe(ctx, hd, fact["fk"], sel, n=nsel, capacity=nsel, out_rows=out_rows,  # noqa: E731
                                  out_payload=out_pay, out_count=ocnt, check=False)
    fn()
    ctx.sync_status()
    ms = timed(fn, it, stream)
    k = int(ocnt.item())
    res["inner_probe"] = entry(ms, nsel, 8 * nsel + 8 * k, outputs=k)
    hd.destroy()

    # open addressing at scale: the dimension's 20M keys, and 50M keys probed
    # by a foreign key uniform over them, in the open-addressing layout
    # (linear probing, 8-byte slots, CAS insert) instead of the dense array
    g50 = torch.Generator(device=dev)
    g50.manual_seed(50)
    for nk in (nd, nd * 5 // 2):
        dk = dim if nk == nd else datagen.star_dim(nk, 1000, seed=6, device=dev)
        pk = fact["fk"] if nk == nd else torch.randint(0, nk, (n,), generator=g50, device=dev, dtype=torch.int32)

        def obuild():
            qe.qe_join_build(ctx, dk["key"], dk["attr"], layout=qe.HT_OPEN, key_range=(0, nk - 1),
                             check=False).destroy()
        obuild()
        ctx.sync_status()
        bms = timed(obuild, it, stream)
        ho = qe.qe_join_build(ctx, dk["key"], dk["attr"], layout=qe.HT_OPEN, key_range=(0, nk - 1))
        fn = lambda: qe.qe_join_probe(ctx, ho, pk, sel, n=nsel, capacity=nsel, out_rows=out_rows,  # noqa: E731
                                      out_payload=out_pay, out_count=ocnt, check=False)
        fn()
        ctx.sync_status()
        ms = timed(fn, it, stream)
        k = int(ocnt.item())
        tag = f"open_{nk // 1_000_000}m"
        res[tag + "_build"] = entry(bms, nk, 8 * nk + 8 * ho.info().slots, slots=int(ho.info().slots))
        res[tag + "_probe"] = entry(ms, nsel, 8 * nsel + 8 * k, outputs=k)
        ho.destroy()
        del dk, pk

    # stand-alone semi- and anti-join
    hs = qe.qe_join_build_set(ctx, half)
    for name, anti in (("semi_join", False), ("anti_join", True)):
        fn = lambda: qe.qe_join_semi(ctx, hs, fact["fk"], sel, n=nsel, anti=anti, capacity=nsel,  # noqa: E731
                                     out_rows=out_rows, out_count=ocnt, check=False)
        fn()
        ctx.sync_status()
        ms = timed(fn, it, stream)
        k = int(ocnt.item())
        res[name] = entry(ms, nsel, 8 * nsel + 4 * k, outputs=k)
    hs.destroy()
    del half

    # many-to-many join
    md = datagen.multi_dim(nd, 4, 1000, seed=4, device=dev)
    nb = md["key"].numel()

    def mbuild():
        qe.qe_join_build_multi(ctx, md["key"], md["attr"], check=False).destroy()
    mbuild()
    ctx.sync_status()
    res["multi_build"] = entry(timed(mbuild, it, stream), nb, 12 * nb)
    hm = qe.qe_join_build_multi(ctx, md["key"], md["attr"])
    fn = lambda: qe.qe_join_probe_multi(ctx, hm, fact["fk"], sel, n=nsel, capacity=out_rows.numel(),  # noqa: E731
                                        out_rows=out_rows, out_payload=out_pay, out_count=ocnt, check=False)
    fn()
    ctx.sync_status()
    ms = timed(fn, it, stream)
    k = int(ocnt.item())
    res["multi_probe"] = entry(ms, nsel, 8 * nsel + 8 * k, outputs=k)
    hm.destroy()
    del md

    # pair-key join
    pd = datagen.pair_dim(nd, 4, seed=5, device=dev)
    plo = datagen.pair_probe_lo(fact["fk"], pd["off"], 5, seed=5)
    nb = pd["hi"].numel()

    def pbuild():
        qe.qe_join_build_pair(ctx, pd["hi"], pd["lo"], pd["payload"], check=False).destroy()
    pbuild()
    ctx.sync_status()
    res["pair_build"] = entry(timed(pbuild, it, stream), nb, 24 * nb)
    hp = qe.qe_join_build_pair(ctx, pd["hi"], pd["lo"], pd["payload"])
    fn = lambda: qe.qe_join_probe_pair(ctx, hp, fact["fk"], plo, sel, n=nsel, capacity=nsel,  # noqa: E731
                                       out_rows=out_rows, out_payload=out_pay, out_count=ocnt, check=False)
    fn()
    ctx.sync_status()
    ms = timed(fn, it, stream)
    k = int(ocnt.item())
    res["pair_probe"] = entry(ms, nsel, 12 * nsel + 8 * k, outputs=k)
    hp.destroy()
    ctx.sync_status()
    res["workload"] = (f"{n} fact rows, filter date < {DATE_LT} ({nsel} selected); key set of {nd // 2} keys; "
                       f"build sides of {4 * nd} rows (4 per key)")
    del pd, plo, sel, out_rows, out_pay, dim, fact, cols, groups, gout
    torch.cuda.empty_cache()
    return res


def run_e2e(args, qe, ctx, fact, dim, key, pay, okeys, opay, offs, groups, gout, dev, stream):
    """Same step through the public API with inputs copied from pinned host
    memory and the results read back, every step."""
    t0 = time.time()
    hfact = {c: torch.empty(fact[c].shape, dtype=fact[c].dtype, pin_memory=True) for c in COLS}
    hdim = {c: torch.empty(dim[c].shape, dtype=dim[c].dtype, pin_memory=True) for c in ("key", "attr")}
    hkey = torch.empty(key.shape, dtype=key.dtype, pin_memory=True)
    hpay = torch.empty(pay.shape, dtype=pay.dtype, pin_memory=True)
    for c in COLS:
        hfact[c].copy_(fact[c])
    for c in ("key", "attr"):
        hdim[c].copy_(dim[c])
    hkey.copy_(key)
    hpay.copy_(pay)
    rk = torch.empty(4096, dtype=torch.int64, pin_memory=True)
    ra = [torch.empty(4096, dtype=torch.int64, pin_memory=True) for _ in range(4)]
    rn = torch.empty(1, dtype=torch.int64, pin_memory=True)
    ro = torch.empty(offs.shape, dtype=torch.int64, pin_memory=True)
    log(f"pinned host inputs ready in {time.time() - t0:.1f}s")
    h2d = sum(t.numel() * t.element_size() for t in list(hfact.values()) + list(hdim.values()) + [hkey, hpay])
    d2h = (rk.numel() + 4 * 4096 + 1 + ro.numel()) * 8
    desc = star_desc(qe, fact, dim, 3000)

    # The host link (about 211 GB/s on this GB300, for copy engines and for
    # kernels reading mapped host memory alike) bounds this step, so the
    # copies run back to back on their own stream, pairs first: the
    # partition runs while the fact table is still arriving.
    cs = torch.cuda.Stream()
    pairs_in, fact_in = torch.cuda.Event(), torch.cuda.Event()

    def e2e_step():
        cur = torch.cuda.current_stream()
        cs.wait_stream(cur)                    # the previous step is done with the buffers
        with torch.cuda.stream(cs):
            key.copy_(hkey, non_blocking=True)
            pay.copy_(hpay, non_blocking=True)
            pairs_in.record(cs)
            for c in COLS:
                fact[c].copy_(hfact[c], non_blocking=True)
            for c in ("key", "attr"):
                dim[c].copy_(hdim[c], non_blocking=True)
            fact_in.record(cs)
        cur.wait_event(pairs_in)
        qe.qe_partition(ctx, key, [pay], args.log2f, qe.PART_HASH, 0, okeys, [opay], offs, check=False)
        cur.wait_event(fact_in)
        qe.qe_pipeline(ctx, desc, 4096, check=False, out=(groups, gout))
        rk.copy_(groups.keys, non_blocking=True)
        for a, b in zip(ra, groups.aggs):
            a.copy_(b, non_blocking=True)
        rn.copy_(groups.ngroups, non_blocking=True)
        ro.copy_(offs, non_blocking=True)

    e2e_step()
    it = max(2, min(args.steps, 5))
    ms = timed(e2e_step, it, stream)
    ctx.sync_status()
    v = (args.fact_rows + args.pairs) / (ms * 1e-3)
    del hfact, hdim, hkey, hpay
    return {"value": v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms,
            "steps": it, "h2d_gbs": round(h2d / (ms * 1e-3) / 1e9, 1)}


def run_forms(args, qe, ctx, dev, stream, fact, dim, peak):
    from paper_2506_09226_gb300 import batch as B
    out = {}
    if "batch" in args.forms:
        out["batch"] = B.bench_batch(ctx, args.batch_count, dev, stream, peak, log=log)
        # join kinds other than the inner join, in one batch
        out["batch"]["mixed_kinds"] = B.bench_batch_kinds(ctx, 600, dev, stream, peak)
    if "serve" in args.forms:
        from paper_2506_09226_gb300 import serve as S
        out["serve"] = S.bench_serve(ctx, dev, stream, peak, duration_s=args.serve_seconds, log=log,
                                     scale=args.serve_scale)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["qe", "reference"], default="qe")
    ap.add_argument("--fact-rows", type=int, default=600_000_000)
    ap.add_argument("--dim-rows", type=int, default=20_000_000)
    ap.add_argument("--pairs", type=int, default=600_000_000)
    ap.add_argument("--log2f", type=int, default=10)
    ap.add_argument("--forms", default="extras,variants,batch,serve")
    ap.add_argument("--batch-count", type=int, default=10_000)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-scale", type=float, default=1.0)
    ap.add_argument("--ref-sample", type=int, default=2_000_000,
                    help="fact rows (and pairs) per reference-arm step")
    ap.add_argument("--cpu-sample", type=int, default=32_000_000,
                    help="fact rows (and pairs) of the cpu_baseline sample")
    ap.add_argument("--skew-sweep", type=lambda v: tuple(float(x) for x in v.split(",")), default=SKEW_SWEEP,
                    help="selectivities of the skewed pipeline's sweeps (comma-separated)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "qe":
        log("warmup raised to 3")
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_qe(args)


if __name__ == "__main__":
    sys.exit(main())
