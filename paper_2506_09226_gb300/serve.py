"""Served form: continuous batching of star pipelines over resident tables.

Requests (a row range of one resident fact table, a date bound) arrive over
time.  The server admits a request when an output slot and its share of the
HBM budget are free, folds every admitted request that has not started into
the next round, and runs the round as one batched launch (qe_batch_*) on the
next free stream of a small pool, so rounds overlap on the device while new
requests keep arriving.  Join tables are built once and stay resident; each
request joins its shape's table.  A request's latency runs from its arrival
to the moment the host sees its round's completion event.

The same trace can be replayed serially, one request at a time in arrival
order, either as separate operator calls or as one fused call each.
"""
from __future__ import annotations

import collections
import contextlib
import gc
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import datagen, qe

STAR_COLS = ("fk", "date", "price", "qty", "flag")
STAR_AGGS = [(qe.SUM, 2, 3), (qe.COUNT, -1, -1), (qe.MIN, 2, -1), (qe.MAX, 2, -1)]
CAPACITY = 3072           # output groups per request (3 flags x up to 1000 attributes)
REQ_BYTES = 560_000       # HBM a request holds while in flight: output slot + batch tables
ROW_CAP = 100_000_000     # fact rows per batched round


def percentile(xs, p: float) -> float:
    """Nearest-rank percentile (p in [0, 100]) of a non-empty sequence."""
    s = sorted(xs)
    k = max(1, math.ceil(p / 100.0 * len(s)))
    return float(s[k - 1])


class Admission:
    """HBM-budget and slot accounting of in-flight requests."""

    def __init__(self, budget_bytes: int, slots: int):
        self.budget, self.slots = budget_bytes, slots
        self.used, self.busy = 0, 0
        self.free_slots = collections.deque(range(slots))   # FIFO: least recently used slot first
        self.rejected = 0

    def try_admit(self, cost: int):
        """A slot id, or None when the budget or the slots are exhausted."""
        if not self.free_slots or self.used + cost > self.budget:
            return None
        self.used += cost
        self.busy += 1
        return self.free_slots.popleft()

    def release(self, slot: int, cost: int):
        self.used -= cost
        self.busy -= 1
        self.free_slots.append(slot)


@dataclass
class Request:
    rid: int
    arrival: float
    shape: int
    offset: int
    n: int
    date_hi: int
    slot: int = -1
    admitted: float = -1.0
    done: float = -1.0
    cancelled: bool = False


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    rows: int = 0
    makespan_s: float = 0.0
    rounds: int = 0
    max_inflight: int = 0
    max_round: int = 0
    cancelled: int = 0

    def summary(self) -> dict:
        lat = self.latencies_ms or [0.0]
        return {"requests": len(self.latencies_ms), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                "mean_ms": float(np.mean(lat)), "rows_per_s": self.rows / max(self.makespan_s, 1e-9),
                "makespan_s": self.makespan_s, "rounds": self.rounds, "max_inflight": self.max_inflight,
                "max_round": self.max_round, "cancelled": self.cancelled}


def serve_loop(trace, executor, admission: Admission, max_round: int = 4096, clock=time.perf_counter,
               idle_sleep: float = 20e-6, row_cap: int | None = None, cancel_at: dict | None = None) -> ServeStats:
    """Continuous batching over `trace` (Arrival list sorted by t).

    A round takes the oldest admitted requests until it holds max_round of
    them or row_cap fact rows (a request larger than row_cap goes alone), so
    rounds stay short and small requests are not held behind a large one.
    executor.launch(reqs) -> handle with .done() and .close(); executor.cost(req)
    is the request's HBM share.  Works with any clock/executor (tests use fakes).

    cancel_at maps a request id to the time (seconds after the start) at
    which its client withdraws it.  A request cancelled before admission is
    dropped; one admitted but not launched gives its output slot and HBM
    share back at once, so a waiting request can take them; one whose round
    is already on the device keeps them until that round completes (kernels
    are never interrupted) and its result is discarded.  Cancelled requests
    count in ServeStats.cancelled, not in the latencies or rows."""
    reqs = [Request(i, a.t, a.shape, a.offset, a.n, a.date_hi) for i, a in enumerate(trace)]
    pending = collections.deque(reqs)
    waiting = collections.deque()
    ready = []
    inflight = []          # (handle, [requests])
    cancels = sorted(((t, rid) for rid, t in (cancel_at or {}).items()), reverse=True)
    st = ServeStats()
    t0 = clock()
    while pending or waiting or ready or inflight:
        now = clock() - t0
        while pending and pending[0].arrival <= now:
            waiting.append(pending.popleft())
        while cancels and cancels[-1][0] <= now:
            r = reqs[cancels.pop()[1]]
            if r.cancelled or r.done >= 0:
                continue
            r.cancelled = True
            st.cancelled += 1
            if r in ready:                 # admitted, not launched: give the slot back now
                ready.remove(r)
                admission.release(r.slot, executor.cost(r))
            elif r in waiting:
                waiting.remove(r)
            elif r in pending:
                pending.remove(r)
        for h, rs in list(inflight):
            if h.done():
                t = clock() - t0
                for r in rs:
                    r.done = t
                    if not r.cancelled:
                        st.latencies_ms.append((t - r.arrival) * 1e3)
                        st.rows += r.n
                    admission.release(r.slot, executor.cost(r))
                h.close()
                inflight.remove((h, rs))
        while waiting:
            slot = admission.try_admit(executor.cost(waiting[0]))
            if slot is None:
                break
            r = waiting.popleft()
            r.slot, r.admitted = slot, now
            ready.append(r)
        st.max_inflight = max(st.max_inflight, admission.busy)
        if ready and executor.can_launch():
            k, rows = 0, 0
            while k < len(ready) and k < max_round and (k == 0 or row_cap is None or rows + ready[k].n <= row_cap):
                rows += ready[k].n
                k += 1
            batch, ready = ready[:k], ready[k:]
            inflight.append((executor.launch(batch), batch))
            st.rounds += 1
            st.max_round = max(st.max_round, len(batch))
            continue
        if not (pending and pending[0].arrival <= clock() - t0):
            if idle_sleep:
                time.sleep(idle_sleep)
    st.makespan_s = clock() - t0
    return st


class ResidentTables:
    """Fact and dimension tables of each request shape, with their join
    tables built once and kept on the device."""

    def __init__(self, ctx, shapes, device, log=print):
        self.ctx, self.shapes, self.device = ctx, shapes, device
        self.fact, self.dim, self.ht, self.rows, self.key_range = [], [], [], [], []
        for i, sh in enumerate(shapes):
            t0 = time.time()
            d = datagen.star_dim(sh["n_dim"], sh["n_attr"], seed=50 + i, device=device)
            f = datagen.star_fact(sh["n_fact"], sh["n_dim"], seed=50 + i, device=device, zipf_s=sh.get("zipf"))
            torch.cuda.synchronize()
            self.fact.append(f)
            self.dim.append(d)
            self.ht.append(qe.qe_join_build(ctx, d["key"], d["attr"]))
            self.rows.append(sh["n_fact"])
            self.key_range.append(((0, 2), (0, sh["n_attr"] - 1)))
            log(f"resident shape {i}: {sh} in {time.time() - t0:.1f}s")

    def bytes(self) -> int:
        tot = 0
        for f, d in zip(self.fact, self.dim):
            tot += sum(t.numel() * t.element_size() for t in f.values())
            tot += sum(t.numel() * t.element_size() for t in d.values())
        return tot + sum(h.info().bytes for h in self.ht)

    def desc(self, r: Request):
        f = self.fact[r.shape]
        cols = [f[c][r.offset:r.offset + r.n] for c in STAR_COLS]
        return qe.pipeline_desc(cols, [(1, qe.LT, r.date_hi)], fk_col=0, ht=self.ht[r.shape], key_hi_col=4,
                                key_lo_col=qe.JOIN_PAYLOAD, aggs=STAR_AGGS, key_range=self.key_range[r.shape],
                                expected_groups=3000)

    def close(self):
        for h in self.ht:
            h.destroy()


class OutputSlots:
    """Per-request group outputs, one slot per admitted request."""

    def __init__(self, slots: int, device):
        import ctypes
        self.keys = torch.empty((slots, CAPACITY), dtype=torch.int64, device=device)
        self.aggs = torch.empty((4, slots, CAPACITY), dtype=torch.int64, device=device)
        self.ngroups = torch.zeros(slots, dtype=torch.int64, device=device)
        ks, as_, ns = self.keys.data_ptr(), self.aggs.data_ptr(), self.ngroups.data_ptr()
        row, plane = CAPACITY * 8, slots * CAPACITY * 8
        self.structs = [qe.qe_groups_out(CAPACITY, ks + i * row,
                                         (ctypes.c_void_p * qe.MAX_AGGS)(*[as_ + a * plane + i * row
                                                                           for a in range(4)]), ns + i * 8)
                        for i in range(slots)]

    def groups(self, slot: int):
        n = min(int(self.ngroups[slot].item()), CAPACITY)
        k = self.keys[slot, :n].cpu().numpy()
        o = np.argsort(k, kind="stable")
        return k[o], [self.aggs[a, slot, :n].cpu().numpy()[o] for a in range(4)]


class _Round:
    def __init__(self, batch, event, stream, streams_free):
        self.batch, self.event, self.stream, self.free = batch, event, stream, streams_free

    def done(self) -> bool:
        return self.event.query()

    def close(self):
        self.batch.destroy(self.stream)
        self.free.append(self.stream)


class _Single:
    """A one-request round run as a fused single-pipeline launch."""

    def __init__(self, event, stream, streams_free):
        self.event, self.stream, self.free = event, stream, streams_free

    def done(self) -> bool:
        return self.event.query()

    def close(self):
        self.free.append(self.stream)


class BatchExecutor:
    """Runs a round of requests as one batched launch on a free stream; a
    round of one request of at least `single_rows` rows runs as a fused
    single-pipeline launch instead."""

    def __init__(self, ctx, tables: ResidentTables, outs: OutputSlots, n_streams: int = 4,
                 opts: qe.qe_batch_opts | None = None, on_round=None, single_rows: int = 50_000_000):
        self.ctx, self.tables, self.outs = ctx, tables, outs
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.free = list(self.streams)
        self.opts = opts if opts is not None else qe.qe_batch_opts(0, 1 << 16, 0, 0)
        self.on_round = on_round
        self.single_rows = single_rows

    def cost(self, r: Request) -> int:
        return REQ_BYTES

    def can_launch(self) -> bool:
        return bool(self.free)

    def launch(self, reqs):
        s = self.free.pop()
        if self.on_round:
            self.on_round(reqs)
        if len(reqs) == 1 and reqs[0].n >= self.single_rows:
            r = reqs[0]
            qe.qe_pipeline(self.ctx, self.tables.desc(r), CAPACITY, stream=s, check=False,
                           out=(None, self.outs.structs[r.slot]))
            ev = torch.cuda.Event()
            ev.record(s)
            return _Single(ev, s, self.free)
        descs = [self.tables.desc(r) for r in reqs]
        outs = [self.outs.structs[r.slot] for r in reqs]
        b = qe.Batch(self.ctx, descs, outs, self.opts, s)
        b.launch(s)
        ev = torch.cuda.Event()
        ev.record(s)
        return _Round(b, ev, s, self.free)


def serial_replay(trace, run_one, clock=time.perf_counter) -> ServeStats:
    """One request at a time, in arrival order; run_one(req) runs it to completion."""
    st = ServeStats()
    t0 = clock()
    for i, a in enumerate(trace):
        now = clock() - t0
        if a.t > now:
            time.sleep(a.t - now)
        r = Request(i, a.t, a.shape, a.offset, a.n, a.date_hi)
        run_one(r)
        t = clock() - t0
        st.latencies_ms.append((t - a.t) * 1e3)
        st.rows += a.n
        st.rounds += 1
    st.makespan_s = clock() - t0
    return st


def per_operator_request(ctx, tables: ResidentTables, r: Request, scratch: dict, stream=None):
    """One request as separate operator calls, sizes read back between them."""
    f = tables.fact[r.shape]
    a, n = r.offset, r.n
    sel, cnt, rows, attr, jc = scratch["sel"], scratch["cnt"], scratch["rows"], scratch["attr"], scratch["jc"]
    qe.qe_filter(ctx, [f["date"][a:a + n]], [(0, qe.LT, r.date_hi)], sel, cnt, stream=stream, check=False)
    nsel = int(cnt.item())
    qe.qe_join_probe(ctx, tables.ht[r.shape], f["fk"][a:a + n], sel, n=nsel, capacity=sel.numel(), out_rows=rows,
                     out_payload=attr, out_count=jc, stream=stream, check=False)
    nj = int(jc.item())
    g = qe.qe_groupby(ctx, attr, [(qe.SUM, f["price"][a:a + n], f["qty"][a:a + n], True), (qe.COUNT, None, None),
                                  (qe.MIN, f["price"][a:a + n], None, True), (qe.MAX, f["price"][a:a + n], None, True)],
                      key_hi=f["flag"][a:a + n], gather_hi=True, rows=rows, n=nj, capacity=CAPACITY,
                      stream=stream, check=False)
    torch.cuda.current_stream().synchronize()
    return g


# shapes of the resident tables: configuration 0, 1 and 2 schemas
def default_shapes(scale: float = 1.0):
    n = int(1.9e9 * scale)
    return [{"n_fact": n, "n_dim": 100_000, "n_attr": 25},
            {"n_fact": n, "n_dim": 20_000_000, "n_attr": 1000},
            {"n_fact": n, "n_dim": 50_000_000, "n_attr": 1000, "zipf": 1.1}]


@contextlib.contextmanager
def gc_paused():
    """The cyclic garbage collector frozen and off for a latency-timed loop,
    so that a full collection of the process's heap (tens of milliseconds
    with PyTorch loaded) cannot land inside it; per-round objects are still
    freed by reference counting."""
    gc.collect()
    gc.freeze()
    gc.disable()
    try:
        yield
    finally:
        gc.enable()
        gc.unfreeze()


def bench_serve(ctx, device, stream, peak_gbs: float, duration_s: float = 10.0, rate: float = 2000.0,
                scale: float = 1.0, serial_s: float = 1.0, log=print, seed: int = 5,
                sat_rates=(1000.0, 2000.0, 4000.0, 8000.0), sat_seconds: float = 1.0) -> dict:
    """Served form on a Poisson trace against serial per-request replays, then
    a saturation sweep over rising arrival rates (each a trace of
    sat_seconds) against serial fused replay.  Every timed loop, served or
    serial, runs with the garbage collector paused (gc_paused)."""
    torch.cuda.empty_cache()
    tables = ResidentTables(ctx, default_shapes(scale), device, log=log)
    resident = tables.bytes()
    trace = datagen.poisson_trace(duration_s, rate, tables.rows, seed=seed, n_lo=1e4,
                                  n_hi=min(5e8, min(tables.rows)))
    slots = 4096
    outs = OutputSlots(slots, device)
    adm = Admission(budget_bytes=slots * REQ_BYTES, slots=slots)
    ex = BatchExecutor(ctx, tables, outs, n_streams=4)
    # warm-up round (module load, first launch)
    warm = serve_loop(trace[:8], ex, Admission(slots * REQ_BYTES, slots), row_cap=ROW_CAP)
    torch.cuda.synchronize()
    log(f"serve: {len(trace)} requests over {duration_s}s, resident {resident / 1e9:.1f} GB")
    with gc_paused():
        st = serve_loop(trace, ex, adm, row_cap=ROW_CAP)
    ctx.sync_status()
    served = st.summary()
    del warm
    # serial replays on the first serial_s seconds of the same trace
    prefix = [a for a in trace if a.t < serial_s]
    with gc_paused():
        st_pre = serve_loop(prefix, ex, Admission(slots * REQ_BYTES, slots), row_cap=ROW_CAP).summary()
    mx = max(a.n for a in prefix) if prefix else 1
    scratch = {"sel": torch.empty(mx, dtype=torch.int32, device=device),
               "cnt": torch.empty(1, dtype=torch.int64, device=device),
               "rows": torch.empty(mx, dtype=torch.int32, device=device),
               "attr": torch.empty(mx, dtype=torch.int32, device=device),
               "jc": torch.empty(1, dtype=torch.int64, device=device)}
    with gc_paused():
        per_op = serial_replay(prefix, lambda r: per_operator_request(ctx, tables, r, scratch)).summary()
    g1, o1 = qe.alloc_groups(CAPACITY, 4, device)

    def fused(r):
        qe.qe_pipeline(ctx, tables.desc(r), CAPACITY, check=False, out=(g1, o1))
        torch.cuda.current_stream().synchronize()
    with gc_paused():
        fused_serial = serial_replay(prefix, fused).summary()
    ctx.sync_status()
    # saturation sweep: the arrival rate rising past what serial fused
    # execution sustains, served (continuous batching) against serial fused
    # replay of the same trace
    sweep = {}
    for lam in sat_rates:
        tr = datagen.poisson_trace(sat_seconds, lam, tables.rows, seed=seed + int(lam), n_lo=1e4,
                                   n_hi=min(5e8, min(tables.rows)))
        with gc_paused():
            sv = serve_loop(tr, ex, Admission(slots * REQ_BYTES, slots), row_cap=ROW_CAP).summary()
        with gc_paused():
            sf = serial_replay(tr, fused).summary()
        ctx.sync_status()
        sweep[str(int(lam))] = {"requests": len(tr), "served": {k: sv[k] for k in ("p50_ms", "p99_ms", "rows_per_s")},
                                "serial_fused": {k: sf[k] for k in ("p50_ms", "p99_ms", "rows_per_s")}}
        log(f"saturation {lam:.0f} req/s: served p99 {sv['p99_ms']:.1f} ms, serial fused p99 {sf['p99_ms']:.1f} ms")
    tables.close()
    del scratch, outs
    torch.cuda.empty_cache()
    return {"arrival_rate_per_s": rate, "duration_s": duration_s, "resident_gb": round(resident / 1e9, 1),
            "served": served,
            "prefix_s": serial_s, "served_prefix": st_pre, "serial_per_operator_prefix": per_op,
            "serial_fused_prefix": fused_serial,
            "saturation": {"trace_s": sat_seconds, "rates": sweep},
            "p99_speedup_vs_per_operator": per_op["p99_ms"] / max(st_pre["p99_ms"], 1e-9),
            "throughput_vs_per_operator": st_pre["rows_per_s"] / max(per_op["rows_per_s"], 1e-9)}
