"""Python binding of libqe (include/qe.h): argument marshalling only.

Every entry point of the C ABI is exposed under its own name (qe_create,
qe_filter, qe_partition, qe_join_build, qe_join_build_set,
qe_join_build_multi, qe_join_build_pair, qe_join_probe, qe_join_semi,
qe_join_probe_multi, qe_join_probe_pair, qe_groupby, qe_pipeline, qe_batch_*) and takes torch CUDA tensors, whose
device pointers are passed straight to the library; torch provides device
memory and streams only.  The exchange planner (qe_plan_*) is host
arithmetic and takes plain numbers and numpy arrays.  All operator work runs
in the library's CUDA kernels.  Importing this module does not load the
library; the first call does, and raises QeError when libqe.so has not been
built or no sm_103a device is present (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_LIB_DIR = os.path.dirname(os.path.abspath(__file__))
# QE_LIB=checked selects the bounds-checked build (libqe_checked.so)
_LIB_PATH = os.path.join(_LIB_DIR, "libqe_checked.so" if os.environ.get("QE_LIB") == "checked" else "libqe.so")

# qe_status
OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_OOM, ERR_DUPLICATE_KEY, ERR_RESERVED_KEY, ERR_TIMEOUT, ERR_CUDA, \
    ERR_NO_DEVICE, ERR_DEVICE_CHECK = range(10)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CAPACITY", 3: "OOM", 4: "DUPLICATE_KEY", 5: "RESERVED_KEY",
                6: "TIMEOUT", 7: "CUDA", 8: "NO_DEVICE", 9: "DEVICE_CHECK"}
# qe_type
I8, I32, I64 = 1, 4, 8
# qe_cmp
LT, LE, GT, GE, EQ, NE, BETWEEN = range(7)
# qe_agg_op
SUM, COUNT, MIN, MAX = range(4)
# partition modes, table layouts, group placements
PART_HASH, PART_RADIX = 0, 1
HT_AUTO, HT_DENSE, HT_OPEN = 0, 1, 2
GB_AUTO, GB_SMEM, GB_HBM = 0, 1, 2
JOIN_PAYLOAD = -2
# qe_join_kind
INNER, SEMI, ANTI = 0, 1, 2
MAX_COLS, MAX_PREDS, MAX_AGGS = 8, 4, 4

_TYPE_OF = {torch.int8: I8, torch.int32: I32, torch.int64: I64}


class QeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class qe_col(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("type", ctypes.c_int32), ("gather", ctypes.c_int32)]


class qe_pred(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("op", ctypes.c_int32), ("lo", ctypes.c_int64), ("hi", ctypes.c_int64)]


class qe_groups_out(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("keys", ctypes.c_void_p),
                ("aggs", ctypes.c_void_p * MAX_AGGS), ("ngroups", ctypes.c_void_p),
                ("avg", ctypes.c_void_p * MAX_AGGS)]


class qe_build_opts(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int32), ("have_range", ctypes.c_int32),
                ("key_min", ctypes.c_int32), ("key_max", ctypes.c_int32)]


class qe_ht_info(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int32), ("full", ctypes.c_int32), ("nkeys", ctypes.c_int64),
                ("slots", ctypes.c_int64), ("bytes", ctypes.c_int64), ("key_min", ctypes.c_int32),
                ("key_max", ctypes.c_int32), ("have_payload_range", ctypes.c_int32),
                ("payload_min", ctypes.c_int32), ("payload_max", ctypes.c_int32), ("key_set", ctypes.c_int32)]


class qe_agg(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("pad", ctypes.c_int32), ("a", qe_col), ("b", qe_col)]


class qe_agg_spec(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("pad", ctypes.c_int32)]


class qe_pipeline_desc(ctypes.Structure):
    _fields_ = [("n_fact", ctypes.c_int64), ("fact", qe_col * MAX_COLS), ("n_fact_cols", ctypes.c_int32),
                ("n_preds", ctypes.c_int32), ("preds", qe_pred * MAX_PREDS), ("fk_col", ctypes.c_int32),
                ("key_hi_col", ctypes.c_int32), ("key_lo_col", ctypes.c_int32), ("n_aggs", ctypes.c_int32),
                ("aggs", qe_agg_spec * MAX_AGGS), ("dim_key", ctypes.c_void_p), ("dim_payload", ctypes.c_void_p),
                ("n_dim", ctypes.c_int64), ("ht", ctypes.c_void_p), ("build", qe_build_opts),
                ("expected_groups", ctypes.c_int64), ("est_selectivity", ctypes.c_double),
                ("have_key_range", ctypes.c_int32), ("join_kind", ctypes.c_int32), ("key_hi_min", ctypes.c_int64),
                ("key_hi_max", ctypes.c_int64), ("key_lo_min", ctypes.c_int64), ("key_lo_max", ctypes.c_int64)]


class qe_batch_opts(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("smem_slots", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("build_ahead_bytes", ctypes.c_int64)]


# exchange planner (include/qe_plan.h)
EXCH_BROADCAST, EXCH_SHUFFLE = 0, 1
JOIN_LOCAL, JOIN_BROADCAST_R, JOIN_BROADCAST_S, JOIN_SHUFFLE_BOTH = range(4)


class qe_link(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("c", ctypes.c_double)]


class qe_cluster(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("V", ctypes.c_int32), ("bcast_net", qe_link), ("bcast_gpu", qe_link),
                ("shuf_net", qe_link), ("shuf_gpu", qe_link)]


_DP = ctypes.POINTER(ctypes.c_double)

_lib = None
_SIGS = {
    "qe_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]),
    "qe_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "qe_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "qe_sync_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "qe_bytes_in_use": (ctypes.c_size_t, [ctypes.c_void_p]),
    "qe_debug_fail_alloc": (None, [ctypes.c_void_p, ctypes.c_int]),
    "qe_debug_set_spin_limit": (None, [ctypes.c_void_p, ctypes.c_int64]),
    "qe_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "qe_build_checked": (ctypes.c_int, []),
    "qe_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int64]),
    "qe_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "qe_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double)]),
    "qe_profile_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "qe_filter": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qe_col), ctypes.c_int, ctypes.POINTER(qe_pred),
                                 ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "qe_filter_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qe_col), ctypes.c_int,
                                         ctypes.POINTER(qe_pred), ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "qe_partition": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(qe_col), ctypes.c_int,
                                    ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p]),
    "qe_join_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.POINTER(qe_build_opts), ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.c_void_p]),
    "qe_join_probe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "qe_join_build_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.POINTER(qe_build_opts), ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.c_void_p]),
    "qe_join_semi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "qe_join_build_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.POINTER(qe_build_opts), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.c_void_p]),
    "qe_join_probe_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "qe_join_build_pair": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "qe_join_probe_pair": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "qe_join_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qe_ht_info)]),
    "qe_join_destroy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qe_groupby": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, qe_col, qe_col,
                                  ctypes.POINTER(qe_agg), ctypes.c_int, ctypes.c_int, ctypes.POINTER(qe_groups_out),
                                  ctypes.c_void_p]),
    "qe_pipeline": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qe_pipeline_desc),
                                   ctypes.POINTER(qe_groups_out), ctypes.c_void_p]),
    "qe_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qe_pipeline_desc),
                                       ctypes.POINTER(qe_groups_out), ctypes.c_int, ctypes.POINTER(qe_batch_opts),
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "qe_batch_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qe_batch_destroy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qe_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qe_pipeline_desc),
                                    ctypes.POINTER(qe_groups_out), ctypes.c_int, ctypes.POINTER(qe_batch_opts),
                                    ctypes.c_void_p]),
    "qe_plan_exchange_time": (ctypes.c_int, [ctypes.POINTER(qe_cluster), ctypes.c_int32, ctypes.c_double, _DP]),
    "qe_plan_shuffle_skew": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _DP, ctypes.c_double, _DP, _DP, _DP]),
    "qe_plan_join": (ctypes.c_int, [ctypes.POINTER(qe_cluster), ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                    _DP, _DP, ctypes.POINTER(ctypes.c_int32), _DP, _DP]),
    "qe_plan_fit_link": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _DP, _DP, ctypes.c_int64,
                                        ctypes.POINTER(qe_link)]),
    "qe_plan_skew_gradient": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_double, _DP]),
    "qe_plan_last_error": (ctypes.c_char_p, []),
}

EXPORTED = sorted(_SIGS)


def load_library(path: str = _LIB_PATH) -> ctypes.CDLL:
    """Load libqe.so and declare its signatures (no device needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise QeError(ERR_NO_DEVICE, f"libqe.so not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name, None)
        if f is None:
            continue
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def col(t: torch.Tensor, gather: bool = False) -> qe_col:
    if t.dtype not in _TYPE_OF:
        raise QeError(ERR_INVALID_ARG, f"unsupported column dtype {t.dtype}")
    if not t.is_cuda or not t.is_contiguous():
        raise QeError(ERR_INVALID_ARG, "columns must be contiguous CUDA tensors")
    return qe_col(t.data_ptr(), _TYPE_OF[t.dtype], int(gather))


class Context:
    """Owns a qe_ctx.  Methods raise QeError on any non-OK status."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load_library()
        self.device = device
        h = ctypes.c_void_p()
        st = self.lib.qe_create(ctypes.byref(h), device, hbm_budget_bytes)
        if st != OK:
            raise QeError(st, "qe_create failed (needs an sm_103a GPU)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.qe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int):
        if st != OK:
            raise QeError(st, self.lib.qe_last_error(self.h).decode())

    def sync_status(self, stream=None) -> int:
        req = ctypes.c_int64(0)
        st = self.lib.qe_sync_status(self.h, _stream(stream), ctypes.byref(req))
        if st != OK:
            e = QeError(st, self.lib.qe_last_error(self.h).decode())
            e.required = req.value
            raise e
        return req.value

    def bytes_in_use(self) -> int:
        return int(self.lib.qe_bytes_in_use(self.h))

    def set_tuning(self, name: str, value: int):
        self.check(self.lib.qe_set_tuning(self.h, name.encode(), int(value)))

    def launch_count(self) -> int:
        return int(self.lib.qe_launch_count(self.h))

    def profile(self, on: bool = True):
        self.check(self.lib.qe_profile_enable(self.h, int(on)))

    def profile_reset(self):
        self.check(self.lib.qe_profile_reset(self.h))

    def profile_read(self, name: str):
        """(launches, total device ms) of kernel `name` since the last reset."""
        n, ms = ctypes.c_int64(0), ctypes.c_double(0)
        self.check(self.lib.qe_profile_read(self.h, name.encode(), ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def debug_fail_alloc(self, n: int):
        self.lib.qe_debug_fail_alloc(self.h, n)

    def debug_set_spin_limit(self, iterations: int):
        self.lib.qe_debug_set_spin_limit(self.h, iterations)


# ------------------------------------------------------------ entry points
# Each function mirrors the C entry point of the same name.

def qe_filter(ctx: Context, cols, preds, out_sel=None, out_count=None, stream=None, check=True):
    """preds: list of (col index, op, lo[, hi]).  Returns (out_sel, out_count)."""
    n = cols[0].numel() if cols else 0
    dev = cols[0].device if cols else torch.device("cuda", ctx.device)
    if out_sel is None:
        out_sel = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=dev)
    ccols = (qe_col * max(1, len(cols)))(*[col(c) for c in cols])
    cpreds = (qe_pred * max(1, len(preds)))(*[qe_pred(p[0], p[1], p[2], p[3] if len(p) > 3 else 0)
                                             for p in preds])
    ctx.check(ctx.lib.qe_filter(ctx.h, ccols, len(cols), cpreds, len(preds), n, _ptr(out_sel),
                                out_sel.numel() if n else 0, _ptr(out_count), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return out_sel, out_count


FILTER_NOALLOC_MAX_ROWS = 65536 * 4096


def qe_filter_noalloc(ctx: Context, cols, preds, out_sel, out_count, nrows=None, stream=None, check=True):
    """qe_filter without device allocation inside the call; the caller
    passes every output buffer (see qe_filter_noalloc in qe.h)."""
    n = (cols[0].numel() if cols else 0) if nrows is None else nrows
    ccols = (qe_col * max(1, len(cols)))(*[col(c) for c in cols])
    cpreds = (qe_pred * max(1, len(preds)))(*[qe_pred(p[0], p[1], p[2], p[3] if len(p) > 3 else 0)
                                             for p in preds])
    ctx.check(ctx.lib.qe_filter_noalloc(ctx.h, ccols, len(cols), cpreds, len(preds), n, _ptr(out_sel),
                                        out_sel.numel(), _ptr(out_count), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return out_sel, out_count


def qe_partition(ctx: Context, keys, payloads, log2f, mode=PART_HASH, shift=0, out_keys=None, out_payloads=None,
                 out_offsets=None, stream=None, check=True):
    """Returns (out_keys, [out_payloads], out_offsets[F+1])."""
    n = keys.numel()
    if out_keys is None:
        out_keys = torch.empty_like(keys)
    if out_payloads is None:
        out_payloads = [torch.empty_like(p) for p in payloads]
    if out_offsets is None:
        out_offsets = torch.empty((1 << log2f) + 1, dtype=torch.int64, device=keys.device)
    cpay = (qe_col * max(1, len(payloads)))(*[col(p) for p in payloads])
    opay = (ctypes.c_void_p * max(1, len(payloads)))(*[p.data_ptr() for p in out_payloads])
    ctx.check(ctx.lib.qe_partition(ctx.h, _ptr(keys), cpay, len(payloads), n, log2f, mode, shift,
                                   _ptr(out_keys), opay, _ptr(out_offsets), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return out_keys, out_payloads, out_offsets


class HashTable:
    def __init__(self, ctx: Context, handle):
        self.ctx, self.h = ctx, handle

    def info(self) -> qe_ht_info:
        i = qe_ht_info()
        self.ctx.check(self.ctx.lib.qe_join_info(self.h, ctypes.byref(i)))
        return i

    def destroy(self, stream=None):
        if self.h:
            self.ctx.check(self.ctx.lib.qe_join_destroy(self.ctx.h, self.h, _stream(stream)))
            self.h = None


def build_opts(layout=HT_AUTO, key_range=None) -> qe_build_opts:
    if key_range is None:
        return qe_build_opts(layout, 0, 0, 0)
    return qe_build_opts(layout, 1, int(key_range[0]), int(key_range[1]))


def qe_join_build(ctx: Context, keys, payload, layout=HT_AUTO, key_range=None, stream=None, check=True):
    h = ctypes.c_void_p()
    o = build_opts(layout, key_range)
    ctx.check(ctx.lib.qe_join_build(ctx.h, _ptr(keys), _ptr(payload), keys.numel(), ctypes.byref(o),
                                    ctypes.byref(h), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return HashTable(ctx, h)


def qe_join_probe(ctx: Context, ht: HashTable, probe_keys, sel=None, n=None, capacity=None, out_rows=None,
                  out_payload=None, out_count=None, stream=None, check=True):
    if n is None:
        n = sel.numel() if sel is not None else probe_keys.numel()
    dev = probe_keys.device
    if capacity is None:
        capacity = max(n, 1)
    if out_rows is None:
        out_rows = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    if out_payload is None:
        out_payload = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=dev)
    ctx.check(ctx.lib.qe_join_probe(ctx.h, ht.h, _ptr(probe_keys), _ptr(sel), n, _ptr(out_rows),
                                    _ptr(out_payload), capacity, _ptr(out_count), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return out_rows, out_payload, out_count


def qe_join_build_pair(ctx: Context, key_hi, key_lo, payload, stream=None, check=True):
    """Table keyed on a pair of int32 columns (unique pairs)."""
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.qe_join_build_pair(ctx.h, _ptr(key_hi), _ptr(key_lo), _ptr(payload), key_hi.numel(),
                                         ctypes.byref(h), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return HashTable(ctx, h)


def qe_join_probe_pair(ctx: Context, ht: HashTable, probe_hi, probe_lo, sel=None, n=None, capacity=None,
                       out_rows=None, out_payload=None, out_count=None, stream=None, check=True):
    if n is None:
        n = sel.numel() if sel is not None else probe_hi.numel()
    dev = probe_hi.device
    if capacity is None:
        capacity = max(n, 1)
    if out_rows is None:
        out_rows = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    if out_payload is None:
        out_payload = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=dev)
    ctx.check(ctx.lib.qe_join_probe_pair(ctx.h, ht.h, _ptr(probe_hi), _ptr(probe_lo), _ptr(sel), n, _ptr(out_rows),
                                         _ptr(out_payload), capacity, _ptr(out_count), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return out_rows, out_payload, out_count


def qe_join_build_multi(ctx: Context, keys, payload, layout=HT_AUTO, key_range=None, stream=None, check=True):
    """Multimap for the many-to-many join (keys may repeat)."""
    h = ctypes.c_void_p()
    o = build_opts(layout, key_range)
    ctx.check(ctx.lib.qe_join_build_multi(ctx.h, _ptr(keys), _ptr(payload), keys.numel(), ctypes.byref(o),
                                          ctypes.byref(h), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return HashTable(ctx, h)


def qe_join_probe_multi(ctx: Context, ht: HashTable, probe_keys, sel=None, n=None, capacity=None, out_rows=None,
                        out_payload=None, out_count=None, stream=None, check=True):
    """Every (probe row, build payload) pair with equal keys, positions in order."""
    if n is None:
        n = sel.numel() if sel is not None else probe_keys.numel()
    dev = probe_keys.device
    if capacity is None:
        capacity = max(n, 1)
    if out_rows is None:
        out_rows = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    if out_payload is None:
        out_payload = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=dev)
    ctx.check(ctx.lib.qe_join_probe_multi(ctx.h, ht.h, _ptr(probe_keys), _ptr(sel), n, _ptr(out_rows),
                                          _ptr(out_payload), capacity, _ptr(out_count), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return out_rows, out_payload, out_count


def qe_join_build_set(ctx: Context, keys, layout=HT_AUTO, key_range=None, stream=None, check=True):
    """Key set for the semi- and anti-join (keys may repeat, no payloads)."""
    h = ctypes.c_void_p()
    o = build_opts(layout, key_range)
    ctx.check(ctx.lib.qe_join_build_set(ctx.h, _ptr(keys), keys.numel(), ctypes.byref(o), ctypes.byref(h),
                                        _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return HashTable(ctx, h)


def qe_join_semi(ctx: Context, ht: HashTable, probe_keys, sel=None, n=None, anti=False, capacity=None,
                 out_rows=None, out_count=None, stream=None, check=True):
    """Rows (in probe order) whose key is (semi) or is not (anti) in the table."""
    if n is None:
        n = sel.numel() if sel is not None else probe_keys.numel()
    dev = probe_keys.device
    if capacity is None:
        capacity = max(n, 1)
    if out_rows is None:
        out_rows = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=dev)
    ctx.check(ctx.lib.qe_join_semi(ctx.h, ht.h, _ptr(probe_keys), _ptr(sel), n, int(bool(anti)), _ptr(out_rows),
                                   capacity, _ptr(out_count), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return out_rows, out_count


@dataclass
class Groups:
    keys: torch.Tensor
    aggs: list
    ngroups: torch.Tensor
    capacity: int
    avg: dict = None      # aggregate index -> float64 tensor of derived averages

    def to_host(self):
        """(keys, [aggs]) trimmed to ngroups, as CPU tensors."""
        n = min(int(self.ngroups.item()), self.capacity)
        return self.keys[:n].cpu(), [a[:n].cpu() for a in self.aggs]

    def avg_host(self, a: int):
        """The derived averages of aggregate a, trimmed to ngroups (CPU)."""
        n = min(int(self.ngroups.item()), self.capacity)
        return self.avg[a][:n].cpu()


def alloc_groups(capacity: int, naggs: int, device, avg=()) -> tuple:
    """Output buffers of a group-by; avg lists the SUM aggregates whose
    derived FP64 average (over the call's COUNT aggregate) is also wanted."""
    keys = torch.empty(max(capacity, 1), dtype=torch.int64, device=device)
    aggs = [torch.empty(max(capacity, 1), dtype=torch.int64, device=device) for _ in range(naggs)]
    ng = torch.zeros(1, dtype=torch.int64, device=device)
    avgs = {a: torch.full((max(capacity, 1),), float("nan"), dtype=torch.float64, device=device) for a in avg}
    out = qe_groups_out(capacity, keys.data_ptr(), (ctypes.c_void_p * MAX_AGGS)(*(
        [a.data_ptr() for a in aggs] + [None] * (MAX_AGGS - naggs))), ng.data_ptr(),
        (ctypes.c_void_p * MAX_AGGS)(*[avgs[a].data_ptr() if a in avgs else None for a in range(MAX_AGGS)]))
    return Groups(keys, aggs, ng, capacity, avgs), out


def qe_groupby(ctx: Context, key_lo, aggs, key_hi=None, rows=None, n=None, capacity=1024, placement=GB_AUTO,
               gather_lo=False, gather_hi=False, stream=None, check=True, avg=()):
    """aggs: list of (op, a, b, gather) with a/b tensors (or None); avg: the
    SUM aggregates whose derived averages are wanted."""
    if n is None:
        n = rows.numel() if rows is not None else key_lo.numel()
    dev = key_lo.device
    groups, out = alloc_groups(capacity, len(aggs), dev, avg)
    carr = []
    for ag in aggs:
        op, a, b = ag[0], ag[1], ag[2]
        g = bool(ag[3]) if len(ag) > 3 else False
        carr.append(qe_agg(op, 0, col(a, g) if a is not None else qe_col(None, I64, 0),
                           col(b, g) if b is not None else qe_col(None, I64, 0)))
    caggs = (qe_agg * max(1, len(aggs)))(*carr)
    khi = col(key_hi, gather_hi) if key_hi is not None else qe_col(None, I32, 0)
    ctx.check(ctx.lib.qe_groupby(ctx.h, n, _ptr(rows), khi, col(key_lo, gather_lo), caggs, len(aggs), placement,
                                 ctypes.byref(out), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return groups


def pipeline_desc(fact, preds, fk_col=-1, dim_key=None, dim_payload=None, ht: HashTable | None = None,
                  key_hi_col=-1, key_lo_col=JOIN_PAYLOAD, aggs=(), dim_key_range=None, layout=HT_AUTO,
                  expected_groups=0, est_selectivity=0.0, key_range=None, join_kind=INNER) -> qe_pipeline_desc:
    """fact: list of tensors; preds: (col, op, lo[, hi]); aggs: (op, a, b) column indices;
    join_kind: INNER, SEMI or ANTI (the latter two take no dim_payload)."""
    d = qe_pipeline_desc()
    d.n_fact = fact[0].numel() if fact else 0
    for i, t in enumerate(fact):
        d.fact[i] = col(t)
    d.n_fact_cols = len(fact)
    d.n_preds = len(preds)
    for i, p in enumerate(preds):
        d.preds[i] = qe_pred(p[0], p[1], p[2], p[3] if len(p) > 3 else 0)
    d.fk_col, d.key_hi_col, d.key_lo_col = fk_col, key_hi_col, key_lo_col
    d.n_aggs = len(aggs)
    for i, (op, a, b) in enumerate(aggs):
        d.aggs[i] = qe_agg_spec(op, a, b, 0)
    d.dim_key = dim_key.data_ptr() if dim_key is not None else None
    d.dim_payload = dim_payload.data_ptr() if dim_payload is not None else None
    d.n_dim = dim_key.numel() if dim_key is not None else 0
    d.ht = ht.h if ht is not None else None
    d.build = build_opts(layout, dim_key_range)
    d.expected_groups = expected_groups
    d.est_selectivity = est_selectivity
    d.join_kind = join_kind
    if key_range is not None:
        # ((hi_min, hi_max), (lo_min, lo_max)) column statistics; lo None takes
        # the join payload's range from the join table
        (d.key_hi_min, d.key_hi_max) = key_range[0] if key_range[0] is not None else (0, 0)
        (d.key_lo_min, d.key_lo_max) = key_range[1] if key_range[1] is not None else (1, 0)
        d.have_key_range = 1
    # the descriptor holds raw device pointers: keep the tensors alive with it
    d._keep = (list(fact), dim_key, dim_payload, ht)
    return d


def qe_pipeline(ctx: Context, desc: qe_pipeline_desc, capacity: int, stream=None, check=True, out=None, avg=()):
    """out: (Groups or None, qe_groups_out) to write into existing buffers;
    avg: the SUM aggregates whose derived averages are wanted."""
    if out is None:
        groups, cout = alloc_groups(capacity, desc.n_aggs, torch.device("cuda", ctx.device), avg)
    else:
        groups, cout = out
    ctx.check(ctx.lib.qe_pipeline(ctx.h, ctypes.byref(desc), ctypes.byref(cout), _stream(stream)))
    if check:
        ctx.sync_status(stream)
    return groups


class Batch:
    """A planned batch of pipelines sharing one persistent launch."""

    def __init__(self, ctx: Context, descs, outs, opts: qe_batch_opts | None = None, stream=None):
        self.ctx = ctx
        n = len(descs)
        self._descs = (qe_pipeline_desc * n)(*descs)
        self._outs = (qe_groups_out * n)(*outs)
        self._keep = (list(descs), list(outs))
        h = ctypes.c_void_p()
        o = opts if opts is not None else qe_batch_opts(0, 0, 0, 1)
        ctx.check(ctx.lib.qe_batch_create(ctx.h, self._descs, self._outs, n, ctypes.byref(o), ctypes.byref(h),
                                          _stream(stream)))
        self.h = h

    def launch(self, stream=None):
        self.ctx.check(self.ctx.lib.qe_batch_launch(self.ctx.h, self.h, _stream(stream)))

    def destroy(self, stream=None):
        if self.h:
            self.ctx.check(self.ctx.lib.qe_batch_destroy(self.ctx.h, self.h, _stream(stream)))
            self.h = None


def qe_batch_create(ctx, descs, outs, opts=None, stream=None) -> Batch:
    return Batch(ctx, descs, outs, opts, stream)


def qe_batch_launch(ctx, batch: Batch, stream=None):
    batch.launch(stream)


def qe_batch_destroy(ctx, batch: Batch, stream=None):
    batch.destroy(stream)


def qe_batch_run(ctx: Context, descs, outs, opts=None, stream=None, check=True):
    n = len(descs)
    cd = (qe_pipeline_desc * n)(*descs)
    co = (qe_groups_out * n)(*outs)
    o = opts if opts is not None else qe_batch_opts(0, 0, 0, 0)
    ctx.check(ctx.lib.qe_batch_run(ctx.h, cd, co, n, ctypes.byref(o), _stream(stream)))
    if check:
        ctx.sync_status(stream)


# ------------------------------------------------------------ exchange planner
# Host-only entry points of include/qe_plan.h: no GPU or context needed.
def link(bandwidth: float | None = None, L: float = 0.0, c: float | None = None) -> qe_link:
    """A link of constant `bandwidth` bytes/s, or Hockney parameters (L, c)."""
    if bandwidth is not None:
        return qe_link(0.0, 1.0 / bandwidth)
    return qe_link(L, 0.0 if c is None else c)


def cluster(k: int, V: int, bcast_net: qe_link, bcast_gpu: qe_link, shuf_net: qe_link | None = None,
            shuf_gpu: qe_link | None = None) -> qe_cluster:
    """V machines of k GPUs; the shuffle links default to the broadcast's."""
    return qe_cluster(k, V, bcast_net, bcast_gpu, shuf_net if shuf_net is not None else bcast_net,
                      shuf_gpu if shuf_gpu is not None else bcast_gpu)


def _plan_check(lib, st):
    if st != OK:
        raise QeError(st, lib.qe_plan_last_error().decode())


def _f64(x):
    import numpy as np
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


def qe_plan_exchange_time(cl: qe_cluster, op: int, nbytes: float) -> float:
    lib = load_library()
    t = ctypes.c_double(0)
    _plan_check(lib, lib.qe_plan_exchange_time(ctypes.byref(cl), op, float(nbytes), ctypes.byref(t)))
    return t.value


def qe_plan_shuffle_skew(k: int, V: int, msg, bn: float):
    """(seconds, per-machine sent bytes, per-machine received bytes)."""
    import numpy as np
    lib = load_library()
    m, mp = _f64(msg)
    if m.size != (k * V) ** 2:
        raise QeError(ERR_INVALID_ARG, "msg must hold N*N sizes")
    send, recv = np.zeros(max(V, 0)), np.zeros(max(V, 0))
    t = ctypes.c_double(0)
    _plan_check(lib, lib.qe_plan_shuffle_skew(k, V, mp, float(bn), ctypes.byref(t), send.ctypes.data_as(_DP),
                                              recv.ctypes.data_as(_DP)))
    return t.value, send, recv


def qe_plan_join(cl: qe_cluster, r_bytes: float, s_bytes: float, copartitioned: bool = False, r_msg=None,
                 s_msg=None):
    """(strategy, broadcast seconds, shuffle seconds)."""
    lib = load_library()
    N = cl.k * cl.V
    ptrs, keep = [], []
    for m in (r_msg, s_msg):
        if m is None:
            ptrs.append(None)
            continue
        a, p = _f64(m)
        if a.size != N * N:
            raise QeError(ERR_INVALID_ARG, "a message matrix must hold N*N sizes")
        keep.append(a)
        ptrs.append(p)
    st, tb, ts = ctypes.c_int32(-1), ctypes.c_double(0), ctypes.c_double(0)
    _plan_check(lib, lib.qe_plan_join(ctypes.byref(cl), float(r_bytes), float(s_bytes), int(bool(copartitioned)),
                                      ptrs[0], ptrs[1], ctypes.byref(st), ctypes.byref(tb), ctypes.byref(ts)))
    return st.value, tb.value, ts.value


def qe_plan_fit_link(op: int, k: int, V: int, sizes, times) -> qe_link:
    lib = load_library()
    b, bp = _f64(sizes)
    t, tp = _f64(times)
    if b.size != t.size:
        raise QeError(ERR_INVALID_ARG, "sizes and times differ in length")
    out = qe_link()
    _plan_check(lib, lib.qe_plan_fit_link(op, k, V, bp, tp, b.size, ctypes.byref(out)))
    return out


def qe_plan_skew_gradient(n_gpus: int, f: float, total: float):
    import numpy as np
    lib = load_library()
    out = np.zeros(max(n_gpus, 0))
    _plan_check(lib, lib.qe_plan_skew_gradient(n_gpus, float(f), float(total), out.ctypes.data_as(_DP)))
    return out
