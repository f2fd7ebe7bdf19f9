"""CPU oracle for the relational operator pipeline (arxiv 2506.09226).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  This module wraps the
plain C oracle in ``qe_oracle.c`` with ctypes and numpy arrays.  It shares no
code with the CUDA library and never loads it.

Operator definitions and the paper passages they follow are documented in
``qe_oracle.c``: selection (Sec. 2.1), partition with per-destination
offsets (Sec. 2.2, Sec. 2.3), inner equi-join (Sec. 2.2), group-by with
SUM/COUNT/MIN/MAX (Sec. 2.3, Sec. 2.4), and the pipeline
group-by(join(filter(fact), dim)) (Sec. 2.4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt oracle library to load instead (the mutation tests point this at
# deliberately broken copies to show the pins catch them).
_OVERRIDE = os.environ.get("QE_ORACLE_LIB")

# Oracle-side enumerations (same meaning as in qe_oracle.c).
I8, I32, I64 = 0, 1, 2
LT, LE, GT, GE, EQ, NE, BETWEEN = range(7)
SUM, COUNT, MIN, MAX = range(4)
JOIN_PAYLOAD = -2
INNER, SEMI, ANTI = 0, 1, 2
DUPLICATE_KEY = 5

_NP_TYPE = {np.dtype(np.int8): I8, np.dtype(np.int32): I32, np.dtype(np.int64): I64}


def build(force: bool = False) -> str:
    """Compile qe_oracle.c into liboracle.so next to it (gcc, -O2, portable)."""
    if _OVERRIDE:
        return _OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i64, i32, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        L.oracle_filter.restype = i64
        L.oracle_filter.argtypes = [i64, vp, vp, ci, vp, vp, vp, vp, vp]
        L.oracle_fmix64.restype = ctypes.c_uint64
        L.oracle_fmix64.argtypes = [ctypes.c_uint64]
        L.oracle_partition_of.restype = i64
        L.oracle_partition_of.argtypes = [i64, ci, ci, ci]
        L.oracle_partition.restype = None
        L.oracle_partition.argtypes = [i64, vp, ci, vp, vp, ci, ci, ci, vp, vp, vp]
        L.oracle_join.restype = ci
        L.oracle_join.argtypes = [i64, vp, vp, i64, vp, vp, vp, vp, vp]
        L.oracle_groupby.restype = i64
        L.oracle_groupby.argtypes = [i64, vp, ci, vp, vp, vp, vp]
        L.oracle_avg.restype = None
        L.oracle_avg.argtypes = [i64, vp, vp, vp]
        L.oracle_group_key.restype = i64
        L.oracle_group_key.argtypes = [ci, i64, i64]
        L.oracle_join_pair.restype = ci
        L.oracle_join_pair.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp]
        L.oracle_join_multi.restype = i64
        L.oracle_join_multi.argtypes = [i64, vp, vp, i64, vp, vp, vp, vp, i64]
        L.oracle_semi_join.restype = i64
        L.oracle_semi_join.argtypes = [i64, vp, i64, vp, vp, ci, vp]
        L.oracle_pipeline.restype = i64
        L.oracle_pipeline.argtypes = [i64, vp, vp, ci, vp, vp, vp, vp, ci, i64, vp, vp, ci,
                                      ci, ci, ci, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_pipeline_group.restype = i64
        L.oracle_pipeline_group.argtypes = [i64, vp, vp, ci, vp, vp, vp, vp, ci, i64, vp, vp, ci,
                                            ci, ci, ci, vp, vp, vp, i64, vp]
        _ = i32
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _ptr_array(arrs):
    return (ctypes.c_void_p * max(1, len(arrs)))(*[a.ctypes.data for a in arrs])


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


@dataclass
class Pred:
    """One comparison of a conjunction: column index, operator, bounds."""
    col: int
    op: int
    lo: int
    hi: int = 0


def filter(cols, preds):
    """Ids (int32, ascending) of the rows where every predicate holds."""
    cols = [np.ascontiguousarray(c) for c in cols]
    n = len(cols[0]) if cols else 0
    types = _c([_NP_TYPE[c.dtype] for c in cols], np.int32)
    pc = _c([p.col for p in preds], np.int32)
    po = _c([p.op for p in preds], np.int32)
    lo = _c([p.lo for p in preds], np.int64)
    hi = _c([p.hi for p in preds], np.int64)
    out = np.empty(max(n, 1), np.int32)
    cnt = lib().oracle_filter(n, _ptr_array(cols), _p(types), len(preds), _p(pc), _p(po),
                              _p(lo), _p(hi), _p(out))
    return out[:cnt].copy()


def fmix64(k: int) -> int:
    return int(lib().oracle_fmix64(k & 0xFFFFFFFFFFFFFFFF))


def partition_of(key: int, log2f: int, mode: int = 0, shift: int = 0) -> int:
    return int(lib().oracle_partition_of(key, log2f, mode, shift))


def partition(keys, payloads, log2f, mode=0, shift=0):
    """Stable partition; returns (out_keys, [out_payloads], offsets[F+1])."""
    keys = _c(keys, np.int64)
    payloads = [np.ascontiguousarray(p) for p in payloads]
    n = len(keys)
    out_keys = np.empty(max(n, 1), np.int64)
    out_pay = [np.empty(max(n, 1), p.dtype) for p in payloads]
    offs = np.empty((1 << log2f) + 1, np.int64)
    types = _c([_NP_TYPE[p.dtype] for p in payloads], np.int32)
    lib().oracle_partition(n, _p(keys), len(payloads), _ptr_array(payloads), _p(types),
                           log2f, mode, shift, _p(out_keys), _ptr_array(out_pay), _p(offs))
    return out_keys[:n], [o[:n] for o in out_pay], offs


def join(build_keys, build_payload, probe_keys, sel=None):
    """Inner equi-join; returns (probe_rows, payloads) in probe order.

    Raises ValueError on a duplicate build key."""
    bk, bp = _c(build_keys, np.int32), _c(build_payload, np.int32)
    pk = _c(probe_keys, np.int32)
    s = None if sel is None else _c(sel, np.int32)
    n = len(pk) if s is None else len(s)
    rows = np.empty(max(n, 1), np.int32)
    pay = np.empty(max(n, 1), np.int32)
    cnt = ctypes.c_int64(0)
    st = lib().oracle_join(len(bk), _p(bk), _p(bp), n, _p(pk), _p(s), _p(rows), _p(pay),
                           ctypes.byref(cnt))
    if st == DUPLICATE_KEY:
        raise ValueError("duplicate build key")
    return rows[:cnt.value].copy(), pay[:cnt.value].copy()


def join_pair(build_hi, build_lo, build_payload, probe_hi, probe_lo, sel=None):
    """Inner equi-join on a pair of key columns; returns (probe_rows,
    payloads) in probe order.  Raises ValueError on a duplicate build pair."""
    bh, bl, bp = _c(build_hi, np.int32), _c(build_lo, np.int32), _c(build_payload, np.int32)
    ph, pl = _c(probe_hi, np.int32), _c(probe_lo, np.int32)
    s = None if sel is None else _c(sel, np.int32)
    n = len(ph) if s is None else len(s)
    rows = np.empty(max(n, 1), np.int32)
    pay = np.empty(max(n, 1), np.int32)
    cnt = ctypes.c_int64(0)
    st = lib().oracle_join_pair(len(bh), _p(bh), _p(bl), _p(bp), n, _p(ph), _p(pl), _p(s), _p(rows), _p(pay),
                                ctypes.byref(cnt))
    if st == DUPLICATE_KEY:
        raise ValueError("duplicate build key pair")
    return rows[:cnt.value].copy(), pay[:cnt.value].copy()


def join_multi(build_keys, build_payload, probe_keys, sel=None):
    """Many-to-many inner equi-join: (probe_rows, payloads), probe positions in
    order and, within one, the build rows in ascending order."""
    bk, bp = _c(build_keys, np.int32), _c(build_payload, np.int32)
    pk = _c(probe_keys, np.int32)
    s = None if sel is None else _c(sel, np.int32)
    n = len(pk) if s is None else len(s)
    total = lib().oracle_join_multi(len(bk), _p(bk), _p(bp), n, _p(pk), _p(s), None, None, 0)
    rows = np.empty(max(total, 1), np.int32)
    pay = np.empty(max(total, 1), np.int32)
    lib().oracle_join_multi(len(bk), _p(bk), _p(bp), n, _p(pk), _p(s), _p(rows), _p(pay), total)
    return rows[:total].copy(), pay[:total].copy()


def semi_join(build_keys, probe_keys, sel=None, anti=False):
    """Probe rows (in probe order) whose key is among the build keys, or,
    with anti, is not; build keys may repeat."""
    bk, pk = _c(build_keys, np.int32), _c(probe_keys, np.int32)
    s = None if sel is None else _c(sel, np.int32)
    n = len(pk) if s is None else len(s)
    rows = np.empty(max(n, 1), np.int32)
    cnt = lib().oracle_semi_join(len(bk), _p(bk), n, _p(pk), _p(s), int(bool(anti)), _p(rows))
    return rows[:cnt].copy()


def groupby(keys, aggs):
    """aggs: list of (op, values or None).  Returns (keys, [agg arrays]) sorted by key."""
    keys = _c(keys, np.int64)
    n = len(keys)
    ops = _c([op for op, _ in aggs], np.int32)
    vals = [(_c(v, np.int64) if v is not None else np.zeros(max(n, 1), np.int64)) for _, v in aggs]
    out_k = np.empty(max(n, 1), np.int64)
    out_a = [np.empty(max(n, 1), np.int64) for _ in aggs]
    ng = lib().oracle_groupby(n, _p(keys), len(aggs), _p(ops), _ptr_array(vals),
                              _p(out_k), _ptr_array(out_a))
    return out_k[:ng].copy(), [a[:ng].copy() for a in out_a]


def avg(sums, counts) -> np.ndarray:
    """Per-group average (double)sum / (double)count from the exact int64
    SUM and COUNT of each group (oracle_avg, Sec. 2.3)."""
    s, c = _c(sums, np.int64), _c(counts, np.int64)
    if len(s) != len(c):
        raise ValueError("sums and counts differ in length")
    out = np.empty(max(len(s), 1), np.float64)
    lib().oracle_avg(len(s), _p(s), _p(c), _p(out))
    return out[:len(s)].copy()


def group_key(has_hi: bool, hi: int, lo: int) -> int:
    return int(lib().oracle_group_key(int(has_hi), hi, lo))


@dataclass
class Query:
    """group-by(join(filter(fact), dim)) over fact column indices.

    fk_col < 0 means no join; key_lo_col == JOIN_PAYLOAD takes the low key
    half from the joined dim payload; aggs are (op, col_a, col_b) with -1 for
    an absent column; join_kind is INNER, SEMI or ANTI."""
    preds: list = field(default_factory=list)
    fk_col: int = -1
    key_hi_col: int = -1
    key_lo_col: int = JOIN_PAYLOAD
    aggs: list = field(default_factory=list)
    join_kind: int = 0


def _query_args(fact, q: Query, dim_key, dim_pay):
    fact = [np.ascontiguousarray(c) for c in fact]
    types = _c([_NP_TYPE[c.dtype] for c in fact], np.int32)
    pc = _c([p.col for p in q.preds], np.int32)
    po = _c([p.op for p in q.preds], np.int32)
    lo = _c([p.lo for p in q.preds], np.int64)
    hi = _c([p.hi for p in q.preds], np.int64)
    dk = _c(dim_key if dim_key is not None else [], np.int32)
    dp = _c(dim_pay if dim_pay is not None else [], np.int32)
    ops = _c([a[0] for a in q.aggs], np.int32)
    aa = _c([a[1] for a in q.aggs], np.int32)
    ab = _c([a[2] for a in q.aggs], np.int32)
    keep = (fact, types, pc, po, lo, hi, dk, dp, ops, aa, ab)
    n = len(fact[0]) if fact else 0
    args = [n, _ptr_array(fact), _p(types), len(q.preds), _p(pc), _p(po), _p(lo), _p(hi),
            q.fk_col, len(dk), _p(dk), _p(dp) if dim_pay is not None else None, q.join_kind,
            q.key_hi_col, q.key_lo_col, len(q.aggs),
            _p(ops), _p(aa), _p(ab)]
    return args, keep


def pipeline(fact, q: Query, dim_key=None, dim_pay=None):
    """Returns dict(keys, aggs, nsel, njoin), groups in ascending key order."""
    args, keep = _query_args(fact, q, dim_key, dim_pay)
    n = args[0]
    out_k = np.empty(max(n, 1), np.int64)
    out_a = [np.empty(max(n, 1), np.int64) for _ in q.aggs]
    nsel, nj = ctypes.c_int64(0), ctypes.c_int64(0)
    ng = lib().oracle_pipeline(*args, _p(out_k), _ptr_array(out_a), ctypes.byref(nsel),
                               ctypes.byref(nj))
    del keep
    if ng == -2:
        raise ValueError("a semi- or anti-join has no payload to group by")
    if ng < 0:
        raise ValueError("duplicate build key")
    return dict(keys=out_k[:ng].copy(), aggs=[a[:ng].copy() for a in out_a],
                nsel=nsel.value, njoin=nj.value)


def pipeline_group(fact, q: Query, gkey: int, dim_key=None, dim_pay=None):
    """Aggregates of one group, computed over the full input on their own."""
    args, keep = _query_args(fact, q, dim_key, dim_pay)
    out = np.zeros(max(1, len(q.aggs)), np.int64)
    cnt = lib().oracle_pipeline_group(*args, int(gkey), _p(out))
    del keep
    return int(cnt), out[:len(q.aggs)].copy()
