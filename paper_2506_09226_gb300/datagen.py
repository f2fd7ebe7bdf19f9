"""Seeded synthetic warehouse tables (star schema) for tests and benchmarks.

This module only draws random columns.  It holds none of the operators'
arithmetic (no predicate, hash, join or aggregate), so the CPU oracle and the
CUDA library can both be fed from it without sharing any method code.

The paper measures on TPC-H and JCC-H (Sec. 4.3); neither is available here,
so these tables stand in for them with the same shape: a fact table joined to
a dimension table on a foreign key, a date column over a seven-year span
(2557 days) filtered by a range predicate, fixed-point prices, small-domain
flags, and, for the skewed case, Zipf-distributed foreign keys in the manner
of JCC-H.

Column layout of the fact table (21 bytes per row):
    fk    int32  uniform over the dimension keys (or Zipf(s) over them)
    date  int32  uniform in [0, 2557)
    price int64  fixed-point cents, uniform in [100, 10^7]
    qty   int32  uniform in [1, 50]
    flag  int8   uniform in {0, 1, 2}
Optional: code int32 (dictionary codes, uniform in [0, n_codes)),
          gkey int64 (drawn from a pool of n_gkeys random 64-bit keys).
Build sides of the join variants: multi_dim (repeated keys, a fixed number
of rows per key) and pair_dim (unique pairs of int32 keys), both shaped like
TPC-H partsupp.
Dimension table: key int32 = a seeded permutation of 0..n_dim-1,
                 attr int32 uniform in [0, n_attr).

Draws use torch generators so that large tables can be produced directly in
device memory; the same call on the CPU gives the bytes the oracle reads.
Large device draws are done in chunks to bound peak memory.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

DATE_SPAN = 2557          # days in the date domain [0, 2557)
PRICE_LO, PRICE_HI = 100, 10 ** 7
QTY_LO, QTY_HI = 1, 50
N_FLAGS = 3
CHUNK = 1 << 26           # rows drawn per chunk on the device


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def _randint(lo, hi_incl, n, dtype, g, device):
    out = torch.empty(n, dtype=dtype, device=device)
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        out[s:e] = torch.randint(lo, hi_incl + 1, (e - s,), generator=g, device=device,
                                 dtype=dtype)
    return out


def zipf_ranks(n: int, n_keys: int, s: float, g, device) -> torch.Tensor:
    """n draws of a 0-based rank r with P(r) proportional to (r+1)^-s, by
    inverse-CDF lookup in an fp64 cumulative table."""
    w = torch.arange(1, n_keys + 1, dtype=torch.float64, device=device).pow_(-s)
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    del w
    out = torch.empty(n, dtype=torch.int32, device=device)
    for a in range(0, n, CHUNK):
        e = min(n, a + CHUNK)
        u = torch.rand(e - a, generator=g, device=device, dtype=torch.float64)
        r = torch.searchsorted(cdf, u, right=True)
        out[a:e] = r.clamp_(max=n_keys - 1).to(torch.int32)
    return out


def star_dim(n_dim: int, n_attr: int, *, seed: int, device="cpu") -> dict:
    g = _gen(seed * 1000 + 1, device)
    key = torch.randperm(n_dim, generator=g, device=device, dtype=torch.int32) \
        if n_dim > 0 else torch.empty(0, dtype=torch.int32, device=device)
    attr = _randint(0, max(n_attr - 1, 0), n_dim, torch.int32, g, device)
    return {"key": key, "attr": attr}


def star_fact(n: int, n_dim: int, *, seed: int, device="cpu", zipf_s: float | None = None,
              n_codes: int = 0, n_gkeys: int = 0) -> dict:
    g = _gen(seed * 1000 + 2, device)
    if zipf_s is None:
        fk = _randint(0, n_dim - 1, n, torch.int32, g, device)
    else:
        ranks = zipf_ranks(n, n_dim, zipf_s, g, device)
        rank_to_key = torch.randperm(n_dim, generator=g, device=device, dtype=torch.int32)
        fk = rank_to_key[ranks.long()] if n else ranks
        del ranks
    cols = {
        "fk": fk,
        "date": _randint(0, DATE_SPAN - 1, n, torch.int32, g, device),
        "price": _randint(PRICE_LO, PRICE_HI, n, torch.int64, g, device),
        "qty": _randint(QTY_LO, QTY_HI, n, torch.int32, g, device),
        "flag": _randint(0, N_FLAGS - 1, n, torch.int8, g, device),
    }
    if n_codes:
        cols["code"] = _randint(0, n_codes - 1, n, torch.int32, g, device)
    if n_gkeys:
        pool = torch.randint(-2 ** 63, 2 ** 63 - 1, (n_gkeys,), generator=g, device=device,
                             dtype=torch.int64)
        idx = _randint(0, n_gkeys - 1, n, torch.int32, g, device)
        cols["gkey"] = pool[idx.long()] if n else torch.empty(0, dtype=torch.int64, device=device)
    return cols


def multi_dim(n_keys: int, per_key: int, n_attr: int, *, seed: int, device="cpu") -> dict:
    """Build side of a many-to-many join, shaped like TPC-H partsupp (a fixed
    number of supplier rows per part): each key of 0..n_keys-1 sits on exactly
    per_key rows, the rows in random order; attr int32 uniform in [0, n_attr)."""
    g = _gen(seed * 1000 + 6, device)
    n = n_keys * per_key
    key = torch.randperm(n, generator=g, device=device, dtype=torch.int32) // per_key \
        if n > 0 else torch.empty(0, dtype=torch.int32, device=device)
    attr = _randint(0, max(n_attr - 1, 0), n, torch.int32, g, device)
    return {"key": key, "attr": attr}


def pair_dim(n_keys: int, per_key: int, *, seed: int, device="cpu") -> dict:
    """Build side of a join on two key columns, shaped like TPC-H partsupp
    keyed on (part, supplier): row (k, j), for k < n_keys and j < per_key, has
    hi = k and lo = off[k] + j, with off[k] uniform in [0, 2^30), so every
    pair is unique while both halves repeat; rows in random order; payload
    int32 uniform.  off is returned for pair_probe_lo."""
    g = _gen(seed * 1000 + 7, device)
    n = n_keys * per_key
    off = _randint(0, (1 << 30) - 1, n_keys, torch.int32, g, device)
    idx = torch.randperm(n, generator=g, device=device, dtype=torch.int32) \
        if n > 0 else torch.empty(0, dtype=torch.int32, device=device)
    hi = idx // per_key
    lo = off[hi.long()] + idx % per_key if n > 0 else idx
    del idx
    pay = _randint(-2 ** 31, 2 ** 31 - 1, n, torch.int32, g, device)
    return {"hi": hi, "lo": lo, "payload": pay, "off": off}


def pair_probe_lo(hi: torch.Tensor, off: torch.Tensor, span: int, *, seed: int) -> torch.Tensor:
    """Second key column of a pair-key probe whose first column is hi (keys
    of pair_dim): off[hi] + j with j uniform in [0, span).  With span =
    per_key + 1, about one row in span has no partner in the build."""
    g = _gen(seed * 1000 + 8, hi.device)
    out = torch.empty_like(hi)
    for s in range(0, hi.numel(), CHUNK):
        e = min(hi.numel(), s + CHUNK)
        out[s:e] = off[hi[s:e].long()] + torch.randint(0, span, (e - s,), generator=g, device=hi.device,
                                                       dtype=torch.int32)
    return out


def key_payload_pairs(n: int, *, seed: int, device="cpu"):
    """(int64 key uniform over all 64-bit values, int64 payload = row id)."""
    g = _gen(seed * 1000 + 3, device)
    key = torch.empty(n, dtype=torch.int64, device=device)
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        key[s:e] = torch.randint(-2 ** 63, 2 ** 63 - 1, (e - s,), generator=g, device=device,
                                 dtype=torch.int64)
    payload = torch.arange(n, dtype=torch.int64, device=device)
    return key, payload


def log_uniform_sizes(count: int, lo: float, hi: float, *, seed: int) -> np.ndarray:
    """count sizes floor(exp(U[ln lo, ln hi]))."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)


@dataclass
class Arrival:
    t: float          # seconds since the start of the trace
    shape: int        # which resident table set (0, 1, 2)
    offset: int       # first fact row of the request's range
    n: int            # fact rows in the request
    date_hi: int      # predicate bound c of date < c


def poisson_trace(duration_s: float, rate: float, table_rows: list, *, seed: int,
                  n_lo: float = 1e4, n_hi: float = 5e8) -> list:
    """Poisson arrivals; each request takes a row range of one resident fact
    table, a log-uniform size and a uniform selectivity in [1%, 90%]."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        shape = int(rng.integers(0, len(table_rows)))
        rows = int(table_rows[shape])
        n = int(min(rows, math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))))
        off = int(rng.integers(0, rows - n + 1))
        sel = rng.uniform(0.01, 0.90)
        out.append(Arrival(t, shape, off, n, int(round(sel * DATE_SPAN))))
    return out


def batch_star(sizes, n_attr: int, *, seed: int, device="cpu") -> dict:
    """Many independent star pipelines stored back to back: pipeline i owns
    fact rows [fact_off[i], fact_off[i] + n_i) and dimension rows
    [dim_off[i], dim_off[i] + n_i // 10) (at least one).  Each dimension's
    keys are a permutation of 0..nd_i-1 and each pipeline's foreign keys are
    uniform over them; the other columns follow star_fact."""
    sizes = [int(x) for x in sizes]
    nds = [max(1, n // 10) for n in sizes]
    fact_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    dim_off = np.concatenate([[0], np.cumsum(nds)]).astype(np.int64)
    total, dtotal = int(fact_off[-1]), int(dim_off[-1])
    g = _gen(seed * 1000 + 5, device)
    cols = {
        "fk": torch.empty(total, dtype=torch.int32, device=device),
        "date": _randint(0, DATE_SPAN - 1, total, torch.int32, g, device),
        "price": _randint(PRICE_LO, PRICE_HI, total, torch.int64, g, device),
        "qty": _randint(QTY_LO, QTY_HI, total, torch.int32, g, device),
        "flag": _randint(0, N_FLAGS - 1, total, torch.int8, g, device),
    }
    key = torch.empty(dtotal, dtype=torch.int32, device=device)
    for i, (n, nd) in enumerate(zip(sizes, nds)):
        a, b = int(fact_off[i]), int(dim_off[i])
        if n:
            cols["fk"][a:a + n] = torch.randint(0, nd, (n,), generator=g, device=device, dtype=torch.int32)
        key[b:b + nd] = torch.randperm(nd, generator=g, device=device, dtype=torch.int32)
    attr = _randint(0, n_attr - 1, dtotal, torch.int32, g, device)
    return {"fact": cols, "dim": {"key": key, "attr": attr}, "fact_off": fact_off, "dim_off": dim_off,
            "sizes": np.asarray(sizes, np.int64), "dim_sizes": np.asarray(nds, np.int64)}
