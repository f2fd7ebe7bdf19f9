"""Planted mistakes in the exchange-model oracle are caught by its pins.

Each case applies one plausible mistake to a copy of oracle/exchange.py (a
wrong step count, the wrong message size, max for min, a dropped exclusion,
a transposed index, an off-by-one placement, a wrong link) and runs
tests/test_exchange_pins.py against it; the pins must fail for every mutant.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "exchange.py")

MUTANTS = {
    "bcast_steps": ("return (N - 1) * (S / N) / B", "return N * (S / N) / B"),
    "bcast_max": ("B = min(net.bw(m), gpu.bw(m))", "B = max(net.bw(m), gpu.bw(m))"),
    "bcast_v1_link": ("    if V == 1:\n        B = gpu.bw(m)", "    if V == 1:\n        B = net.bw(m)"),
    "bcast_msg": ("    m = S / N\n    if V == 1:\n        B", "    m = S / (N * N)\n    if V == 1:\n        B"),
    "shuffle_v": ("return S * (V - 1) / (V * V * net.bw(m))", "return S * V / (V * V * net.bw(m))"),
    "shuffle_msg": ("m = S / (N * N)\n    if V == 1:\n        return", "m = S / N\n    if V == 1:\n        return"),
    "shuffle_v1": ("return S * (N - 1) / (N * N * gpu.bw(m))", "return S * (N - 1) / (N * gpu.bw(m))"),
    "skew_self": ("            for p in range(V):\n                if p == i:\n                    continue\n",
                  "            for p in range(V):\n"),
    "skew_recv_index": ("recv[i] += msg[p * k + q][i * k + j]", "recv[i] += msg[i * k + j][p * k + q]"),
    "skew_flat_index": ("send[i] += msg[i * k + j][p * k + q]", "send[i] += msg[j * V + i][p * k + q]"),
    "gradient_offset": ("return [x * (1.0 + i * f) for i in range(n_gpus)]",
                        "return [x * (1.0 + (i + 1) * f) for i in range(n_gpus)]"),
    "plan_small": ("small = min(r_bytes, s_bytes)", "small = r_bytes"),
    "plan_side": ("(BROADCAST_R if r_bytes <= s_bytes else BROADCAST_S)", "BROADCAST_R"),
    "fit_swap": ("return Link(float(sol[0]), float(sol[1]))", "return Link(float(sol[1]), float(sol[0]))"),
    "eq3_k": ("return (N - 1) / (N - k) * V - 1", "return (N - 1) / (N - 1) * V - 1"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mpath = tmp_path / "exchange_mutant.py"
    mpath.write_text(src.replace(old, new))
    env = dict(os.environ, QE_EXCHANGE_ORACLE=str(mpath))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_exchange_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
