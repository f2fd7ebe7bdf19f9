"""Planted mistakes in the oracle are caught by its pins.

Each case applies one plausible mistake to a copy of oracle/qe_oracle.c (a
boundary off by one, a dropped step of the hash, a wrong index, a flipped
sign, swapped key halves, an unstable placement, a dropped predicate term, a
wrong payload index, a flipped or shortened membership test, a swapped join
kind, a zero-extended group key, an integer or single-precision average),
compiles it, and runs
tests/test_oracle_pins.py against it; the pin suite must fail for every
mutant.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qe_oracle.c")

MUTANTS = {
    "lt_boundary": ("case OR_LT: return x < lo;", "case OR_LT: return x <= lo;"),
    "hash_drop_step": ("    k ^= k >> 33;\n    k *= 0xff51afd7ed558ccdULL;",
                       "    k *= 0xff51afd7ed558ccdULL;"),
    "offsets_index": ("out_offsets[oracle_partition_of(keys[i], log2f, mode, shift) + 1] += 1;",
                      "out_offsets[oracle_partition_of(keys[i], log2f, mode, shift)] += 1;"),
    "unstable_place": ("int64_t dst = next[p]++;",
                       "int64_t dst = out_offsets[p + 1] - 1 - (next[p]++ - out_offsets[p]);"),
    "sum_sign": ("sum += (uint64_t)v;\n                if (v < mn)",
                 "sum -= (uint64_t)v;\n                if (v < mn)"),
    "key_swap": ("return (int64_t)(((uint64_t)hi << 32) | (uint64_t)(uint32_t)lo);",
                 "return (int64_t)(((uint64_t)lo << 32) | (uint64_t)(uint32_t)hi);"),
    "min_flip": ("if (v < mn) mn = v;\n                if (v > mx)",
                 "if (v > mn) mn = v;\n                if (v > mx)"),
    "drop_pred": ("for (int p = 0; p < npreds; p++) {\n            int c = pred_col[p];\n            if (!pred_holds",
                  "for (int p = 0; p + 1 < npreds; p++) {\n            int c = pred_col[p];\n            if (!pred_holds"),
    "payload_index": ("out_pay[count] = b[lo].payload;",
                      "out_pay[count] = b[lo > 0 ? lo - 1 : 0].payload;"),
    "pair_drop_lo": ("    return (x->lo > y->lo) - (x->lo < y->lo);\n}", "    return 0;\n}"),
    "multi_unstable": ("    return (x->payload > y->payload) - (x->payload < y->payload);   /* payload holds j here */",
                       "    return (x->payload < y->payload) - (x->payload > y->payload);   /* payload holds j here */"),
    "multi_last_row": ("for (int64_t t = lo; t < nb && b[t].key == k; t++) {",
                       "for (int64_t t = lo; t + 1 < nb && b[t].key == k; t++) {"),
    "semi_flip": ("if (found != (anti != 0)) out_row[count++] = row;",
                  "if (found == (anti != 0)) out_row[count++] = row;"),
    "semi_last_key": ("int found = lo < nb && b[lo] == k;", "int found = lo + 1 < nb && b[lo] == k;"),
    "pipeline_kind": ("join_kind == 2, rows);", "join_kind == 1, rows);"),
    "key_zero_extend": ("    if (!has_hi) return lo;", "    if (!has_hi) return (int64_t)(uint32_t)lo;"),
    "avg_int_div": ("out[g] = (double)sum[g] / (double)count[g];", "out[g] = (double)(sum[g] / count[g]);"),
    "avg_float": ("out[g] = (double)sum[g] / (double)count[g];", "out[g] = (float)sum[g] / (float)count[g];"),
    "avg_count_index": ("out[g] = (double)sum[g] / (double)count[g];",
                        "out[g] = (double)sum[g] / (double)count[g > 0 ? g - 1 : 0];"),
    "radix_shift": ("return (int64_t)(((uint64_t)key >> shift) & (fanout - 1));",
                    "return (int64_t)(((uint64_t)key >> (shift + 1)) & (fanout - 1));"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(lib), str(mpath)])
    env = dict(os.environ, QE_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
