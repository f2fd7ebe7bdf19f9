"""Host-side checks that need no GPU: the C ABI library loads and exports
every entry point qe.h declares, the ctypes mirrors of the ABI structs match
the C layout (compiled with gcc from qe.h), and the autotuner's search and
cache logic."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2506_09226_gb300 import qe, tune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "qe.h")
HDRS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))
LIB = os.path.join(ROOT, "paper_2506_09226_gb300", "libqe.so")


def declared_functions():
    src = "".join(open(h).read() for h in HDRS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qe_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2506_09226_gb300 import build
        build.build()
    return qe.load_library()


def test_library_exports_every_declared_entry_point(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(qe.EXPORTED) <= set(names)        # the binding declares nothing the header lacks


def test_checked_build_is_marked(lib):
    """libqe.so is the plain build and libqe_checked.so the bounds-checked one."""
    assert lib.qe_build_checked() == 0
    chk = os.path.join(ROOT, "paper_2506_09226_gb300", "libqe_checked.so")
    if not os.path.exists(chk):
        from paper_2506_09226_gb300 import build
        build.build()
    c = ctypes.CDLL(chk)
    c.qe_build_checked.restype = ctypes.c_int
    assert c.qe_build_checked() == 1


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.qe_create(ctypes.byref(h), 0, 0) == qe.ERR_NO_DEVICE


STRUCTS = {
    "qe_col": qe.qe_col, "qe_pred": qe.qe_pred, "qe_groups_out": qe.qe_groups_out,
    "qe_build_opts": qe.qe_build_opts, "qe_ht_info": qe.qe_ht_info, "qe_agg": qe.qe_agg,
    "qe_agg_spec": qe.qe_agg_spec, "qe_pipeline_desc": qe.qe_pipeline_desc, "qe_batch_opts": qe.qe_batch_opts,
    "qe_link": qe.qe_link, "qe_cluster": qe.qe_cluster,
}


def test_ctypes_layouts_match_header(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qe.h"', '#include "qe_plan.h"',
             "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HDR), "-o", str(exe), str(c)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    for line in filter(None, out):
        name, field, val = line.split()
        cls = STRUCTS[name]
        got = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(val), (name, field, got, val)


def test_autotuner_search_and_cache(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def time_one(c):
        calls.append(c)
        return {(1, 0): 5.0, (2, 0): 3.0, (2, -1): 4.0}[c]
    best = tune.search("k", [(1, 0), (2, 0), (2, -1)], time_one, path)
    assert best == (2, 0) and len(calls) == 3
    best2 = tune.search("k", [(1, 0), (2, 0), (2, -1)], lambda c: 1 / 0, path)   # cached: no timing
    assert best2 == (2, 0)
    assert tune.search("j", [3, 2], lambda c: c, path) == 2
    assert tune.batch_bucket([1000, 10 ** 7]) != tune.batch_bucket([1000, 2000])
