"""The bounds-checked build (libqe_checked.so, compiled with QE_CHECKED) on
the small parity cases.

compute-sanitizer is not available on the machines these tests target, so
the library carries its own checks: in the checked build every scatter
write of the partition kernels, every row of the partitioned group-by's
segments and every shared-memory slot of the star kernels is tested against
the bound it is derived from, and an index out of bounds records
QE_ERR_DEVICE_CHECK instead of being written.  This test runs the operator,
partitioned group-by and average parity suites in a child process that
loads the checked library (QE_LIB=checked), so every kernel path those
suites reach runs with the checks on and must still match the oracle with no
check firing.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_passes_small_parity_suites():
    env = dict(os.environ, QE_LIB="checked")
    probe = subprocess.run([sys.executable, "-c", "from paper_2506_09226_gb300 import qe; "
                            "print(qe.load_library().qe_build_checked())"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0 and probe.stdout.strip() == "1", probe.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
                        os.path.join("tests", "test_gpu_ops.py"), os.path.join("tests", "test_gpu_part_groupby.py"),
                        os.path.join("tests", "test_gpu_avg.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
