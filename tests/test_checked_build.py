"""The checked build (UMI_CHECKED): every kernel checks its shared-memory
tile reads, its work items and its shared-memory size, records failures in
a flag word and skips the access.  It stands in for a device memory checker,
which does not run on this GPU pool.  CPU: the build compiles and reports
itself; GPU: representative calls of every entry point run clean (flag word
0) and match the oracle."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    return shutil.which("nvcc") or (os.path.exists("/usr/local/cuda/bin/nvcc") and "/usr/local/cuda/bin/nvcc")


@pytest.fixture(scope="module")
def checked_lib():
    if not _nvcc():
        pytest.skip("nvcc not available")
    from paper_2604_06602_gb300 import build
    return build.build(checked=True)


def test_checked_build_reports_itself(checked_lib):
    import ctypes
    lib = ctypes.CDLL(checked_lib)
    lib.umi_checked_build.restype = ctypes.c_int32
    assert lib.umi_checked_build() == 1
    # The normal build says it ran no checks.
    from paper_2604_06602_gb300 import umi
    normal = ctypes.CDLL(umi.lib_path())
    normal.umi_checked_build.restype = ctypes.c_int32
    assert normal.umi_checked_build() == 0
    f = ctypes.c_uint32(7)
    assert normal.umi_check_flags(ctypes.byref(f), 0) == 1 and f.value == 0   # UMI_ERR_INVALID_ARG


@pytest.mark.gpu
def test_checked_build_runs_clean(checked_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")],
                       capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["checked"] and res["cases"] > 60 and res["launches"] > 60
    assert res["flags"] == 0
