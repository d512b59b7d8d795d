"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/umi.h declares, and validates arguments on the host
(no kernel is launched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2604_06602_gb300 import build as libbuild
from paper_2604_06602_gb300 import umi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return umi.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "umi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(umi_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_matches_binding_list():
    assert declared_functions() == sorted(umi.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_window_length_matches_oracle(lib):
    for dt_min in list(np.linspace(0.2, 60.0, 997)) + [2.0, 29.4, 30.0, 20.0 / 60.0]:
        dt = dt_min / 1440.0
        for wd in (0.25, 0.5, 1.5):
            assert umi.window_length(dt, wd) == oracle.window_length(dt, wd)
    assert umi.window_length(0.0) == -1
    assert umi.window_length(float("inf")) == -1


def test_default_params(lib):
    p = umi.default_params()
    assert (p.alpha, p.c, p.iters, p.min_valid) == (2.0, 5.0, 5, -1)
    assert umi.max_window() >= 2161


def test_host_validation_without_gpu(lib):
    p = umi.default_params()
    buf = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    bad = [
        (buf, 100, 4, p),   # even window
        (buf, 100, 0, p),   # zero window
        (buf, -1, 3, p),    # negative length
        (buf, 100, umi.max_window() + 2, p),
    ]
    for flux, n, W, pp in bad:
        st = lib.umi_detrend(flux, n, W, ctypes.byref(pp), buf, buf, None)
        assert st == umi.UMI_ERR_INVALID_ARG
        assert lib.umi_last_error()
    for field, val in (("alpha", 0.0), ("c", -1.0), ("iters", -2), ("min_valid", -5)):
        q = umi.default_params()
        setattr(q, field, val)
        assert lib.umi_detrend(buf, 10, 3, ctypes.byref(q), buf, buf, None) == umi.UMI_ERR_INVALID_ARG
    # n == 0 is a no-op, not an error.
    assert lib.umi_detrend(None, 0, 3, None, None, None, None) == umi.UMI_OK
    # Batched: bad offsets and windows are caught before any device work.
    off = np.array([0, 5, 3], np.int64)
    W = np.array([3, 3], np.int32)
    st = lib.umi_detrend_batched(buf, off.ctypes.data_as(ctypes.c_void_p),
                                 W.ctypes.data_as(ctypes.c_void_p), 2, None, buf, buf, None)
    assert st == umi.UMI_ERR_INVALID_ARG
    off = np.array([1, 5, 8], np.int64)
    st = lib.umi_detrend_batched(buf, off.ctypes.data_as(ctypes.c_void_p),
                                 W.ctypes.data_as(ctypes.c_void_p), 2, None, buf, buf, None)
    assert st == umi.UMI_ERR_INVALID_ARG
    off = np.array([0, 5, 8], np.int64)
    W = np.array([3, 6], np.int32)
    st = lib.umi_detrend_batched(buf, off.ctypes.data_as(ctypes.c_void_p),
                                 W.ctypes.data_as(ctypes.c_void_p), 2, None, buf, buf, None)
    assert st == umi.UMI_ERR_INVALID_ARG
    # The autotuners check the window and the tuning batch's shape first.
    for W_, lens in ((360, [1000] * 4), (361, [1000, 0, 5]), (361, [1000, -3]), (361, [1 << 30] * 3),
                     (0, [10]), (361, [])):
        arr = np.array(lens + [7], np.int64)
        assert lib.umi_autotune_batch(W_, None, arr.ctypes.data_as(ctypes.c_void_p), len(lens),
                                      None, None, None) == umi.UMI_ERR_INVALID_ARG
    assert lib.umi_autotune_batch(361, None, None, 3, None, None, None) == umi.UMI_ERR_INVALID_ARG
    assert lib.umi_autotune(360, 1000, None, None, None) == umi.UMI_ERR_INVALID_ARG
    assert lib.umi_autotune(361, 0, None, None, None) == umi.UMI_ERR_INVALID_ARG


def test_binding_rejects_offsets_past_the_buffers():
    """The C ABI cannot see buffer sizes, so the binding refuses offsets that
    run past the flux buffer, or outputs shorter than the offsets need, before
    it calls the library (on a GPU the kernels would read or write past the
    buffers).  CPU tensors stand in for the device buffers: the size check
    comes before the device-type check."""
    torch = pytest.importorskip("torch")
    flux = torch.ones(100)
    short = torch.empty(50)
    W = np.array([3, 3], np.int32)
    over = np.array([0, 60, 120], np.int64)          # runs 20 samples past flux
    fits = np.array([0, 30, 50], np.int64)
    for fn in (umi.detrend_batched, umi.detrend_batched_noalloc):
        with pytest.raises(ValueError, match="flux holds 100"):
            fn(flux, over, W, trend=torch.empty(120), detr=torch.empty(120))
        with pytest.raises(ValueError, match="trend holds 50"):
            fn(flux, np.array([0, 30, 80], np.int64), W, trend=short, detr=torch.empty(100))
    with pytest.raises(ValueError, match="detr holds 50"):
        umi.detrend_segmented(flux, fits + np.array([0, 0, 30]), W, trend=torch.empty(100), detr=short)
    with pytest.raises(ValueError, match="trend holds 50"):
        umi.detrend(flux, 3, trend=short, detr=torch.empty(100))
    # Host entry point: all buffers on the host, no GPU involved.
    fh = np.ones(100, np.float32)
    with pytest.raises(ValueError, match="flux holds 100"):
        umi.detrend_batched_host(fh, over, W)
    with pytest.raises(ValueError, match="detr holds 50"):
        umi.detrend_batched_host(fh, np.array([0, 30, 80], np.int64), W,
                                 trend=np.empty(80, np.float32), detr=np.empty(50, np.float32))


def test_version(lib):
    assert "sm_103a" in umi.version()


def test_built_for_sm103a_only():
    assert libbuild.ARCH_FLAGS == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_header_is_c99_and_host_calls_work(tmp_path, lib):
    """Compile a C99 program against include/umi.h, link libumi.so and run
    its host-only calls (no GPU needed)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    exe = tmp_path / "c_abi_check"
    libdir = os.path.dirname(umi.lib_path())
    src = os.path.join(ROOT, "tests", "c_abi_check.c")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    src, "-o", str(exe), "-L", libdir, "-lumi", "-Wl,-rpath," + libdir],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert "sm_103a" in r.stdout


def _cuda_home():
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build_c_gpu_program(tmp_path):
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    cuda = _cuda_home()
    exe = tmp_path / "c_abi_gpu"
    libdir = os.path.dirname(umi.lib_path())
    cmd = ["gcc", "-std=gnu11", "-O1", "-Wall", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"),
           os.path.join(ROOT, "tests", "c_abi_gpu.c"), os.path.join(ROOT, "oracle", "umi_oracle.c"),
           "-o", str(exe), "-L", libdir, "-lumi", "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-lm", "-lpthread", "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(cuda, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_gpu_program_builds(tmp_path, lib):
    """The plain-C GPU client compiles and links against libumi and the CUDA
    runtime (running it needs a GPU)."""
    _build_c_gpu_program(tmp_path)


@pytest.mark.gpu
def test_c_gpu_program_runs(tmp_path, lib):
    """A C99 program drives the batched, host-buffer, single-curve and server
    entry points through include/umi.h alone, checked against the C oracle."""
    import subprocess
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _build_c_gpu_program(tmp_path)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr[-3000:])
    assert "c gpu ok" in r.stdout
