"""FP64 CPU oracle for the UMI sliding-window robust trend.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never imports or links it, and it shares no code with that library.

The arithmetic lives in ``umi_oracle.c`` (plain C, IEEE double): it follows
Section 2 of the paper (window rule, Phase 1 median, Phase 2 upper-RMS scale,
Eq. 1, Phase 3 asymmetric bisquare iterations, Eqs. 2-4) step by step.  This
module only compiles it with gcc and marshals numpy arrays through ctypes.

Pins (tests/test_oracle_pins.py) tie it to the paper's printed values, closed
forms, invariants and brute force; none of them reuse this code's arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "umi_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libumi_oracle.so")
_lock = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile umi_oracle.c with gcc (-O2, no fast-math) into _build/."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.umi_oracle_window_length.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.umi_oracle_window_length.restype = ctypes.c_int
        lib.umi_oracle_weight.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.umi_oracle_weight.restype = ctypes.c_double
        lib.umi_oracle_window_estimate.argtypes = [
            _f64p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.umi_oracle_window_estimate.restype = ctypes.c_int
        lib.umi_oracle_detrend.argtypes = [
            _f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p, _i32p, _i32p, _f64p]
        lib.umi_oracle_detrend.restype = ctypes.c_int
        lib.umi_oracle_window_estimate_mode.argtypes = [
            _f64p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.umi_oracle_window_estimate_mode.restype = ctypes.c_int
        lib.umi_oracle_detrend_mode.argtypes = [
            _f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p, _i32p, _i32p, _f64p]
        lib.umi_oracle_detrend_mode.restype = ctypes.c_int
        lib.umi_oracle_detrend_positions.argtypes = [
            _f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, _i64p, ctypes.c_int64, _f64p, _f64p, _f64p, _i32p,
            _i32p, _f64p]
        lib.umi_oracle_detrend_positions.restype = ctypes.c_int
        lib.umi_oracle_detrend_segmented.argtypes = [
            _f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _f64p, _f64p]
        lib.umi_oracle_detrend_segmented.restype = ctypes.c_int
        lib.umi_oracle_detrend_batch.argtypes = [
            _f32p, _i64p, _i32p, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, _f64p, _f64p, ctypes.c_int]
        lib.umi_oracle_detrend_batch.restype = ctypes.c_int
        _lib = lib
        return lib


def window_length(cadence_days: float, window_days: float = 0.5) -> int:
    """W = round(window / cadence) | 1 (Section 2 opening paragraph); -1 if invalid."""
    return int(_load().umi_oracle_window_length(float(cadence_days), float(window_days)))


def weight(u: float, alpha: float) -> float:
    """Asymmetric bisquare weight of a standardised residual u (Eqs. 2-3)."""
    return float(_load().umi_oracle_weight(float(u), float(alpha)))


SCALE_UPPER_RMS = 0
SCALE_MAD = 1


def window_estimate(values, alpha=2.0, c=5.0, iters=5, scale_mode=SCALE_UPPER_RMS):
    """One window given as its valid samples.

    Returns (median, n_plus, s, mu) after Phases 1-3 of Section 2; scale_mode
    1 uses the MAD instead of the upper-RMS scale.
    """
    v = np.array(values, dtype=np.float64).ravel().copy()
    m, s, mu = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    npl = ctypes.c_int()
    rc = _load().umi_oracle_window_estimate_mode(v, int(v.size), float(alpha), float(c), int(iters),
                                                 int(scale_mode), ctypes.byref(m), ctypes.byref(npl),
                                                 ctypes.byref(s), ctypes.byref(mu))
    if rc != 0:
        raise ValueError("window_estimate needs at least one value")
    return m.value, npl.value, s.value, mu.value


def detrend(flux, W, alpha=2.0, c=5.0, iters=5, min_valid=-1, scale_mode=SCALE_UPPER_RMS):
    """Whole curve.  Returns a dict of float64/int32 arrays:
    trend, detr, median, nvalid, nplus, scale (see umi_oracle.c)."""
    x = np.ascontiguousarray(flux, dtype=np.float32)
    n = x.size
    out = {k: np.empty(n, np.float64) for k in ("trend", "detr", "median", "scale")}
    out.update({k: np.empty(n, np.int32) for k in ("nvalid", "nplus")})
    rc = _load().umi_oracle_detrend_mode(x, n, int(W), float(alpha), float(c), int(iters),
                                         int(min_valid), int(scale_mode), out["trend"], out["detr"],
                                         out["median"], out["nvalid"], out["nplus"], out["scale"])
    if rc != 0:
        raise ValueError("invalid oracle arguments")
    return out


def detrend_positions(flux, W, positions, alpha=2.0, c=5.0, iters=5, min_valid=-1):
    """Selected positions of one curve; arrays indexed like ``positions``."""
    x = np.ascontiguousarray(flux, dtype=np.float32)
    pos = np.ascontiguousarray(positions, dtype=np.int64)
    q = pos.size
    out = {k: np.empty(q, np.float64) for k in ("trend", "detr", "median", "scale")}
    out.update({k: np.empty(q, np.int32) for k in ("nvalid", "nplus")})
    rc = _load().umi_oracle_detrend_positions(x, x.size, int(W), float(alpha), float(c),
                                              int(iters), int(min_valid), pos, q,
                                              out["trend"], out["detr"], out["median"],
                                              out["nvalid"], out["nplus"], out["scale"])
    if rc != 0:
        raise ValueError("invalid oracle arguments")
    return out


def detrend_segmented(flux, W, gap_min=0, min_seg=-1, alpha=2.0, c=5.0, iters=5, min_valid=-1):
    """Gap-split detrend of one curve: segments end at runs of >= gap_min
    missing samples (0 means W); segments with < min_seg valid samples (-1
    means W // 3) are dropped.  Returns (trend, detr, kept_segments)."""
    x = np.ascontiguousarray(flux, dtype=np.float32)
    trend = np.empty(x.size, np.float64)
    detr = np.empty(x.size, np.float64)
    kept = _load().umi_oracle_detrend_segmented(x, x.size, int(W), float(alpha), float(c), int(iters),
                                                int(min_valid), int(gap_min), int(min_seg), trend, detr)
    if kept < 0:
        raise ValueError("invalid oracle arguments")
    return trend, detr, kept


def detrend_batch(flux, offsets, W, alpha=2.0, c=5.0, iters=5, min_valid=-1, nthreads=None):
    """CSR batch (flux[offsets[b]:offsets[b+1]] is curve b, window W[b]).

    Runs one curve per task over ``nthreads`` pthreads.  Returns (trend, detr).
    """
    x = np.ascontiguousarray(flux, dtype=np.float32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    w = np.ascontiguousarray(W, dtype=np.int32)
    B = off.size - 1
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    trend = np.empty(x.size, np.float64)
    detr = np.empty(x.size, np.float64)
    rc = _load().umi_oracle_detrend_batch(x, off, w, B, float(alpha), float(c), int(iters),
                                          int(min_valid), trend, detr, int(nthreads))
    if rc != 0:
        raise ValueError("invalid oracle arguments")
    return trend, detr
