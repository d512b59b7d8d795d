"""Thin ctypes binding of libumi.so (include/umi.h).

Argument marshalling only: every step of the detrend runs inside libumi's CUDA
kernels.  Device buffers are torch CUDA tensors (float32, contiguous); streams
are torch CUDA streams (the current stream by default).  If libumi.so is not
built, or no GPU is present, calls raise instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

UMI_OK = 0
UMI_ERR_INVALID_ARG = 1
UMI_ERR_CUDA = 2
UMI_ERR_OOM = 3
UMI_ERR_BUSY = 4
UMI_ERR_NOT_READY = 5
UMI_ERR_TIMEOUT = 6
UMI_ERR_UNKNOWN_TICKET = 7
UMI_ERR_FAILED = 8

STATUS_NAMES = {0: "UMI_OK", 1: "UMI_ERR_INVALID_ARG", 2: "UMI_ERR_CUDA", 3: "UMI_ERR_OOM",
                4: "UMI_ERR_BUSY", 5: "UMI_ERR_NOT_READY", 6: "UMI_ERR_TIMEOUT",
                7: "UMI_ERR_UNKNOWN_TICKET", 8: "UMI_ERR_FAILED"}

# Every function include/umi.h declares (checked by the ABI test).
EXPORTS = [
    "umi_default_params", "umi_window_length", "umi_detrend", "umi_detrend_batched",
    "umi_detrend_batched_host", "umi_detrend_batched_noalloc", "umi_detrend_diag", "umi_max_window", "umi_get_plan",
    "umi_autotune", "umi_autotune_batch", "umi_save_tuning", "umi_load_tuning", "umi_clear_tuning",
    "umi_set_graph_cache", "umi_server_default_config", "umi_server_create", "umi_server_submit",
    "umi_server_poll", "umi_server_wait", "umi_server_copy_out", "umi_server_release",
    "umi_server_get_stats", "umi_server_inject_fault", "umi_server_destroy", "umi_last_error",
    "umi_version", "umi_kernel_launch_count", "umi_default_segment_params",
    "umi_detrend_segmented", "umi_checked_build", "umi_check_flags", "umi_server_timeline",
]


class UmiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


SCALE_UPPER_RMS = 0
SCALE_MAD = 1


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("c", ctypes.c_float), ("iters", ctypes.c_int32),
                ("min_valid", ctypes.c_int32), ("scale_mode", ctypes.c_int32)]


class Plan(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("slots", ctypes.c_int32), ("chain", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("variant", ctypes.c_int32), ("latency", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SegmentParams(ctypes.Structure):
    _fields_ = [("gap_min", ctypes.c_int64), ("min_seg", ctypes.c_int64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("max_batch_curves", ctypes.c_int32),
                ("device", ctypes.c_int32), ("max_wait_s", ctypes.c_double),
                ("busy_poll", ctypes.c_int32), ("batch_by_window", ctypes.c_int32),
                ("priority_window", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("released", ctypes.c_uint64),
                ("batches_launched", ctypes.c_uint64), ("resident_bytes", ctypes.c_uint64),
                ("peak_resident_bytes", ctypes.c_uint64), ("queued_requests", ctypes.c_uint64),
                ("mean_batch_curves", ctypes.c_double), ("launch_host_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libumi.so (optionally building it first)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libumi.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2604_06602_gb300.build)")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        sig = {
            "umi_default_params": (None, [P(Params)]),
            "umi_window_length": (_i32, [ctypes.c_double, ctypes.c_double]),
            "umi_detrend": (ctypes.c_int, [_vp, _i64, _i32, P(Params), _vp, _vp, _vp]),
            "umi_detrend_batched": (ctypes.c_int, [_vp, _vp, _vp, _i32, P(Params), _vp, _vp, _vp]),
            "umi_detrend_batched_host": (ctypes.c_int, [_vp, _vp, _vp, _i32, P(Params), _vp, _vp, _vp]),
            "umi_detrend_batched_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _i32, P(Params), _vp, _vp,
                                                           _vp]),
            "umi_detrend_diag": (ctypes.c_int, [_vp, _i64, _i32, P(Params), _vp, _vp, _vp, _vp, _vp,
                                                _vp, _vp]),
            "umi_max_window": (_i32, []),
            "umi_get_plan": (ctypes.c_int, [_i32, _i64, P(Plan)]),
            "umi_autotune": (ctypes.c_int, [_i32, _i64, _vp, P(Plan), P(ctypes.c_double)]),
            "umi_autotune_batch": (ctypes.c_int, [_i32, _vp, _vp, _i32, _vp, P(Plan), P(ctypes.c_double)]),
            "umi_save_tuning": (ctypes.c_int, [ctypes.c_char_p]),
            "umi_load_tuning": (ctypes.c_int, [ctypes.c_char_p]),
            "umi_clear_tuning": (None, []),
            "umi_set_graph_cache": (None, [ctypes.c_int]),
            "umi_server_default_config": (None, [P(ServerConfig)]),
            "umi_server_create": (ctypes.c_int, [P(ServerConfig), P(_vp)]),
            "umi_server_submit": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _i64, _i32, P(Params),
                                                 P(ctypes.c_uint64)]),
            "umi_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, P(_vp), P(_vp), P(ctypes.c_double)]),
            "umi_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double]),
            "umi_server_timeline": (ctypes.c_int, [_vp, ctypes.c_uint64, P(ctypes.c_double),
                                                   P(ctypes.c_double), P(ctypes.c_double)]),
            "umi_server_copy_out": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, _vp]),
            "umi_server_release": (ctypes.c_int, [_vp, ctypes.c_uint64]),
            "umi_server_get_stats": (ctypes.c_int, [_vp, P(ServerStats)]),
            "umi_server_inject_fault": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
            "umi_server_destroy": (None, [_vp]),
            "umi_last_error": (ctypes.c_char_p, []),
            "umi_version": (ctypes.c_char_p, []),
            "umi_kernel_launch_count": (ctypes.c_longlong, []),
            "umi_checked_build": (_i32, []),
            "umi_check_flags": (ctypes.c_int, [P(ctypes.c_uint32), _i32]),
            "umi_default_segment_params": (None, [P(SegmentParams)]),
            "umi_detrend_segmented": (ctypes.c_int, [_vp, _vp, _vp, _i32, P(Params), P(SegmentParams),
                                                     _vp, _vp, P(ctypes.c_int64), _vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(status):
    if status != UMI_OK:
        msg = load().umi_last_error()
        raise UmiError(status, msg.decode() if msg else "")
    return status


def params(alpha=2.0, c=5.0, iters=5, min_valid=-1, scale_mode=SCALE_UPPER_RMS) -> Params:
    return Params(float(alpha), float(c), int(iters), int(min_valid), int(scale_mode))


def default_params() -> Params:
    p = Params()
    load().umi_default_params(ctypes.byref(p))
    return p


def window_length(cadence_days: float, window_days: float = 0.5) -> int:
    return int(load().umi_window_length(float(cadence_days), float(window_days)))


def max_window() -> int:
    return int(load().umi_max_window())


def version() -> str:
    return load().umi_version().decode()


def kernel_launch_count() -> int:
    return int(load().umi_kernel_launch_count())


def checked_build() -> bool:
    """True when the loaded library is the UMI_CHECKED build."""
    return bool(load().umi_checked_build())


def check_flags(clear=False) -> int:
    """Checked builds: the current device's flag word of failed index checks."""
    f = ctypes.c_uint32()
    _check(load().umi_check_flags(ctypes.byref(f), int(bool(clear))))
    return int(f.value)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_f32(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def detrend(flux, W, p: Params | None = None, trend=None, detr=None, stream=None):
    """One curve on the GPU.  Returns (trend, detr) float32 CUDA tensors."""
    import torch
    n = flux.numel()
    trend = torch.empty_like(flux) if trend is None else trend
    detr = torch.empty_like(flux) if detr is None else detr
    _check_sizes(n, trend=trend, detr=detr)
    _check(load().umi_detrend(_dev_f32(flux, "flux"), n, int(W), None if p is None else ctypes.byref(p),
                              _dev_f32(trend, "trend"), _dev_f32(detr, "detr"), _stream_handle(stream)))
    return trend, detr


def detrend_diag(flux, W, p: Params | None = None, stream=None):
    """One curve with diagnostics.  Returns a dict of CUDA tensors:
    trend, detr, median, nvalid, nplus, scale."""
    import torch
    n = flux.numel()
    out = {"trend": torch.empty_like(flux), "detr": torch.empty_like(flux),
           "median": torch.empty_like(flux), "scale": torch.empty_like(flux),
           "nvalid": torch.empty(n, dtype=torch.int32, device=flux.device),
           "nplus": torch.empty(n, dtype=torch.int32, device=flux.device)}
    _check(load().umi_detrend_diag(_dev_f32(flux, "flux"), n, int(W),
                                   None if p is None else ctypes.byref(p),
                                   _dev_f32(out["trend"], "trend"), _dev_f32(out["detr"], "detr"),
                                   ctypes.c_void_p(out["median"].data_ptr()),
                                   ctypes.c_void_p(out["nvalid"].data_ptr()),
                                   ctypes.c_void_p(out["nplus"].data_ptr()),
                                   ctypes.c_void_p(out["scale"].data_ptr()), _stream_handle(stream)))
    return out


def _host_i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _host_i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _check_sizes(total, **bufs):
    """The C ABI takes bare pointers and cannot see buffer sizes: refuse, before
    anything is launched, offsets that run past the flux buffer and outputs too
    short for them (the kernels would read or write past their ends)."""
    for name, b in bufs.items():
        size = b.numel() if hasattr(b, "numel") else int(np.asarray(b).size)
        if size < total:
            raise ValueError("%s holds %d samples but the offsets (or n) need %d" % (name, size, total))


def _csr_total(off):
    if off.size < 1:
        raise ValueError("offsets must hold B + 1 >= 1 entries")
    return int(off.max())


def detrend_batched(flux, offsets, W, p: Params | None = None, trend=None, detr=None, stream=None):
    """CSR batch on the GPU.  `offsets` [B+1] and `W` [B] are host arrays."""
    import torch
    off, offp = _host_i64(offsets)
    w, wp = _host_i32(W)
    B = off.size - 1
    if w.size != B:
        raise ValueError("W must have one entry per curve")
    trend = torch.empty_like(flux) if trend is None else trend
    detr = torch.empty_like(flux) if detr is None else detr
    _check_sizes(_csr_total(off), flux=flux, trend=trend, detr=detr)
    _check(load().umi_detrend_batched(_dev_f32(flux, "flux"), offp, wp, B,
                                      None if p is None else ctypes.byref(p),
                                      _dev_f32(trend, "trend"), _dev_f32(detr, "detr"),
                                      _stream_handle(stream)))
    return trend, detr


def detrend_batched_noalloc(flux, offsets, W, p: Params | None = None, trend=None, detr=None,
                            stream=None):
    """CSR batch through umi_detrend_batched_noalloc: the library allocates no
    device memory for it (its work-queue tables go to a fixed 4 MiB device
    array), for callers that cannot allocate at this point.  Calls that
    overlap on the GPU share that array; keep them on one stream."""
    import torch
    off, offp = _host_i64(offsets)
    w, wp = _host_i32(W)
    B = off.size - 1
    if w.size != B:
        raise ValueError("W must have one entry per curve")
    trend = torch.empty_like(flux) if trend is None else trend
    detr = torch.empty_like(flux) if detr is None else detr
    _check_sizes(_csr_total(off), flux=flux, trend=trend, detr=detr)
    _check(load().umi_detrend_batched_noalloc(_dev_f32(flux, "flux"), offp, wp, B,
                                              None if p is None else ctypes.byref(p),
                                              _dev_f32(trend, "trend"), _dev_f32(detr, "detr"),
                                              _stream_handle(stream)))
    return trend, detr


def detrend_segmented(flux, offsets, W, p: Params | None = None, gap_min=0, min_seg=-1, trend=None,
                      detr=None, stream=None):
    """CSR batch with gap handling (umi_detrend_segmented).  Returns
    (trend, detr, kept_segments).  Synchronises the stream once (segment scan)."""
    import torch
    off, offp = _host_i64(offsets)
    w, wp = _host_i32(W)
    B = off.size - 1
    if w.size != B:
        raise ValueError("W must have one entry per curve")
    trend = torch.empty_like(flux) if trend is None else trend
    detr = torch.empty_like(flux) if detr is None else detr
    _check_sizes(_csr_total(off), flux=flux, trend=trend, detr=detr)
    sp = SegmentParams(int(gap_min), int(min_seg))
    kept = ctypes.c_int64()
    _check(load().umi_detrend_segmented(_dev_f32(flux, "flux"), offp, wp, B,
                                        None if p is None else ctypes.byref(p), ctypes.byref(sp),
                                        _dev_f32(trend, "trend"), _dev_f32(detr, "detr"),
                                        ctypes.byref(kept), _stream_handle(stream)))
    return trend, detr, kept.value


def detrend_batched_host(flux, offsets, W, p: Params | None = None, trend=None, detr=None,
                         stream=None):
    """CSR batch from host memory (numpy or pinned torch CPU tensors); blocks
    until the results are back on the host."""
    import torch

    def host_ptr(a, name):
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
                raise TypeError("%s must be a contiguous float32 CPU tensor" % name)
            return ctypes.c_void_p(a.data_ptr())
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError("%s must be a contiguous float32 array" % name)
        return a.ctypes.data_as(ctypes.c_void_p)

    off, offp = _host_i64(offsets)
    w, wp = _host_i32(W)
    B = off.size - 1
    if w.size != B:
        raise ValueError("W must have one entry per curve")
    total = _csr_total(off)
    if trend is None:
        trend = np.empty(total, np.float32)
    if detr is None:
        detr = np.empty(total, np.float32)
    _check_sizes(total, flux=flux, trend=trend, detr=detr)
    _check(load().umi_detrend_batched_host(host_ptr(flux, "flux"), offp, wp, B,
                                           None if p is None else ctypes.byref(p),
                                           host_ptr(trend, "trend"), host_ptr(detr, "detr"),
                                           _stream_handle(stream)))
    return trend, detr


def get_plan(W, positions=-1) -> dict:
    pl = Plan()
    _check(load().umi_get_plan(int(W), int(positions), ctypes.byref(pl)))
    return pl.as_dict()


def autotune(W, positions=2_000_000, stream=None):
    pl = Plan()
    ms = ctypes.c_double()
    _check(load().umi_autotune(int(W), int(positions), _stream_handle(stream), ctypes.byref(pl),
                               ctypes.byref(ms)))
    return pl.as_dict(), ms.value


def autotune_batch(W, curve_lengths, flux=None, stream=None):
    """Tune W's plan on a batch of curves of the given lengths (the tile
    rounding at every curve's end counts): the curves in `flux` (a CUDA
    float32 tensor holding them back to back), or synthetic noise."""
    lens = np.ascontiguousarray(curve_lengths, np.int64)
    if lens.ndim != 1 or lens.size == 0:
        raise ValueError("curve_lengths must be a non-empty 1-D sequence")
    ptr = None
    if flux is not None:
        import torch
        if flux.dtype != torch.float32 or not flux.is_cuda or not flux.is_contiguous():
            raise ValueError("flux must be a contiguous float32 CUDA tensor")
        _check_sizes(int(lens.sum()), flux=flux)
        ptr = flux.data_ptr()
    pl = Plan()
    ms = ctypes.c_double()
    _check(load().umi_autotune_batch(int(W), ptr, lens.ctypes.data_as(ctypes.c_void_p), int(lens.size),
                                     _stream_handle(stream), ctypes.byref(pl), ctypes.byref(ms)))
    return pl.as_dict(), ms.value


def save_tuning(path):
    _check(load().umi_save_tuning(str(path).encode()))


def load_tuning(path):
    _check(load().umi_load_tuning(str(path).encode()))


def clear_tuning():
    load().umi_clear_tuning()


def set_graph_cache(enabled: bool):
    load().umi_set_graph_cache(1 if enabled else 0)


class Server:
    """Continuous-batching server (umi_server_*)."""

    def __init__(self, mem_budget_bytes=None, max_slots=None, n_streams=None, max_batch_curves=None,
                 device=0, max_wait_s=None, busy_poll=None, batch_by_window=None,
                 priority_window=None):
        cfg = ServerConfig()
        load().umi_server_default_config(ctypes.byref(cfg))
        if mem_budget_bytes is not None:
            cfg.mem_budget_bytes = int(mem_budget_bytes)
        if max_slots is not None:
            cfg.max_slots = int(max_slots)
        if n_streams is not None:
            cfg.n_streams = int(n_streams)
        if max_batch_curves is not None:
            cfg.max_batch_curves = int(max_batch_curves)
        if max_wait_s is not None:
            cfg.max_wait_s = float(max_wait_s)
        if busy_poll is not None:
            cfg.busy_poll = int(busy_poll)
        if batch_by_window is not None:
            cfg.batch_by_window = int(batch_by_window)
        if priority_window is not None:
            cfg.priority_window = int(priority_window)
        cfg.device = int(device)
        h = ctypes.c_void_p()
        _check(load().umi_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.config = cfg

    def submit(self, flux, W, p: Params | None = None) -> int:
        """Queue a curve (numpy float32 / CPU tensor, or CUDA tensor kept alive
        by the caller until the ticket is done)."""
        import torch
        t = ctypes.c_uint64()
        if isinstance(flux, torch.Tensor) and flux.is_cuda:
            ptr, is_dev, n = _dev_f32(flux, "flux"), 1, flux.numel()
        else:
            a = flux.numpy() if isinstance(flux, torch.Tensor) else flux
            if a.dtype != np.float32 or not a.flags.c_contiguous:
                raise TypeError("flux must be contiguous float32")
            ptr, is_dev, n = a.ctypes.data_as(ctypes.c_void_p), 0, a.size
        _check(load().umi_server_submit(self._h, ptr, is_dev, n, int(W),
                                        None if p is None else ctypes.byref(p), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        """Returns None while not ready, else (trend_ptr, detr_ptr, latency_s)."""
        tr, de, lat = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_double()
        st = load().umi_server_poll(self._h, ticket, ctypes.byref(tr), ctypes.byref(de), ctypes.byref(lat))
        if st == UMI_ERR_NOT_READY:
            return None
        _check(st)
        return tr.value, de.value, lat.value

    def wait(self, ticket, timeout_s=60.0):
        _check(load().umi_server_wait(self._h, ticket, float(timeout_s)))

    def timeline(self, ticket):
        """None while not ready, else seconds after submit: {admit, launch, done}."""
        a, l, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = load().umi_server_timeline(self._h, ticket, ctypes.byref(a), ctypes.byref(l), ctypes.byref(d))
        if st == UMI_ERR_NOT_READY:
            return None
        _check(st)
        return {"admit": a.value, "launch": l.value, "done": d.value}

    def copy_out(self, ticket, n):
        trend = np.empty(n, np.float32)
        detr = np.empty(n, np.float32)
        _check(load().umi_server_copy_out(self._h, ticket, trend.ctypes.data_as(ctypes.c_void_p),
                                          detr.ctypes.data_as(ctypes.c_void_p)))
        return trend, detr

    def release(self, ticket):
        _check(load().umi_server_release(self._h, ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().umi_server_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def inject_fault(self, kind, count):
        _check(load().umi_server_inject_fault(self._h, int(kind), int(count)))

    def close(self):
        if self._h:
            load().umi_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
