"""umi_detrend_batched_noalloc: the batched detrend for callers that cannot
allocate device memory when they call it (a framework's caching allocator
already holds the GPU's memory, a real-time pipeline forbids cudaMalloc /
cudaFree after start-up because they can synchronise the device, or the
stream-ordered pool is disabled).  Its work-queue tables live in a fixed
4 MiB device array inside libumi instead.

These tests call it through the C ABI.  It plans the same bands as the
regular umi_detrend_batched entry point and runs the same kernels on them, so
its outputs must equal that entry point's bit for bit; this is checked on
three calls in a row with different batches, so a later call must not see an
earlier call's tables or counters.  A warmed-up call must leave the device's
memory untouched.  This file is collected last."""
import ctypes

import numpy as np
import pytest

from paper_2604_06602_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def umi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_06602_gb300 import umi as u
    u.load(build_if_missing=True)
    return u


def _batch(b, umi):
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    return torch.from_numpy(b.flux).cuda(), b.offsets, W


def _bits(t):
    return t.view(torch.int32)


def test_noalloc_equals_batched_bit_for_bit_on_consecutive_calls(umi):
    batches = [synth.config3(n_curves=40),          # windows 25 and 361, uneven lengths
               synth.config2(n_curves=12, n=7000),  # fewer tiles than the first call
               synth.config3(n_curves=300)]         # tables of about 90 KB: several writer kernels
    for k, b in enumerate(batches):
        flux, off, W = _batch(b, umi)
        ref_t, ref_d = umi.detrend_batched(flux, off, W)
        got_t, got_d = umi.detrend_batched_noalloc(flux, off, W)
        torch.cuda.synchronize()
        assert torch.equal(_bits(got_t), _bits(ref_t)), "trend differs on call %d" % (k + 1)
        assert torch.equal(_bits(got_d), _bits(ref_d)), "detr differs on call %d" % (k + 1)
        assert torch.isfinite(got_t).any()


class _DefaultPool:
    """Used and reserved bytes of the device's default stream-ordered memory
    pool (the pool cudaMallocAsync draws from), through the driver API."""
    USED_MEM_CURRENT, USED_MEM_HIGH, RESERVED_MEM_CURRENT = 7, 8, 5

    def __init__(self, ordinal):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ctypes.c_int(ordinal)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, ctypes.c_int(attr), ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, ctypes.c_int(self.USED_MEM_HIGH),
                                             ctypes.byref(zero)) == 0


def test_noalloc_call_allocates_no_device_memory(umi):
    b = synth.config3(n_curves=64)
    flux, off, W = _batch(b, umi)
    trend = torch.empty_like(flux)
    detr = torch.empty_like(flux)
    for _ in range(2):                               # warm-up: kernels loaded, array address known
        umi.detrend_batched_noalloc(flux, off, W, trend=trend, detr=detr)
    torch.cuda.synchronize()
    pool = _DefaultPool(torch.cuda.current_device())
    pool.reset_high()
    used0 = pool.get(pool.USED_MEM_CURRENT)
    reserved0 = pool.get(pool.RESERVED_MEM_CURRENT)
    torch_alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        umi.detrend_batched_noalloc(flux, off, W, trend=trend, detr=detr)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) <= used0, "the call drew on the stream-ordered pool"
    assert pool.get(pool.RESERVED_MEM_CURRENT) == reserved0
    assert torch.cuda.memory_allocated() == torch_alloc0
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "device free memory changed by %d bytes" % (free0 - free1)


def test_noalloc_rejects_batches_above_its_limit(umi):
    B = 100000                                    # 56 B per curve alone exceeds 4 MiB
    flux = torch.ones(B, dtype=torch.float32, device="cuda")
    off = np.arange(B + 1, dtype=np.int64)
    W = np.ones(B, np.int32)
    with pytest.raises(umi.UmiError) as e:
        umi.detrend_batched_noalloc(flux, off, W)
    assert e.value.status == umi.UMI_ERR_INVALID_ARG
    assert "no-alloc" in str(e.value)
