"""umi_detrend_batched_noalloc: the batched detrend for callers that cannot
allocate device memory when they call it (a framework's caching allocator
already holds the GPU's memory, a real-time pipeline forbids cudaMalloc /
cudaFree after start-up because they can synchronise the device, or the
stream-ordered pool is disabled).  Its work-queue tables live in a fixed
4 MiB device array inside libumi instead.

These tests call it through the C ABI and compare it with the regular
umi_detrend_batched entry point, within the parity tolerance the other tests
use, on two calls in a row (different batches, so the second call must not
see the first call's tables or counters).  This file is collected last."""
import numpy as np
import pytest

from paper_2604_06602_gb300 import synth
from tests.helpers import compare_detr, compare_trend

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


def test_noalloc_matches_batched_on_two_calls(umi):
    first = synth.config3(n_curves=40)            # windows 25 and 361, uneven lengths
    second = synth.config2(n_curves=12, n=7000)   # fewer tiles than the first call
    for k, b in enumerate((first, second)):
        flux, off, W = _batch(b, umi)
        ref_t, ref_d = umi.detrend_batched(flux, off, W)
        got_t, got_d = umi.detrend_batched_noalloc(flux, off, W)
        torch.cuda.synchronize()
        rt = ref_t.cpu().numpy().astype(np.float64)
        rd = ref_d.cpu().numpy().astype(np.float64)
        compare_trend(got_t.cpu().numpy(), rt, what="no-alloc call %d" % (k + 1))
        compare_detr(got_d.cpu().numpy(), rd, what="no-alloc call %d" % (k + 1))


def test_noalloc_rejects_batches_above_its_limit(umi):
    B = 100000                                    # 48 B per curve alone exceeds 4 MiB
    flux = torch.ones(B, dtype=torch.float32, device="cuda")
    off = np.arange(B + 1, dtype=np.int64)
    W = np.ones(B, np.int32)
    with pytest.raises(umi.UmiError) as e:
        umi.detrend_batched_noalloc(flux, off, W)
    assert e.value.status == umi.UMI_ERR_INVALID_ARG
    assert "no-alloc" in str(e.value)
