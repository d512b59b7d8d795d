"""Gap handling on the GPU (umi_detrend_segmented) against the oracle's
segmented detrend: same kept-segment count, NaN outside kept segments, trend
within 1e-5 relative inside them."""
import numpy as np
import pytest

import oracle
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


def gappy_curve(seed, n, W):
    rng = np.random.default_rng(seed)
    x = synth.random_curve(seed, n)
    for _ in range(int(rng.integers(2, 12))):
        s0 = int(rng.integers(0, n))
        x[s0:s0 + int(rng.integers(1, 3 * W))] = np.nan
    x[rng.uniform(size=n) < 0.02] = np.nan
    return x


@pytest.mark.parametrize("W,gap_min,min_seg", [(361, 0, -1), (361, 40, 120), (25, 0, -1),
                                               (25, 3, 0), (7, 1, 2), (2161, 0, 3000),
                                               (61, 64, -1)])
def test_segmented_matches_oracle(umi, W, gap_min, min_seg):
    lens = [1, 5, 3 * W + 7, 20000, 777, 9000]
    xs = [gappy_curve(10 * W + k, n, W) for k, n in enumerate(lens)]
    xs[1][:] = np.nan                                  # an all-missing curve
    flux = np.concatenate(xs).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    Wv = np.full(len(lens), W, np.int32)
    tr, de, kept = umi.detrend_segmented(torch.from_numpy(flux).cuda(), off, Wv,
                                         gap_min=gap_min, min_seg=min_seg)
    torch.cuda.synchronize()
    tr, de = tr.cpu().numpy(), de.cpu().numpy()
    total_kept = 0
    for k, x in enumerate(xs):
        rt, rd, rk = oracle.detrend_segmented(x, W, gap_min=gap_min, min_seg=min_seg)
        total_kept += rk
        s = slice(off[k], off[k + 1])
        compare_trend(tr[s], rt, what="curve %d" % k)
        compare_detr(de[s], rd, what="curve %d" % k)
    assert kept == total_kept


def test_segmented_kepler_batch(umi):
    """Kepler-like curves with 3-day gaps every ~90 d and a short-gap split."""
    b = synth.config3(n_curves=40)
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    flux = torch.from_numpy(b.flux).cuda()
    for gap_min in (0, 10):
        tr, _, kept = umi.detrend_segmented(flux, b.offsets, W, gap_min=gap_min)
        torch.cuda.synchronize()
        tr = tr.cpu().numpy()
        n_ref = 0
        for i in range(b.B):
            rt, _, rk = oracle.detrend_segmented(b.curve(i), W[i], gap_min=gap_min)
            n_ref += rk
            compare_trend(tr[b.offsets[i]:b.offsets[i + 1]], rt, what="curve %d gap_min %d" % (i, gap_min))
        assert kept == n_ref


def test_segmented_defaults_equal_plain_batched(umi):
    """With gap_min = W and min_seg = W/3 splitting changes nothing (windows
    cannot span a gap of W samples, and shorter islands already fail the
    per-window minimum), so the output equals the plain batched path."""
    b = synth.config3(n_curves=24)
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    flux = torch.from_numpy(b.flux).cuda()
    t1, d1, _ = umi.detrend_segmented(flux, b.offsets, W)
    t0, d0 = umi.detrend_batched(flux, b.offsets, W)
    torch.cuda.synchronize()
    assert torch.equal(torch.nan_to_num(t1, 3.0), torch.nan_to_num(t0, 3.0))
    assert torch.equal(torch.nan_to_num(d1, 3.0), torch.nan_to_num(d0, 3.0))
