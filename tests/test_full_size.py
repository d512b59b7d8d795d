"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (its autotuned plans, one batched launch over the whole batch): the
4096-curve uneven TESS/Kepler batch (1.0e8 samples) and 256 curves of
118,000 samples at W = 2161, checked on sampled positions of every curve
(the curve ends, both sides of each gap, and random positions) against the
oracle evaluated one position at a time."""
import numpy as np
import pytest

import bench
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


def sample_positions(x, W, rng, k=6):
    n = x.size
    h = (W - 1) // 2
    pos = [0, 1, n - 2, n - 1, h, n - 1 - h]
    miss = np.isnan(x)
    edges = np.flatnonzero(np.diff(miss.astype(np.int8)))      # last index before a change
    for e in edges[:6]:
        pos += [e - 1, e, e + 1, e + 2]
    pos += list(rng.integers(0, n, k))
    pos = np.unique(np.array(pos, np.int64))
    return pos[(pos >= 0) & (pos < n)]


@pytest.mark.parametrize("workload", ["c3", "c4"])
def test_full_size_batch_sampled(umi, workload):
    b = synth.config3() if workload == "c3" else synth.config4()
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    try:
        umi.clear_tuning()
        flux = torch.from_numpy(b.flux).cuda()
        bench.tune_for_batch(umi, b, W, flux)
        tr, de = umi.detrend_batched(flux, b.offsets, W)
        torch.cuda.synchronize()
        tr, de = tr.cpu().numpy(), de.cpu().numpy()
    finally:
        umi.clear_tuning()
    rng = np.random.default_rng(11)
    for i in range(b.B):
        x = b.curve(i)
        pos = sample_positions(x, int(W[i]), rng)
        ref = oracle.detrend_positions(x, int(W[i]), pos)
        o = b.offsets[i]
        compare_trend(tr[o + pos], ref["trend"], what="%s curve %d" % (workload, i))
        compare_detr(de[o + pos], ref["detr"], what="%s curve %d" % (workload, i))
