"""Host-side pieces of bench.py and the serving stream generator, on CPU: the
sampled oracle check the benchmark reports for every workload accepts the
oracle's own outputs and rejects a planted error; steady-state latency
percentiles drop the first second; the serving stream follows its mixture and
every request's flux is a slice inside its class's tape; the kernel code hash
that keys the measured traffic ignores comments; each band is tuned on its
own curves."""
import numpy as np
import pytest

import bench
import oracle
from paper_2604_06602_gb300 import synth


def _oracle_outputs(b, W):
    trend = np.empty(b.flux.size, np.float32)
    detr = np.empty(b.flux.size, np.float32)
    for i in range(b.B):
        o, e = b.offsets[i], b.offsets[i + 1]
        r = oracle.detrend(b.curve(i), int(W[i]))
        trend[o:e] = r["trend"]
        detr[o:e] = r["detr"]
    return trend, detr


def test_sampled_parity_accepts_oracle_and_catches_a_planted_error():
    b = synth.config3(n_curves=6)
    W = np.array([oracle.window_length(c) for c in b.cadence], np.int32)
    trend, detr = _oracle_outputs(b, W)
    res = bench.sampled_parity(b, W, trend, detr)
    assert res["ok"] and res["nan_pattern_equal"] and res["curves"] == 6
    assert res["max_rel_err_trend"] < 1e-7          # float32 rounding of the FP64 values
    # A planted error of 3e-5 relative at the first sampled position of curve 2.
    pos = bench.sample_positions(b.curve(2), int(W[2]), np.random.default_rng(0))
    k = b.offsets[2] + next(p for p in pos if np.isfinite(trend[b.offsets[2] + p]))
    bad = trend.copy()
    bad[k] *= np.float32(1 + 3e-5)
    res = bench.sampled_parity(b, W, bad, detr)
    assert not res["ok"] and res["max_rel_err_trend"] > 1e-5
    # A NaN where the oracle has a value.
    bad = trend.copy()
    bad[k] = np.nan
    assert not bench.sampled_parity(b, W, bad, detr)["nan_pattern_equal"]


def test_latency_summary_takes_steady_state_after_first_second():
    arrivals = np.linspace(0.0, 4.0, 4001)
    lat = np.where(arrivals < 1.0, 1.0, 0.001)          # a slow start, then 1 ms
    r = bench.latency_summary(arrivals, lat, 4.0, 1000.0, 1000.0, arrivals.size)
    assert abs(r["p50_ms"] - 1.0) < 1e-9 and abs(r["p99_ms"] - 1.0) < 1e-9
    assert r["steady_requests"] == int((arrivals >= 1.0).sum())
    assert r["p99_ms_all"] > 100.0


def test_serving_stream_mixture_and_slices():
    st = synth.serving_stream(n_requests=20000, tape_samples=(300_000, 600_000, 400_000))
    again = synth.serving_stream(n_requests=20000, tape_samples=(300_000, 600_000, 400_000))
    assert np.array_equal(st.n, again.n) and np.array_equal(st.start, again.start)
    assert all(np.array_equal(a, b, equal_nan=True) for a, b in zip(st.tapes, again.tapes))
    frac = np.bincount(st.kind, minlength=3) / st.kind.size
    assert np.allclose(frac, [0.45, 0.45, 0.10], atol=0.015)
    for k, (lo, hi) in enumerate(((5000, 20000), (4000, 70000), (60000, 118000))):
        nk = st.n[st.kind == k]
        assert nk.min() >= lo and nk.max() <= hi
    ends = st.start + st.n
    assert (st.start >= 0).all() and (ends <= np.array([t.size for t in st.tapes])[st.kind]).all()
    assert np.all(np.diff(st.arrivals) > 0)
    assert abs(np.mean(np.diff(st.arrivals)) - 1.0) < 0.03      # unit-rate Poisson process
    x = st.flux(7)
    assert x.dtype == np.float32 and x.size == st.n[7]
    assert np.isnan(st.tapes[1]).any()                              # Kepler tapes carry gaps


def test_kernel_code_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The measured-traffic record is keyed by a hash of the kernel's code:
    comment and blank-line edits keep it, any code edit changes it."""
    src = tmp_path / "k.cuh"
    src.write_text("// header\nint f(int x)\n{\n    return x + 1;  /* one */\n}\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(src))
    h0 = bench.kernel_sha256()
    src.write_text("// another header\n\nint f(int x)\n{\n    /* a\n       block */\n    return x + 1;  // one\n}\n")
    assert bench.kernel_sha256() == h0
    src.write_text("// header\nint f(int x)\n{\n    return x + 2;  /* one */\n}\n")
    assert bench.kernel_sha256() != h0


class _FakeTuner:
    """Records the tuning calls tune_for_batch makes (no GPU)."""

    def __init__(self, latency_below):
        self.batch_calls, self.single_calls = [], []
        self.latency_below = latency_below

    def autotune_batch(self, W, lengths, flux=None):
        self.batch_calls.append((W, np.asarray(lengths).copy(), flux.clone()))

    def autotune(self, W, positions):
        self.single_calls.append((W, positions))

    def get_plan(self, W, positions):
        return {"latency": int(positions < self.latency_below)}


def test_tune_for_batch_tunes_each_band_on_its_own_curves():
    """Each window length is tuned on its own curves: every k-th when the
    band holds more than 2e7 positions, repeated up to 1e6 when it holds
    fewer; the flux handed over is those curves back to back; a single
    latency-regime median curve is tuned on its own."""
    torch = pytest.importorskip("torch")
    b = synth.config3(n_curves=40)
    W = np.array([oracle.window_length(c) for c in b.cadence], np.int32)
    flux = torch.from_numpy(b.flux)
    fake = _FakeTuner(latency_below=20000)
    bench.tune_for_batch(fake, b, W, flux)
    assert [c[0] for c in fake.batch_calls] == sorted(set(W.tolist()))
    for w, lens, got in fake.batch_calls:
        idx = np.flatnonzero(W == w)
        own = b.lengths[idx]
        reps = lens.size // own.size
        assert reps * own.size == lens.size and lens.sum() >= 1_000_000
        assert np.array_equal(lens, np.tile(own, reps))
        want = np.concatenate([b.curve(int(i)) for i in idx] * reps)
        assert np.array_equal(got.numpy(), want, equal_nan=True)
    meds = {w: int(np.median(b.lengths[W == w])) for w in set(W.tolist())}
    assert fake.single_calls == [(w, meds[w]) for w in sorted(meds) if meds[w] < 20000]
    # A band above 2e7 positions is sampled: every k-th curve.
    big = synth.config2(n_curves=1200)
    Wb = np.full(big.B, 361, np.int32)
    fake = _FakeTuner(latency_below=0)
    bench.tune_for_batch(fake, big, Wb, torch.from_numpy(big.flux))
    (w, lens, got), = fake.batch_calls
    assert lens.size == 600 and lens.sum() <= 20_000_000
    assert np.array_equal(got[:18000].numpy(), big.curve(0), equal_nan=True)
    assert np.array_equal(got[18000:36000].numpy(), big.curve(2), equal_nan=True)
