"""Pins for the FP64 oracle: values the paper prints, closed forms, invariants
and brute force.  None of these recompute the oracle's own arithmetic; each is
chosen so that a plausible slip (alpha on the wrong side, s divided instead of
multiplied by 0.6745, both-sided scale, upper median, early exit, floor in the
window rule) fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2604_06602_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ---- window rule (Section 2 opening paragraph; Section 4, Kepler Long-Cadence) ----

@pytest.mark.parametrize("case", GOLDEN["window_length"])
def test_window_length_paper_values(case):
    assert oracle.window_length(case["cadence_min"] / 1440.0, case["window_days"]) == case["W"]


def test_window_span_printed():
    g = GOLDEN["window_span_days"]
    span = g["W"] * g["cadence_min"] / 1440.0
    assert round(span, g["decimals"]) == g["span_days"]


def test_window_length_other_cadences():
    # Kepler's true long cadence (29.4 min) and TESS 20-s data.
    assert oracle.window_length(29.4 / 1440.0) == 25
    assert oracle.window_length(20.0 / 86400.0) == 2161
    # Always odd, also when round() lands on an even number.
    for dt_min in np.linspace(0.3, 40.0, 400):
        assert oracle.window_length(dt_min / 1440.0) % 2 == 1
    assert oracle.window_length(0.0) == -1
    assert oracle.window_length(-1.0) == -1
    assert oracle.window_length(float("nan")) == -1


def test_window_length_from_time_differences():
    """The cadence recovered from FP64 time stamps is 1/720 d only up to
    rounding; 0.5/dt then sits just below 360.  Rounding (our reading of the
    garbled bracket) still gives 361; a floor would give 359."""
    t = 1500.0 + np.arange(20000) * (2.0 / 1440.0)
    dt = float(np.median(np.diff(t)))
    assert 0.5 / dt != 360.0
    assert oracle.window_length(dt) == 361


# ---- weights, Eqs. 2-3 (numbers printed in Section 2.3 and Figure 1) ----

@pytest.mark.parametrize("case", GOLDEN["weights"])
def test_weight_paper_values(case):
    w = oracle.weight(case["u"], case["alpha"])
    assert round(w, case["decimals"]) == case["w"]


def test_weight_shape():
    # Upward residuals ignore alpha; downward ones are stretched by alpha.
    for u in (0.1, 0.3, 0.7, 0.99):
        assert oracle.weight(u, 2.0) == oracle.weight(u, 1.0) == oracle.weight(u, 10.0)
        assert oracle.weight(-u / 2.0, 2.0) == oracle.weight(u, 1.0)
    assert oracle.weight(0.0, 2.0) == 1.0
    assert oracle.weight(1.0, 2.0) == 0.0            # |u_eff| < 1 is strict
    assert oracle.weight(-0.5, 2.0) == 0.0           # alpha * u = -1
    assert oracle.weight(-0.49, 2.0) > 0.0
    assert oracle.weight(3.0, 1.0) == 0.0


# ---- Phase 1: exact lower median, brute force on tiny curves ----

def _brute_windows(x, W):
    h = (W - 1) // 2
    n = len(x)
    for j in range(n):
        lo, hi = max(0, j - h), min(n - 1, j + h)
        vals = sorted(float(v) for v in x[lo:hi + 1] if np.isfinite(v))
        yield j, vals


@pytest.mark.parametrize("seed", range(12))
def test_median_and_nplus_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    W = int(rng.choice([1, 3, 5, 7, 9, 15, 31, 61]))
    x = rng.integers(-4, 5, size=n).astype(np.float32) * 0.25   # many ties
    if seed % 3 == 0:
        x = rng.normal(size=n).astype(np.float32)
    x[rng.uniform(size=n) < 0.2] = np.nan
    if seed % 4 == 1 and n > 3:
        x[: n // 3] = np.inf                                     # non-finite run at the edge
    out = oracle.detrend(x, W, min_valid=0)
    for j, vals in _brute_windows(x, W):
        assert out["nvalid"][j] == len(vals)
        if not vals:
            assert math.isnan(out["median"][j])
            continue
        m = vals[(len(vals) - 1) // 2]
        assert out["median"][j] == m
        assert out["nplus"][j] == sum(v > m for v in vals)


def test_even_window_takes_lower_median():
    x = np.array([4, 1, 3, 2], np.float32)          # one window of 4 at j=1 (W=5)
    out = oracle.detrend(x, 5, min_valid=0)
    assert out["median"][1] == 2.0                   # sorted 1,2,3,4 -> rank 1
    assert out["nplus"][1] == 2


# ---- Phase 2: closed forms for the upper-RMS scale (Eq. 1) ----

def test_scale_exponential_closed_form():
    """For Exp(1) the median is ln 2 and the excess above it is again Exp(1)
    (memorylessness), so E[(x - m)^2 | x > m] = 2 and s -> 0.6745 sqrt(2).
    A both-sided RMS, a MAD, or s = sigma/0.6745 all miss this by far."""
    v = np.random.default_rng(3).exponential(1.0, 400001)
    m, nplus, s, _ = oracle.window_estimate(v)
    assert abs(m - math.log(2.0)) < 0.01
    assert nplus == 200000
    assert s == pytest.approx(0.6745 * math.sqrt(2.0), rel=0.01)


def test_scale_gaussian_closed_form_and_paper_residual():
    """Gaussian noise sigma: sigma_up -> sigma, s -> 0.6745 sigma, so a dip of
    depth sigma standardises to |u| = 1/(5 * 0.6745) = 0.2965, the paper's
    u ~ 0.3 (Section 2.5), with weights ~0.83 / ~0.41 (Section 2.3)."""
    g = GOLDEN["dip_residual"]
    sigma = 1e-3
    v = 1.0 + np.random.default_rng(2).normal(0.0, sigma, 400001)
    m, nplus, s, _ = oracle.window_estimate(v)
    assert s / sigma == pytest.approx(GOLDEN["defaults"]["scale_factor"], rel=0.01)
    u = -g["depth_over_sigma"] * sigma / (GOLDEN["defaults"]["c"] * s)
    assert abs(u) == pytest.approx(g["u"], abs=0.01)
    assert round(oracle.weight(u, 1.0), 2) == g["w_alpha1"]
    assert oracle.weight(u, 2.0) == pytest.approx(g["w_alpha2"], abs=0.015)


def test_scale_ignores_points_below_median():
    """Pushing below-median points further down leaves the median, n_plus and
    s bit-identical (Section 2.2: dips never enter the scale)."""
    rng = np.random.default_rng(5)
    v = rng.normal(size=301)
    m0, p0, s0, mu0 = oracle.window_estimate(v)
    w = v.copy()
    low = w < m0
    w[low] -= rng.uniform(0.0, 50.0, size=low.sum())
    m1, p1, s1, mu1 = oracle.window_estimate(w)
    assert (m1, p1, s1) == (m0, p0, s0)
    # ... while raising above-median points does change s.
    w2 = v.copy()
    w2[v > m0] *= 1.5
    assert oracle.window_estimate(w2)[2] != s0


# ---- Phase 3 and the whole estimator: special cases and invariants ----

def test_constant_returns_itself():
    x = np.full(200, 1.2345, np.float32)
    out = oracle.detrend(x, 31)
    assert np.all(out["trend"] == np.float64(np.float32(1.2345)))
    assert np.all(out["detr"] == 1.0)


def test_alpha1_symmetric_window_keeps_median():
    """alpha = 1 is the symmetric biweight (Section 2.3); on a window symmetric
    about its median every step keeps mu at the median."""
    for vals in ([0, 1, 2, 3, 4, 5, 6], [-3, -1, 0, 1, 3], [2.5, 2.5, 4.0, 1.0, 2.5]):
        m, _, _, mu = oracle.window_estimate(vals, alpha=1.0)
        assert mu == m
    rng = np.random.default_rng(9)
    half = rng.exponential(size=150)
    sym = np.concatenate([7.0 - half, [7.0], 7.0 + half])
    m, _, _, mu = oracle.window_estimate(sym, alpha=1.0)
    assert m == 7.0 and abs(mu - 7.0) < 1e-12


def test_alpha_pushes_trend_up():
    """With alpha > 1 downward residuals lose weight, so the trend floats above
    the symmetric one (Section 1 and Section 2.3), monotonically in alpha."""
    v = np.random.default_rng(11).normal(size=361)
    mus = [oracle.window_estimate(v, alpha=a)[3] for a in (1.0, 2.0, 3.0, 10.0)]
    assert mus[0] < mus[1] < mus[2] < mus[3]
    # Mirroring the data must not mirror the estimate (the method is one-sided).
    assert oracle.window_estimate(-v, alpha=2.0)[3] != -mus[1]


def test_hand_worked_window():
    """x = 0..6, alpha 2, c 5.  By hand: median 3, above-median residuals
    1, 2, 3, so sigma_up = sqrt(14/3) = 2.16025 and s = 1.45709, c s = 7.28543.
    First step from mu = 3: standardised residuals -0.41178, -0.27452,
    -0.13726, 0, 0.13726, 0.27452, 0.41178; the three negative ones doubled
    give weights 0.10352, 0.48797, 0.85496, then 1, 0.96268, 0.85496, 0.68963;
    sum w = 4.95372, sum w x = 17.46119, so mu_1 = 3.52490."""
    m, nplus, s, mu1 = oracle.window_estimate(np.arange(7.0), iters=1)
    assert (m, nplus) == (3.0, 3)
    assert s == pytest.approx(0.6745 * math.sqrt(14.0 / 3.0), rel=1e-12)
    assert mu1 == pytest.approx(3.52490, abs=5e-5)


def test_iteration_count_is_fixed():
    v = np.random.default_rng(13).normal(size=361)
    m, _, _, mu0 = oracle.window_estimate(v, iters=0)
    assert mu0 == m
    mu5 = oracle.window_estimate(v, iters=5)[3]
    mu50 = oracle.window_estimate(v, iters=50)[3]
    # Five steps are not converged: an early-exit rule would change results.
    assert abs(mu5 - mu50) > 1e-3 * abs(mu50 - m)


def test_degenerate_scale_returns_median():
    # No sample above the median.
    m, nplus, s, mu = oracle.window_estimate([1.0, 1.0, 1.0, 0.0, 0.5])
    assert nplus == 0 and mu == m == 1.0
    # A single sample.
    out = oracle.detrend(np.array([3.5], np.float32), 1)
    assert out["trend"][0] == 3.5 and out["detr"][0] == 1.0


def test_w1_is_identity():
    x = synth.random_curve(1, 500, nan_frac=0.1)
    out = oracle.detrend(x, 1)
    ok = np.isfinite(x)
    assert np.array_equal(out["trend"][ok], x[ok].astype(np.float64))
    assert np.all(out["detr"][ok] == 1.0)
    assert np.all(np.isnan(out["trend"][~ok]))


def test_location_scale_equivariance():
    """For a > 0 the estimator commutes with x -> a x + b (u is invariant).
    Powers of two are exact in binary floating point."""
    x = synth.random_curve(4, 400, nan_frac=0.05)
    base = oracle.detrend(x, 61)["trend"]
    for k in (-3, 1, 5):
        y = (x * np.float32(2.0 ** k)).astype(np.float32)
        t = oracle.detrend(y, 61)["trend"]
        assert np.array_equal(np.isnan(t), np.isnan(base))
        ok = ~np.isnan(base)
        assert np.array_equal(t[ok], base[ok] * 2.0 ** k)
    y = (x.astype(np.float64) * 3.0 - 2.0).astype(np.float32)
    t = oracle.detrend(y, 61)["trend"]
    ok = ~np.isnan(base)
    np.testing.assert_allclose(t[ok], 3.0 * base[ok] - 2.0, rtol=0, atol=1e-6)


def test_missing_centre_and_min_valid():
    x = synth.random_curve(6, 300)
    x[100] = np.nan
    x[200:290] = np.nan
    W = 31
    out = oracle.detrend(x, W)                       # default min_valid = W // 3 = 10
    assert np.isnan(out["trend"][100]) and not np.isnan(out["median"][100])
    # Position 289 sits on a gap sample -> NaN.  The truncated window of the
    # last position, 284..299, holds exactly the 10 valid samples 290..299.
    assert np.isnan(out["trend"][289])
    assert out["nvalid"][299] == 10 and not np.isnan(out["trend"][299])
    out2 = oracle.detrend(x, W, min_valid=11)
    assert np.isnan(out2["trend"][299])


def test_positions_match_full_curve():
    x = synth.random_curve(8, 700, nan_frac=0.05, nan_runs=3)
    full = oracle.detrend(x, 101)
    pos = np.array([0, 1, 50, 349, 698, 699])
    part = oracle.detrend_positions(x, 101, pos)
    for k in ("trend", "detr", "median", "nvalid", "nplus", "scale"):
        np.testing.assert_array_equal(part[k], full[k][pos])


def test_batch_matches_single_curves():
    b = synth.config3(n_curves=6)
    W = np.array([oracle.window_length(c) for c in b.cadence], np.int32)
    tr, de = oracle.detrend_batch(b.flux, b.offsets, W, nthreads=3)
    for i in range(b.B):
        s = slice(b.offsets[i], b.offsets[i + 1])
        one = oracle.detrend(b.curve(i), W[i])
        np.testing.assert_array_equal(tr[s], one["trend"])
        np.testing.assert_array_equal(de[s], one["detr"])


def test_invalid_arguments_rejected():
    x = np.ones(10, np.float32)
    for W in (0, 2, -3):
        with pytest.raises(ValueError):
            oracle.detrend(x, W)
    with pytest.raises(ValueError):
        oracle.detrend(x, 3, alpha=0.0)
    with pytest.raises(ValueError):
        oracle.detrend(x, 3, c=-1.0)
    with pytest.raises(ValueError):
        oracle.detrend(x, 3, iters=-1)


# ---- the paper's bias figures (Sections 2.4, 3.1, 4.1): shape and ratios ----

def test_bias_shape_matches_paper():
    """Flat white-noise star, sigma = 1000 ppm, W = 361.  The paper prints the
    detrended offset as -451 ppm (alpha 2, c 5), -1857 ppm (alpha 10, c 2.5)
    and -2 ppm (alpha 1) on real stars of unstated noise.  The noise level
    fixes the absolute value, so the pins are: the sign, alpha 1 near zero,
    and the aggressive/default ratio (4.12 printed) within 10 %.  Reading
    s = sigma_up / 0.6745 would give a ratio near 19; recomputing s about mu
    each iteration would give about 3."""
    bias = GOLDEN["bias_ppm"]
    rng = np.random.default_rng(21)
    n, sig = 60000, 1e-3
    x = (1.0 + rng.normal(0.0, sig, n)).astype(np.float32)
    off = {}
    for key, a, c in (("a1", 1.0, 5.0), ("a2", 2.0, 5.0), ("a10", 10.0, 2.5)):
        _, de = oracle.detrend_batch(x, np.array([0, n]), np.array([361]), alpha=a, c=c)
        off[key] = float(np.nanmean(de - 1.0) * 1e6)
    assert abs(off["a1"]) < 20.0
    assert off["a2"] < 0 and off["a10"] < off["a2"]
    assert 0.5 * abs(bias["alpha2_c5"]) < abs(off["a2"]) < 1.5 * abs(bias["alpha2_c5"])
    ratio = off["a10"] / off["a2"]
    assert ratio == pytest.approx(bias["alpha10_c2p5"] / bias["alpha2_c5"], rel=0.10)


# ---- gap handling (Table 3's pipeline step; W/3 rule of Section 4) ----

def _brute_segments(x, gap_min, min_seg):
    """Segments as maximal runs between missing runs of length >= gap_min,
    found on the validity string with a regular expression."""
    import re
    s = "".join("1" if np.isfinite(v) else "0" for v in x)
    out = []
    for m in re.finditer(r"1(?:0{0,%d}1)*" % (gap_min - 1), s):
        valid = m.group(0).count("1")
        if valid >= max(1, min_seg):
            out.append((m.start(), m.end()))
    return out


@pytest.mark.parametrize("seed", range(10))
def test_segments_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 300))
    W = int(rng.choice([3, 7, 15, 31]))
    x = synth.random_curve(seed, n)
    for _ in range(int(rng.integers(0, 6))):
        s0 = int(rng.integers(0, n))
        x[s0:s0 + int(rng.integers(1, 3 * W))] = np.nan
    x[rng.uniform(size=n) < 0.05] = np.nan
    gap_min = int(rng.choice([1, 2, W // 2 + 1, W]))
    min_seg = int(rng.choice([0, 3, W // 3, W]))
    tr, de, kept = oracle.detrend_segmented(x, W, gap_min=gap_min, min_seg=min_seg)
    segs = _brute_segments(x, gap_min, min_seg)
    assert kept == len(segs)
    covered = np.zeros(n, bool)
    for a, b in segs:
        covered[a:b] = True
        ref = oracle.detrend(x[a:b], W)["trend"]          # each segment on its own
        np.testing.assert_array_equal(tr[a:b], ref)
    assert np.all(np.isnan(tr[~covered]))


def test_segments_without_splits_equal_plain():
    """No gap reaches gap_min and nothing is dropped: plain detrend."""
    x = synth.random_curve(3, 2000, nan_frac=0.05, nan_runs=4, run_len=(1, 40))
    tr, _, kept = oracle.detrend_segmented(x, 61, gap_min=10 ** 6, min_seg=0)
    assert kept == 1
    np.testing.assert_array_equal(tr, oracle.detrend(x, 61)["trend"])


def test_long_gaps_only_drop_short_segments():
    """A gap of at least W samples already separates the windows on both
    sides, so splitting there changes nothing except dropping segments with
    fewer than min_seg valid samples.  (With the defaults min_seg equals the
    per-window minimum W/3, so such islands are NaN either way; a larger
    min_seg shows the drop.)"""
    W = 61
    x = synth.random_curve(5, 3000)
    x[1000:1000 + W] = np.nan
    x[1500:1500 + 2 * W] = np.nan
    x[2500:2500 + W] = np.nan
    x[2500 + W + 30:2500 + 2 * W + 30] = np.nan   # a 30-sample island
    island = slice(2500 + W, 2500 + W + 30)
    plain = oracle.detrend(x, W)["trend"]
    assert not np.any(np.isnan(plain[island]))    # 30 >= W // 3
    tr, _, _ = oracle.detrend_segmented(x, W)     # gap_min = W, min_seg = W // 3
    np.testing.assert_array_equal(tr, plain)
    tr, _, kept = oracle.detrend_segmented(x, W, min_seg=W)
    assert kept == 4                              # five segments, the island dropped
    assert np.all(np.isnan(tr[island]))
    keep = np.ones(x.size, bool)
    keep[island] = False
    np.testing.assert_array_equal(tr[keep], plain[keep])


# ---- MAD scale (the comparison scale of Sections 1, 2.2 and 3.1) ----

def test_mad_closed_forms():
    """MAD about the median: Exp(1) gives sinh(d) = 1/2, so d = asinh(1/2);
    a Gaussian gives Phi^-1(3/4) sigma = 0.67449 sigma (the convention the
    0.6745 of Eq. 1 is matched to)."""
    v = np.random.default_rng(3).exponential(1.0, 400001)
    assert oracle.window_estimate(v, scale_mode=oracle.SCALE_MAD)[2] == pytest.approx(
        math.asinh(0.5), rel=0.015)
    g = 2.0 + 3.0 * np.random.default_rng(4).normal(size=400001)
    assert oracle.window_estimate(g, scale_mode=oracle.SCALE_MAD)[2] / 3.0 == pytest.approx(
        0.674489750, rel=0.01)


@pytest.mark.parametrize("seed", range(6))
def test_mad_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 50))
    x = (rng.integers(-5, 6, size=n) * 0.5).astype(np.float32)
    x[rng.uniform(size=n) < 0.15] = np.nan
    W = 9
    out = oracle.detrend(x, W, min_valid=0, scale_mode=oracle.SCALE_MAD)
    for j, vals in _brute_windows(x, W):
        if not vals or not np.isfinite(x[j]):
            continue
        m = vals[(len(vals) - 1) // 2]
        dev = sorted(abs(v - m) for v in vals)
        assert out["scale"][j] == dev[(len(dev) - 1) // 2]


def test_dips_inflate_mad_but_not_upper_rms():
    """Section 2.2: transit-like dips below the median enter the MAD but not
    the upper-RMS scale."""
    rng = np.random.default_rng(12)
    v = rng.normal(size=361)
    m = np.median(v)
    w = v.copy()
    low = np.nonzero(v < m)[0][:60]
    w[low] -= 10.0
    assert oracle.window_estimate(w)[2] == oracle.window_estimate(v)[2]
    assert oracle.window_estimate(w, scale_mode=oracle.SCALE_MAD)[2] > \
        1.05 * oracle.window_estimate(v, scale_mode=oracle.SCALE_MAD)[2]
