"""Seeded synthetic light curves: the inputs shared by the oracle and the GPU path.

This module holds no arithmetic of the detrending method itself (no window
rule, median, scale or weights).  It only draws light curves whose shapes,
cadences, gaps and signal content follow the paper's workloads (TESS 2-min,
Kepler 29.4-min and TESS 20-s cadences; transits, flares, stellar variability
and NaN gaps), since the real TESS / Kepler light curves of the paper's
Section 3 are not available here.  Every array is a pure function of the seed.

All batches use the CSR layout the library consumes: curve ``b`` is
``flux[offsets[b]:offsets[b+1]]``.  Cadences are returned in days; callers
turn them into window lengths with the method's own rule.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CADENCE_TESS_2MIN = 2.0 / 1440.0
CADENCE_KEPLER_LC = 29.4 / 1440.0
CADENCE_TESS_20S = 20.0 / 86400.0
BASE_SEED = 20260406


@dataclass
class CurveBatch:
    """A CSR batch of light curves plus the injected-signal truth."""
    flux: np.ndarray            # float32 [total]; NaN marks a gap
    offsets: np.ndarray         # int64 [B+1]
    cadence: np.ndarray         # float64 [B], days
    transit: np.ndarray         # float32 [total], injected transit depth profile (>= 0)
    depth: np.ndarray           # float64 [B], nominal transit depth
    duration_d: np.ndarray      # float64 [B], total transit duration in days
    period_d: np.ndarray        # float64 [B]
    epoch_d: np.ndarray         # float64 [B], centre of the first transit
    window_days: float = 0.5
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def curve(self, b: int) -> np.ndarray:
        return self.flux[self.offsets[b]:self.offsets[b + 1]]

    def transit_curve(self, b: int) -> np.ndarray:
        return self.transit[self.offsets[b]:self.offsets[b + 1]]

    def subset(self, idx) -> "CurveBatch":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths[idx]
        off = np.zeros(idx.size + 1, np.int64)
        np.cumsum(lens, out=off[1:])
        flux = np.concatenate([self.curve(int(b)) for b in idx]) if idx.size else np.zeros(0, np.float32)
        tr = np.concatenate([self.transit_curve(int(b)) for b in idx]) if idx.size else np.zeros(0, np.float32)
        return CurveBatch(flux.astype(np.float32), off, self.cadence[idx].copy(), tr.astype(np.float32),
                          self.depth[idx].copy(), self.duration_d[idx].copy(),
                          self.period_d[idx].copy(), self.epoch_d[idx].copy(),
                          self.window_days, self.name + "[subset]", dict(self.meta))


def curve_rng(seed: int, index: int) -> np.random.Generator:
    """Independent stream per curve: SeedSequence over (seed, index)."""
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(index)]))


def _trapezoid(t, depth, duration, period, epoch, ingress_frac=0.1):
    """Periodic trapezoid dip profile (positive numbers = flux removed);
    ingress_frac = 0 gives a box."""
    if depth <= 0 or duration <= 0:
        return np.zeros_like(t)
    phase = np.mod(t - epoch + 0.5 * period, period) - 0.5 * period
    half = 0.5 * duration
    if ingress_frac <= 0:
        return depth * (np.abs(phase) <= half)
    tau = ingress_frac * duration
    frac = np.clip((half - np.abs(phase)) / tau, 0.0, 1.0)
    return depth * frac


def _flares(rng, t, count, amp, efold_days):
    out = np.zeros_like(t)
    if count <= 0:
        return out
    starts = rng.uniform(t[0], t[-1], size=count)
    for ts in starts:
        k = int(np.searchsorted(t, ts, side="left"))    # t is ascending: t >= ts from k on
        out[k:] += amp * np.exp(-(t[k:] - ts) / efold_days)
    return out


def _ar1(rng, n, sigma, phi):
    """AR(1) series with stationary standard deviation sigma."""
    from scipy.signal import lfilter
    e = rng.normal(0.0, sigma * np.sqrt(1.0 - phi * phi), size=n)
    e[0] = rng.normal(0.0, sigma)
    return lfilter([1.0], [1.0, -phi], e)


def make_curve(rng, n, cadence, *, sigma=1e-3, depth=1e-3, duration_h=3.0, period_d=3.7,
               n_sines=3, sine_amp=1e-3, red_phi=None, red_sigma=None, n_flares=5,
               flare_amp=5e-3, flare_efold_min=10.0, mid_gap_days=1.0, periodic_gap=None,
               spike_frac=0.0, spike_sigmas=10.0):
    """One light curve.  Returns (flux float32, transit profile float32, epoch).

    flux = 1 + sinusoids + red noise + white noise + flares + spikes - transits,
    with NaN over the gaps.  ``periodic_gap`` = (gap_days, every_days, jitter_days).
    """
    t = np.arange(n, dtype=np.float64) * cadence
    flux = np.ones(n, dtype=np.float64)
    for _ in range(int(n_sines)):
        p = rng.uniform(1.0, 10.0)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        flux += sine_amp * np.sin(2.0 * np.pi * t / p + ph)
    if red_phi is not None:
        flux += _ar1(rng, n, sigma if red_sigma is None else red_sigma, red_phi)
    flux += rng.normal(0.0, sigma, size=n)
    flux += _flares(rng, t, n_flares, flare_amp, flare_efold_min / 1440.0)
    if spike_frac > 0:
        k = int(round(spike_frac * n))
        idx = rng.choice(n, size=k, replace=False)
        flux[idx] += rng.choice([-1.0, 1.0], size=k) * spike_sigmas * sigma
    duration = duration_h / 24.0
    epoch = rng.uniform(0.0, period_d)
    transit = _trapezoid(t, depth, duration, period_d, epoch)
    flux -= transit
    if mid_gap_days and mid_gap_days > 0:
        g = int(round(mid_gap_days / cadence))
        s = max(0, n // 2 - g // 2)
        flux[s:s + g] = np.nan
    if periodic_gap is not None:
        gap_days, every_days, jitter = periodic_gap
        g = int(round(gap_days / cadence))
        start = every_days + rng.uniform(-jitter, jitter)
        while start < t[-1]:
            s = int(round(start / cadence))
            flux[s:s + g] = np.nan
            start += every_days + rng.uniform(-jitter, jitter)
    return flux.astype(np.float32), transit.astype(np.float32), epoch


def _assemble(curves, cadences, depths, durations, periods, epochs, name, meta=None):
    lens = np.array([c[0].size for c in curves], dtype=np.int64)
    off = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    flux = np.concatenate([c[0] for c in curves]) if curves else np.zeros(0, np.float32)
    tr = np.concatenate([c[1] for c in curves]) if curves else np.zeros(0, np.float32)
    return CurveBatch(flux, off, np.asarray(cadences, np.float64), tr,
                      np.asarray(depths, np.float64), np.asarray(durations, np.float64) / 24.0,
                      np.asarray(periods, np.float64), np.asarray(epochs, np.float64),
                      0.5, name, meta or {})


def config1(seed: int = BASE_SEED + 0) -> CurveBatch:
    """One TESS-like 2-min curve: N=18,000, a 1-day NaN gap mid-series,
    3 sinusoids (P 1-10 d, 1e-3), white noise 1e-3, 0.1 % / 3 h / 3.7 d
    trapezoid transits, 5 upward flares (5e-3, 10-min e-folding)."""
    rng = curve_rng(seed, 0)
    f, tr, ep = make_curve(rng, 18000, CADENCE_TESS_2MIN)
    return _assemble([(f, tr)], [CADENCE_TESS_2MIN], [1e-3], [3.0], [3.7], [ep], "tess-1x18000")


def _loguniform(rng, lo, hi):
    return float(np.exp(rng.uniform(np.log(lo), np.log(hi))))


def config2(seed: int = BASE_SEED + 1, n_curves: int = 1000, n: int = 18000) -> CurveBatch:
    """Equal-length TESS-like batch: sigma log-U(2e-4, 5e-3), depth
    log-U(1e-4, 5e-2), duration U(1, 8) h, period U(1, 15) d, 0-3 sinusoids,
    AR(1) red noise (phi 0.99, stationary std sigma) plus white noise sigma,
    and the same 1-day mid-series gap as the single-curve case."""
    curves, dep, dur, per, ep = [], [], [], [], []
    for b in range(n_curves):
        rng = curve_rng(seed, b)
        sigma = _loguniform(rng, 2e-4, 5e-3)
        depth = _loguniform(rng, 1e-4, 5e-2)
        duration = rng.uniform(1.0, 8.0)
        period = rng.uniform(1.0, 15.0)
        ns = int(rng.integers(0, 4))
        f, tr, e = make_curve(rng, n, CADENCE_TESS_2MIN, sigma=sigma, depth=depth,
                              duration_h=duration, period_d=period, n_sines=ns,
                              red_phi=0.99, n_flares=0)
        curves.append((f, tr)); dep.append(depth); dur.append(duration); per.append(period); ep.append(e)
    return _assemble(curves, [CADENCE_TESS_2MIN] * n_curves, dep, dur, per, ep,
                     "tess-%dx%d" % (n_curves, n))


def config3(seed: int = BASE_SEED + 2, n_curves: int = 4096) -> CurveBatch:
    """Uneven CSR batch: half TESS 2-min (N U(5k, 20k)), half Kepler 29.4-min
    (N U(4k, 70k), 3-day NaN gaps every 90 +- 5 d), in a seeded random order.
    Signal model of the single-curve case."""
    order = curve_rng(seed, 1 << 30).permutation(n_curves)
    curves, cad, dep, dur, per, ep = [], [], [], [], [], []
    for b in range(n_curves):
        rng = curve_rng(seed, b)
        kepler = order[b] % 2 == 1
        if kepler:
            n = int(rng.integers(4000, 70001))
            f, tr, e = make_curve(rng, n, CADENCE_KEPLER_LC, mid_gap_days=0,
                                  periodic_gap=(3.0, 90.0, 5.0))
            cad.append(CADENCE_KEPLER_LC)
        else:
            n = int(rng.integers(5000, 20001))
            f, tr, e = make_curve(rng, n, CADENCE_TESS_2MIN)
            cad.append(CADENCE_TESS_2MIN)
        curves.append((f, tr)); dep.append(1e-3); dur.append(3.0); per.append(3.7); ep.append(e)
    return _assemble(curves, cad, dep, dur, per, ep, "uneven-%d" % n_curves)


def config4(seed: int = BASE_SEED + 3, n_curves: int = 256, n: int = 118000) -> CurveBatch:
    """Large-window stress: TESS 20-s curves, N=118,000, single-curve signal
    model plus +-10 sigma spikes on 1 % of the samples."""
    curves, ep = [], []
    for b in range(n_curves):
        rng = curve_rng(seed, b)
        f, tr, e = make_curve(rng, n, CADENCE_TESS_20S, spike_frac=0.01)
        curves.append((f, tr)); ep.append(e)
    return _assemble(curves, [CADENCE_TESS_20S] * n_curves, [1e-3] * n_curves, [3.0] * n_curves,
                     [3.7] * n_curves, ep, "tess20s-%dx%d" % (n_curves, n))


@dataclass
class ServingStream:
    """A stream of detrend requests.  Request i arrives at ``arrivals[i] / rate``
    seconds, is of class ``kind[i]`` (0 TESS 2-min, 1 Kepler 29.4-min, 2 TESS
    20-s) and its flux is ``tapes[kind[i]][start[i]:start[i] + n[i]]``."""
    arrivals: np.ndarray        # float64 [R], Poisson process of unit rate
    kind: np.ndarray            # int8 [R]
    n: np.ndarray               # int64 [R]
    start: np.ndarray           # int64 [R]
    tapes: list                 # three float32 arrays
    cadences: tuple             # days, per class

    def flux(self, i: int) -> np.ndarray:
        k = int(self.kind[i])
        return self.tapes[k][self.start[i]:self.start[i] + self.n[i]]


SERVING_CLASSES = (
    # (share, N range, cadence, curve options): the mixture of the uneven
    # TESS / Kepler batch and the 20-s large-window curves.
    (0.45, (5000, 20000), CADENCE_TESS_2MIN, {}),
    (0.45, (4000, 70000), CADENCE_KEPLER_LC, {"mid_gap_days": 0, "periodic_gap": (3.0, 90.0, 5.0)}),
    (0.10, (60000, 118000), CADENCE_TESS_20S, {"spike_frac": 0.01}),
)


def serving_stream(seed: int = BASE_SEED + 4, n_requests: int = 200000,
                   tape_samples=(8_000_000, 16_000_000, 8_000_000)) -> ServingStream:
    """Poisson arrivals (unit rate) whose sizes are drawn from the full serving
    mixture: 45 % TESS 2-min (N U(5k, 20k)), 45 % Kepler 29.4-min (N U(4k, 70k),
    3-day gaps every 90 d) and 10 % TESS 20-s (N U(60k, 118k), 1 % spikes).
    Every request gets its own size and its own slice of a long tape of curves
    of its class (the tape is the class's light curves end to end), so no two
    requests need be alike while host memory stays bounded."""
    rng = curve_rng(seed, 1 << 31)
    arrivals = np.cumsum(rng.exponential(1.0, size=n_requests))
    u = rng.uniform(size=n_requests)
    shares = np.cumsum([c[0] for c in SERVING_CLASSES])
    kind = np.searchsorted(shares, u, side="right").astype(np.int8)
    kind = np.minimum(kind, len(SERVING_CLASSES) - 1)
    lo = np.array([c[1][0] for c in SERVING_CLASSES], np.int64)
    hi = np.array([c[1][1] for c in SERVING_CLASSES], np.int64)
    n = rng.integers(lo[kind], hi[kind] + 1)
    tapes = []
    for k, (_, (nlo, nhi), cad, opts) in enumerate(SERVING_CLASSES):
        parts, total, i = [], 0, 0
        while total < tape_samples[k]:
            r = curve_rng(seed, (k + 1) * 1_000_000 + i)
            f, _, _ = make_curve(r, int(r.integers(nlo, nhi + 1)), cad, **opts)
            parts.append(f)
            total += f.size
            i += 1
        tapes.append(np.concatenate(parts)[:tape_samples[k]].astype(np.float32))
    tape_len = np.array([t.size for t in tapes], np.int64)
    start = np.floor(rng.uniform(size=n_requests) * (tape_len[kind] - n + 1)).astype(np.int64)
    return ServingStream(arrivals, kind, n, start, tapes, tuple(c[2] for c in SERVING_CLASSES))


def injection_base(seed, n_stars, mission="tess"):
    """Noise-and-variability curves for box-transit injection (stand-ins for
    the TESS sector-6 / Kepler Q5 stars of Section 3.2).  TESS: 2-min cadence,
    18,000 samples, white noise log-U(500, 2000) ppm, AR(1) red noise at 30 %
    of it, 0-2 sinusoids of up to 2 sigma, the 1-day mid gap.  Kepler: 29.4-min
    cadence, 4,400 samples (one quarter), white noise log-U(50, 200) ppm, the
    same red-noise and variability recipe, no gap.  Returns (batch without
    transits, box-transit unit profiles: 1 inside a transit, P = 3 d,
    D = 3 h, random epoch)."""
    kepler = mission == "kepler"
    cad = CADENCE_KEPLER_LC if kepler else CADENCE_TESS_2MIN
    n = 4400 if kepler else 18000
    lo, hi = (5e-5, 2e-4) if kepler else (5e-4, 2e-3)
    curves, profiles, ep = [], [], []
    for b in range(n_stars):
        rng = curve_rng(seed, b)
        sigma = _loguniform(rng, lo, hi)
        f, _, e = make_curve(rng, n, cad, sigma=sigma, depth=0.0, n_sines=int(rng.integers(0, 3)),
                             sine_amp=float(rng.uniform(0.0, 2.0)) * sigma, red_phi=0.99,
                             red_sigma=0.3 * sigma, n_flares=0,
                             mid_gap_days=0.0 if kepler else 1.0)
        t = np.arange(n) * cad
        epoch = rng.uniform(0.0, 3.0)
        profiles.append(_trapezoid(t, 1.0, 3.0 / 24.0, 3.0, epoch, ingress_frac=0.0).astype(np.float32))
        curves.append((f, np.zeros(n, np.float32)))
        ep.append(epoch)
    batch = _assemble(curves, [cad] * n_stars, [0.0] * n_stars, [3.0] * n_stars, [3.0] * n_stars, ep,
                      "%s-injection-%d" % (mission, n_stars))
    return batch, np.concatenate(profiles)


def inject(base, unit_profile, depth):
    """Copy of `base` with box transits of the given fractional depth."""
    b = CurveBatch(base.flux - np.float32(depth) * unit_profile, base.offsets.copy(), base.cadence.copy(),
                   (np.float32(depth) * unit_profile).astype(np.float32),
                   np.full(base.B, depth, np.float64), base.duration_d.copy(), base.period_d.copy(),
                   base.epoch_d.copy(), base.window_days, base.name + "+%gppm" % (depth * 1e6),
                   dict(base.meta))
    b.flux = b.flux.astype(np.float32)
    return b


def random_curve(seed, n, *, nan_frac=0.0, nan_runs=0, run_len=(1, 50), ties=False,
                 level=1.0, sigma=1e-3, quantum=None):
    """Small unit-test curve: level + N(0, sigma), optional isolated NaNs,
    NaN runs, and value ties (rounding to ``quantum``)."""
    rng = curve_rng(seed, 7)
    x = level + rng.normal(0.0, sigma, size=n)
    if ties or quantum:
        q = quantum if quantum else sigma
        x = np.round(x / q) * q
    if nan_frac > 0:
        x[rng.uniform(size=n) < nan_frac] = np.nan
    for _ in range(int(nan_runs)):
        if n == 0:
            break
        L = int(rng.integers(run_len[0], run_len[1] + 1))
        s = int(rng.integers(0, max(1, n)))
        x[s:s + L] = np.nan
    return x.astype(np.float32)
