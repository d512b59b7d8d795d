"""GPU parity: libumi (through the C ABI) against the FP64 oracle.

Bar: valid counts, above-median counts and medians bit-exact; trend within
1e-5 relative per sample (scale-aware only for synthetic curves centred near
zero, see helpers.py); NaN outputs at identical positions; the depth-recovery
aggregate within 0.1 percentage points of the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2604_06602_gb300 import synth
from tests.helpers import compare_diag, compare_trend, compare_detr, depth_recovery_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def umi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_06602_gb300 import umi as u
    u.load(build_if_missing=True)
    return u


def run_diag(umi, x, W, p=None):
    xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    out = umi.detrend_diag(xd, W, p)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def oracle_params(p):
    if p is None:
        return {}
    return dict(alpha=p.alpha, c=p.c, iters=p.iters, min_valid=p.min_valid)


def tile_of(umi, W):
    pl = umi.get_plan(W, -1)
    return pl["threads"] // pl["lanes"] * pl["chain"]


# Every variant's capacity edge (the last W a variant serves and the first W
# of the next), plus the workload windows 25, 361 and 2161.
WINDOWS = [1, 3, 7, 9, 15, 17, 25, 27, 31, 33, 63, 65, 127, 129, 191, 193, 361, 367, 369, 383,
           385, 767, 769, 1535, 1537, 2161, 2175, 2177, 4095]


@pytest.mark.parametrize("W", WINDOWS)
def test_lengths_around_window_and_tiles(umi, W):
    T = tile_of(umi, W)
    for n in sorted({1, 2, max(1, W - 1), W, W + 1, 3 * T + 5}):
        x = synth.random_curve(1000 + n, n, level=1.0, sigma=1e-3)
        compare_diag(run_diag(umi, x, W), oracle.detrend(x, W), what="W=%d n=%d" % (W, n))


@pytest.mark.parametrize("W", [3, 25, 361, 2161])
def test_gaps_ties_and_edges(umi, W):
    n = 3 * tile_of(umi, W) + 17
    cases = {
        "nan_runs": synth.random_curve(1, n, nan_runs=6, run_len=(1, 2 * W)),
        "isolated_nan": synth.random_curve(2, n, nan_frac=0.2),
        "ties": synth.random_curve(3, n, quantum=5e-4),
        "heavy_ties": synth.random_curve(4, n, quantum=3e-3, nan_frac=0.05),
        "edge_gaps": synth.random_curve(5, n),
        "inf_and_nan": synth.random_curve(6, n, nan_frac=0.05),
    }
    x = cases["edge_gaps"]
    x[: W // 2 + 3] = np.nan
    x[-(W // 3 + 2):] = np.nan
    y = cases["inf_and_nan"]
    y[::97] = np.inf
    y[5::89] = -np.inf
    for name, x in cases.items():
        compare_diag(run_diag(umi, x, W), oracle.detrend(x, W), what="%s W=%d" % (name, W))


@pytest.mark.parametrize("W", [3, 25, 361, 2161])
def test_all_missing_constant_and_sparse(umi, W):
    n = 2 * tile_of(umi, W) + 3
    x = np.full(n, np.nan, np.float32)
    got = run_diag(umi, x, W)
    assert np.all(np.isnan(got["trend"])) and np.all(got["nvalid"] == 0)
    compare_diag(got, oracle.detrend(x, W), what="all-NaN")
    x = np.full(n, 1.25, np.float32)
    got = run_diag(umi, x, W)
    assert np.all(got["trend"] == 1.25) and np.all(got["detr"] == 1.0)
    # Constant runs separated by gaps, and isolated samples below min_valid.
    x = synth.random_curve(9, n)
    x[n // 4: n // 2] = 0.9995
    x[n // 2: n // 2 + W] = np.nan
    x[min(n - 1, n // 2 + W // 2)] = 1.0
    compare_diag(run_diag(umi, x, W), oracle.detrend(x, W), what="runs W=%d" % W)
    x = np.full(n, np.nan, np.float32)
    x[:: max(2, W // 2)] = 1.0 + np.arange(x[:: max(2, W // 2)].size, dtype=np.float32) * 1e-4
    compare_diag(run_diag(umi, x, W), oracle.detrend(x, W), what="sparse W=%d" % W)
    compare_diag(run_diag(umi, x, W, umi.params(min_valid=0)), oracle.detrend(x, W, min_valid=0),
                 what="sparse min_valid=0 W=%d" % W)


@pytest.mark.parametrize("alpha", [0.2, 0.25, 4.0, 4.5])
def test_sign_select_forms_at_their_boundary(umi, alpha):
    """The iteration loop selects the Eq. 2 branch through |t| for
    1/4 <= alpha <= 4 and by the min of two scaled residuals otherwise: both
    sides of both edges against the oracle, on flux-like data with flares and
    dips and on a gappy noise curve."""
    x = synth.config1().curve(0)[:6000].copy()
    p = umi.params(alpha=alpha)
    compare_diag(run_diag(umi, x, 361, p), oracle.detrend(x, 361, alpha=alpha), what="alpha=%g" % alpha)
    y = synth.random_curve(77, 3000, nan_frac=0.05, nan_runs=2, run_len=(1, 61))
    compare_diag(run_diag(umi, y, 61, p), oracle.detrend(y, 61, alpha=alpha), what="gappy alpha=%g" % alpha)


@pytest.mark.parametrize("preset", [(2.0, 5.0), (3.0, 5.0), (1.0, 5.0), (10.0, 2.5), (0.5, 4.0)])
def test_parameter_presets(umi, preset):
    """Table 4 presets (and alpha < 1) on flux-like data with flares and dips."""
    alpha, c = preset
    b = synth.config1()
    x = b.curve(0)[:6000].copy()
    p = umi.params(alpha=alpha, c=c)
    compare_diag(run_diag(umi, x, 361, p), oracle.detrend(x, 361, alpha=alpha, c=c),
                 what="alpha=%g c=%g" % preset)


@pytest.mark.parametrize("c", [0.02, 0.3, 1e4])
@pytest.mark.parametrize("alpha", [2.0, 10.0])
def test_extreme_tuning_constant(umi, c, alpha):
    """c far from the paper's presets, in both sign-select forms: c = 0.02
    and 0.3 leave most samples outside the bisquare support (zero weight),
    c = 1e4 gives every sample a weight near 1 (a plain mean)."""
    x = synth.config1().curve(0)[:5000].copy()
    p = umi.params(alpha=alpha, c=c)
    compare_diag(run_diag(umi, x, 361, p), oracle.detrend(x, 361, alpha=alpha, c=c), c=c,
                 what="alpha=%g c=%g" % (alpha, c))


@pytest.mark.parametrize("iters", [0, 1, 2, 7])
def test_iteration_counts(umi, iters):
    x = synth.config1().curve(0)[:3000].copy()
    p = umi.params(iters=iters)
    compare_diag(run_diag(umi, x, 361, p), oracle.detrend(x, 361, iters=iters), what="iters=%d" % iters)


def test_zero_centred_and_scaled(umi):
    """Curves centred on zero and far from unit scale; the trend bound is
    1e-5 of max(|trend|, c s) here."""
    rng = np.random.default_rng(77)
    # sigma 5e-20: the squared residuals of Eq. 1 are subnormal (about 2.5e-39),
    # so the mean square takes the kernel's IEEE root instead of rsqrt; level
    # 1e15 and sigma 1e17 take mean squares near 1e26 and 1e34.
    for level, sigma in ((0.0, 1.0), (0.0, 1e-6), (1e4, 30.0), (-5.0, 0.1), (0.0, 5e-20),
                         (1e15, 1e13), (0.0, 1e17)):
        x = (level + sigma * rng.standard_normal(3000)).astype(np.float32)
        x[rng.uniform(size=x.size) < 0.03] = np.nan
        compare_diag(run_diag(umi, x, 129), oracle.detrend(x, 129), scale_aware=True,
                     what="level=%g sigma=%g" % (level, sigma), x=x)
    x = rng.integers(-3, 4, 2000).astype(np.float32)   # integers: ties everywhere
    compare_diag(run_diag(umi, x, 61), oracle.detrend(x, 61), scale_aware=True, what="integers", x=x)


@pytest.mark.parametrize("W", [25, 61, 361, 2161])
def test_signed_zeros_and_extreme_magnitudes(umi, W):
    """Exact selection on windows mixing -0 and +0, both signs and
    magnitudes from 2^-60 to 2^55: the select's candidates then span the
    whole order, NaN bit patterns included.  Medians and counts exact."""
    rng = np.random.default_rng(W)
    n = 3 * W + 101
    x = rng.choice(np.array([-0.0, 0.0, -1.0, 1.0, 2.0], np.float32), n)
    compare_diag(run_diag(umi, x, W), oracle.detrend(x, W), scale_aware=True, what="zeros W=%d" % W, x=x)
    mag = np.exp2(rng.uniform(-60, 55, n))
    x = (np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0) * mag).astype(np.float32)
    x[rng.uniform(size=n) < 0.05] = 0.0
    got = run_diag(umi, x, W)
    ref = oracle.detrend(x, W)
    ok = ~np.isnan(ref["median"])
    assert np.array_equal(got["median"][ok].astype(np.float64), ref["median"][ok])
    np.testing.assert_array_equal(got["nvalid"], ref["nvalid"])
    np.testing.assert_array_equal(got["nplus"], ref["nplus"])


def test_config1_full_and_depth_recovery(umi):
    b = synth.config1()
    x = b.curve(0)
    W = umi.window_length(b.cadence[0])
    assert W == 361
    got = run_diag(umi, x, W)
    ref = oracle.detrend(x, W)
    compare_diag(got, ref, what="config1")
    e_gpu = depth_recovery_errors(got["detr"], b)
    e_ref = depth_recovery_errors(ref["detr"], b)
    assert e_gpu.size == 1 and abs(e_gpu[0] - e_ref[0]) < 0.1


@pytest.fixture(scope="module")
def config2(umi):
    """The full benchmark batch, run in the plans bench.py times (its autotuner)."""
    import bench
    b = synth.config2()
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    assert np.all(W == 361)
    flux = torch.from_numpy(b.flux).cuda()
    try:
        umi.clear_tuning()
        bench.tune_for_batch(umi, b, W, flux)
        tr, de = umi.detrend_batched(flux, b.offsets, W)
        torch.cuda.synchronize()
    finally:
        umi.clear_tuning()
    return b, W, tr.cpu().numpy(), de.cpu().numpy()


def test_config2_batched_full_curves_and_depth(umi, config2):
    b, W, tr, de = config2
    sub = np.arange(0, b.B, b.B // 48)[:48]
    s = b.subset(sub)
    rt, rd = oracle.detrend_batch(s.flux, s.offsets, W[sub])
    gt = np.concatenate([tr[b.offsets[i]:b.offsets[i + 1]] for i in sub])
    gd = np.concatenate([de[b.offsets[i]:b.offsets[i + 1]] for i in sub])
    compare_trend(gt, rt, what="config2 subset")
    compare_detr(gd, rd, what="config2 subset")
    e_gpu = np.median(depth_recovery_errors(gd, s))
    e_ref = np.median(depth_recovery_errors(rd, s))
    assert abs(e_gpu - e_ref) < 0.1, (e_gpu, e_ref)


def test_config2_batched_sampled_positions_all_curves(umi, config2):
    b, W, tr, de = config2
    rng = np.random.default_rng(5)
    for i in range(b.B):
        x = b.curve(i)
        n = x.size
        pos = np.unique(np.concatenate([[0, 1, 179, 180, 181, n // 2 - 361, n // 2 + 361, n - 2, n - 1],
                                        rng.integers(0, n, 6)]))
        pos = pos[(pos >= 0) & (pos < n)]
        ref = oracle.detrend_positions(x, W[i], pos)
        o = b.offsets[i]
        compare_trend(tr[o + pos], ref["trend"], what="config2 curve %d" % i)
        compare_detr(de[o + pos], ref["detr"], what="config2 curve %d" % i)


def test_config3_uneven_batch(umi):
    b = synth.config3(n_curves=96)
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    assert set(W.tolist()) == {25, 361}
    flux = torch.from_numpy(b.flux).cuda()
    tr, de = umi.detrend_batched(flux, b.offsets, W)
    torch.cuda.synchronize()
    tr, de = tr.cpu().numpy(), de.cpu().numpy()
    rt, rd = oracle.detrend_batch(b.flux, b.offsets, W)
    compare_trend(tr, rt, what="config3")
    compare_detr(de, rd, what="config3")
    # One launch per curve: bit-identical where the curve alone plans to the
    # same kernel variant as its band in the batch, else the same up to the
    # rounding of the lane-split sums (the parity tolerance).
    lens = np.diff(b.offsets)
    same = differ = 0
    for i in range(0, b.B, 7):
        x = torch.from_numpy(b.curve(i).copy()).cuda()
        t1, d1 = umi.detrend(x, int(W[i]))
        torch.cuda.synchronize()
        s = slice(b.offsets[i], b.offsets[i + 1])
        band = umi.get_plan(int(W[i]), int(lens[W == W[i]].sum()))
        alone = umi.get_plan(int(W[i]), int(lens[i]))
        if band["variant"] == alone["variant"]:
            same += 1
            assert np.array_equal(t1.cpu().numpy(), tr[s], equal_nan=True)
            assert np.array_equal(d1.cpu().numpy(), de[s], equal_nan=True)
        else:
            differ += 1
            compare_trend(t1.cpu().numpy(), tr[s].astype(np.float64), what="alone vs batch %d" % i)
            compare_detr(d1.cpu().numpy(), de[s].astype(np.float64), what="alone vs batch %d" % i)
    assert same + differ > 0 and differ > 0          # single curves take latency plans here


def test_config4_large_window_sampled(umi):
    b = synth.config4(n_curves=6)
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    assert np.all(W == 2161)
    flux = torch.from_numpy(b.flux).cuda()
    tr, de = umi.detrend_batched(flux, b.offsets, W)
    torch.cuda.synchronize()
    tr, de = tr.cpu().numpy(), de.cpu().numpy()
    rng = np.random.default_rng(8)
    for i in range(b.B):
        x = b.curve(i)
        n = x.size
        g0 = int(np.argmax(np.isnan(x)))
        pos = np.unique(np.concatenate([np.arange(0, 40), np.arange(n - 40, n),
                                        np.arange(g0 - 1100, g0 + 20), rng.integers(0, n, 300)]))
        ref = oracle.detrend_positions(x, 2161, pos)
        o = b.offsets[i]
        compare_trend(tr[o + pos], ref["trend"], what="config4 curve %d" % i)
        compare_detr(de[o + pos], ref["detr"], what="config4 curve %d" % i)


def test_batch_with_empty_and_tiny_curves(umi):
    lens = [0, 5, 0, 1, 2000, 0, 3, 700]
    Ws = [3, 361, 25, 1, 361, 7, 2161, 25]
    xs = [synth.random_curve(40 + k, n) for k, n in enumerate(lens)]
    flux = np.concatenate(xs).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    tr, de = umi.detrend_batched(torch.from_numpy(flux).cuda(), off, np.array(Ws, np.int32))
    torch.cuda.synchronize()
    tr = tr.cpu().numpy()
    for k in range(len(lens)):
        if lens[k] == 0:
            continue
        ref = oracle.detrend(xs[k], Ws[k])
        compare_trend(tr[off[k]:off[k + 1]], ref["trend"], what="curve %d" % k)


def test_graph_cache_and_host_entry_point_identical(umi):
    b = synth.config3(n_curves=24)
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    flux = torch.from_numpy(b.flux).cuda()
    umi.set_graph_cache(False)
    t0, d0 = umi.detrend_batched(flux, b.offsets, W)
    umi.set_graph_cache(True)
    outs = [umi.detrend_batched(flux, b.offsets, W) for _ in range(3)]  # capture, then replays
    torch.cuda.synchronize()
    for t, d in outs:
        assert torch.equal(torch.nan_to_num(t, 7.0), torch.nan_to_num(t0, 7.0))
        assert torch.equal(torch.nan_to_num(d, 7.0), torch.nan_to_num(d0, 7.0))
    pinned = torch.from_numpy(b.flux).pin_memory()
    th = torch.empty(b.flux.size, dtype=torch.float32).pin_memory()
    dh = torch.empty(b.flux.size, dtype=torch.float32).pin_memory()
    umi.detrend_batched_host(pinned, b.offsets, W, trend=th, detr=dh)
    assert np.array_equal(th.numpy(), t0.cpu().numpy(), equal_nan=True)
    assert np.array_equal(dh.numpy(), d0.cpu().numpy(), equal_nan=True)


def test_autotune_keeps_parity(umi, tmp_path):
    try:
        plan, ms = umi.autotune(361, positions=300000)
        assert plan["lanes"] * plan["slots"] >= 361 and ms > 0 and plan["latency"] == 0
        assert umi.get_plan(361, -1)["chain"] == plan["chain"]
        x = synth.config1().curve(0)
        compare_diag(run_diag(umi, x, 361), oracle.detrend(x, 361), what="tuned")
        # A single TESS-sized curve is a latency-regime band: tuned separately,
        # used as tuned at the size it was tuned at, and kept by save/load.
        small, _ = umi.autotune(361, positions=12500)
        assert small["latency"] == 1
        assert umi.get_plan(361, 12500) == small
        assert umi.get_plan(361, -1)["chain"] == plan["chain"]
        f = tmp_path / "tuning.txt"
        umi.save_tuning(str(f))
        umi.clear_tuning()
        umi.load_tuning(str(f))
        assert umi.get_plan(361, 12500) == small
        assert umi.get_plan(361, -1)["chain"] == plan["chain"]
        xs = synth.random_curve(91, 12500)
        compare_diag(run_diag(umi, xs, 361), oracle.detrend(xs, 361), what="tuned latency plan")
    finally:
        umi.clear_tuning()


def test_autotune_batch_keeps_parity(umi):
    """Plans tuned on a batch (its own curves, or synthetic curves of its
    lengths) are throughput plans, become the band's plan, and keep parity on
    that batch; the tuner leaves the caller's flux untouched."""
    try:
        b = synth.config3(n_curves=48)
        W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
        lens = np.diff(b.offsets)
        flux = torch.from_numpy(b.flux).cuda()
        tess = np.flatnonzero(W == 361)
        own = torch.cat([flux[int(b.offsets[i]):int(b.offsets[i + 1])] for i in tess] * 8)
        before = own.clone()
        plan, ms = umi.autotune_batch(361, np.tile(lens[tess], 8), flux=own)
        torch.cuda.synchronize()
        assert torch.equal(own.isnan(), before.isnan()) and torch.equal(own.nan_to_num(), before.nan_to_num())
        assert plan["latency"] == 0 and ms > 0 and plan["lanes"] * plan["slots"] >= 361
        assert umi.get_plan(361, -1)["chain"] == plan["chain"]
        kplan, _ = umi.autotune_batch(25, np.tile(lens[W == 25], 8))
        assert kplan["latency"] == 0 and kplan["lanes"] * kplan["slots"] >= 25
        tr, de = umi.detrend_batched(flux, b.offsets, W)
        torch.cuda.synchronize()
        rt, rd = oracle.detrend_batch(b.flux, b.offsets, W)
        compare_trend(tr.cpu().numpy(), rt, what="batch-tuned config3")
        compare_detr(de.cpu().numpy(), rd, what="batch-tuned config3")
    finally:
        umi.clear_tuning()


def test_autotune_batch_tiny_curves(umi):
    """Curves shorter than, equal to and just past the window, each a
    single partial tile: a latency-regime band whose tuned plan serves such a
    batch with parity."""
    try:
        lens = np.array([1, 3, 24, 25, 26, 60], np.int64)
        plan, ms = umi.autotune_batch(25, lens)
        assert plan["latency"] == 1 and ms > 0 and plan["lanes"] * plan["slots"] >= 25
        assert umi.get_plan(25, int(lens.sum())) == plan
        xs = [synth.random_curve(300 + i, int(n), nan_frac=0.1) for i, n in enumerate(lens)]
        flux = np.concatenate(xs).astype(np.float32)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        W = np.full(lens.size, 25, np.int32)
        tr, de = umi.detrend_batched(torch.from_numpy(flux).cuda(), off, W)
        torch.cuda.synchronize()
        rt, rd = oracle.detrend_batch(flux, off, W)
        compare_trend(tr.cpu().numpy(), rt, what="tiny curves")
        compare_detr(de.cpu().numpy(), rd, what="tiny curves")
    finally:
        umi.clear_tuning()


def test_plan_rule_choices(umi):
    """The planner's regimes on this GPU: single curves take a 32-lane
    variant where one covers W within 2W (every window can start a chain),
    large bands the smallest covering capacity with long chains."""
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("thresholds are stated for 152 SMs")
    umi.clear_tuning()
    p = umi.get_plan(361, 12500)
    assert (p["lanes"], p["slots"], p["latency"], p["threads"]) == (32, 12, 1, 128)
    p = umi.get_plan(361, 18_000_000)
    assert (p["lanes"], p["slots"], p["latency"], p["chain"], p["threads"]) == (8, 46, 0, 136, 256)
    p = umi.get_plan(361, 288_000)                     # fills the GPU: throughput, shorter chain
    assert (p["lanes"], p["latency"]) == (8, 0) and p["chain"] < 136
    p = umi.get_plan(25, 37000)                        # no 32-lane variant near W = 25
    assert (p["lanes"], p["slots"], p["latency"]) == (1, 32, 1)
    assert umi.get_plan(25, 22_000_000)["slots"] == 26
    p = umi.get_plan(2161, 90000)
    assert (p["lanes"], p["slots"], p["latency"]) == (32, 68, 0)
    p = umi.get_plan(721, 30000)
    assert (p["lanes"], p["slots"], p["latency"]) == (16, 48, 1)


def _compiled_variants():
    import glob
    import os
    import re
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2604_06602_gb300", "csrc")
    out = []
    for f in sorted(glob.glob(os.path.join(root, "umi_variants_*.cu"))):
        for m in re.finditer(r"^UMI_DEFINE_VARIANT\((\d+),\s*(\d+),\s*(\d+)\)", open(f).read(), re.M):
            out.append(tuple(int(v) for v in m.groups()))
    assert len(out) >= 10
    return out


@pytest.mark.parametrize("variant", _compiled_variants())
def test_every_variant_forced(umi, tmp_path, variant):
    """Each compiled variant, forced through a tuning line for both regimes,
    at its full capacity and at a third of it (the general load path), over
    several tiles with a ragged tail, against the oracle."""
    G, R, M = variant
    S = G * R
    chain = 5 if G == 32 else 3 * G
    gpu = torch.cuda.get_device_name()
    try:
        for W in sorted({S - 1, max(1, (S // 3) | 1)}):
            f = tmp_path / "force.txt"
            f.write_text("".join("%s|%d|%s|%d|%d|%d|%d|128\n" % (gpu, W, r, G, R, M, chain)
                                 for r in ("throughput", "latency")))
            umi.clear_tuning()
            umi.load_tuning(str(f))
            tile = (32 // G) * chain
            n = max(16 * tile + 37, 2 * W + 101)
            pl = umi.get_plan(W, n)
            assert (pl["lanes"], pl["slots"]) == (G, R)
            x = synth.random_curve(7000 + S + W, n, nan_runs=2, run_len=(1, W))
            compare_diag(run_diag(umi, x, W), oracle.detrend(x, W), what="forced %s W=%d" % (variant, W))
    finally:
        umi.clear_tuning()


@pytest.mark.parametrize("variant", [(2, 32, 3), (4, 32, 3), (8, 46, 2), (16, 24, 4)])
def test_short_chains_forced(umi, tmp_path, variant):
    """Chains shorter than the group width (the groups of a warp then walk
    overlapping windows) for each narrow variant, forced through tuning lines
    in both regimes, against the oracle with gaps and a ragged tail."""
    G, R, M = variant
    S = G * R
    gpu = torch.cuda.get_device_name()
    try:
        for chain in sorted({1, max(1, G // 2), G - 1}):
            W = S - 2 if (S - 2) % 2 else S - 3
            f = tmp_path / "short.txt"
            f.write_text("".join("%s|%d|%s|%d|%d|%d|%d|128\n" % (gpu, W, r, G, R, M, chain)
                                 for r in ("throughput", "latency")))
            umi.clear_tuning()
            umi.load_tuning(str(f))
            n = 37 * (32 // G) * chain + 2 * W + 13
            pl = umi.get_plan(W, n)
            assert (pl["lanes"], pl["slots"], pl["chain"]) == (G, R, chain)
            x = synth.random_curve(9100 + S + chain, n, nan_runs=2, run_len=(1, W))
            compare_diag(run_diag(umi, x, W), oracle.detrend(x, W),
                         what="short chain %d %s W=%d" % (chain, variant, W))
    finally:
        umi.clear_tuning()


def test_stream_ordering_on_side_stream(umi):
    x = synth.config1().curve(0)[:5000].copy()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xd = torch.from_numpy(x).cuda(non_blocking=False)
        tr, de = umi.detrend(xd, 361, stream=s)
    s.synchronize()
    compare_trend(tr.cpu().numpy(), oracle.detrend(x, 361)["trend"], what="side stream")


def test_graph_cache_follows_tuning_changes(umi, tmp_path):
    """A cached graph must not replay a plan that tuning has since replaced."""
    import torch as _t
    b = synth.config2(n_curves=8, n=6000)
    W = np.full(b.B, 361, np.int32)
    flux = _t.from_numpy(b.flux).cuda()
    tr = _t.empty_like(flux)
    de = _t.empty_like(flux)
    gpu = _t.cuda.get_device_name()
    try:
        umi.set_graph_cache(True)
        umi.detrend_batched(flux, b.offsets, W, trend=tr, detr=de)
        launches0 = umi.kernel_launch_count()
        assert umi.get_plan(361, 48000)["latency"] == 1
        assert umi.get_plan(361, 48000)["lanes"] == 32
        f = tmp_path / "tune.txt"
        f.write_text("%s|361|32|12|4|24|128\n%s|361|latency|16|24|4|16|128\n" % (gpu, gpu))
        umi.load_tuning(str(f))
        assert umi.get_plan(361, -1)["lanes"] == 32      # a line without regime: throughput
        assert umi.get_plan(361, 48000)["lanes"] == 16
        umi.detrend_batched(flux, b.offsets, W, trend=tr, detr=de)
        _t.cuda.synchronize()
        ref = oracle.detrend_batch(b.flux, b.offsets, W)[0]
        compare_trend(tr.cpu().numpy(), ref, what="retuned graph")
        assert umi.kernel_launch_count() > launches0
    finally:
        umi.clear_tuning()


@pytest.mark.parametrize("W", [25, 361, 2161])
@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_mad_scale_mode(umi, W, alpha):
    """MAD scale (the comparison estimator; alpha 1 is the symmetric
    biweight).  The GPU's MAD is the FP32 rounding of the exact MAD (|x - m|
    is correctly rounded and rounding is monotone), so the scale agrees to one
    FP32 ulp; the trend to 1e-5."""
    n = 3 * tile_of(umi, W) + 11
    x = synth.random_curve(77 + W, n, nan_runs=3, run_len=(1, W))
    x[::41] -= 5e-3                                      # dips below the median
    p = umi.params(alpha=alpha, scale_mode=umi.SCALE_MAD)
    got = run_diag(umi, x, W, p)
    ref = oracle.detrend(x, W, alpha=alpha, scale_mode=oracle.SCALE_MAD)
    compare_diag(got, ref, what="MAD W=%d alpha=%g" % (W, alpha))
    ok = ~np.isnan(ref["scale"])
    np.testing.assert_allclose(got["scale"][ok], ref["scale"][ok], rtol=2 ** -23, atol=0)
    # The same through the batched path.
    xd = torch.from_numpy(x).cuda()
    tr, _ = umi.detrend_batched(xd, np.array([0, n]), np.array([W], np.int32), p)
    torch.cuda.synchronize()
    assert np.array_equal(tr.cpu().numpy(), got["trend"], equal_nan=True)


def test_mad_degenerate_and_ties(umi):
    """Half the window on one value gives MAD 0 and the median as trend."""
    x = np.ones(900, np.float32)
    x[::3] = 1.5
    x[1::7] = np.nan
    p = umi.params(scale_mode=umi.SCALE_MAD)
    got = run_diag(umi, x, 61, p)
    ref = oracle.detrend(x, 61, scale_mode=oracle.SCALE_MAD)
    compare_diag(got, ref, what="MAD ties")


def test_host_entry_point_pipelined_chunks_identical(umi):
    """Large host batches are split into pipelined chunks of whole curves;
    the output must equal the device-resident batched call bit for bit."""
    b = synth.config3(n_curves=400)                 # about 1e7 samples, mixed windows
    W = np.array([umi.window_length(c) for c in b.cadence], np.int32)
    umi.set_graph_cache(False)
    t0, d0 = umi.detrend_batched(torch.from_numpy(b.flux).cuda(), b.offsets, W)
    umi.set_graph_cache(True)
    fh = torch.from_numpy(b.flux).pin_memory()
    th = torch.empty(b.flux.size, dtype=torch.float32).pin_memory()
    dh = torch.empty(b.flux.size, dtype=torch.float32).pin_memory()
    umi.detrend_batched_host(fh, b.offsets, W, trend=th, detr=dh)
    assert b.flux.size > 4 * (2 << 20)
    assert np.array_equal(th.numpy(), t0.cpu().numpy(), equal_nan=True)
    assert np.array_equal(dh.numpy(), d0.cpu().numpy(), equal_nan=True)
    # Pageable numpy buffers take the same path (copies serialise).
    tn, dn = umi.detrend_batched_host(b.flux, b.offsets, W)
    assert np.array_equal(tn, t0.cpu().numpy(), equal_nan=True)


@pytest.mark.parametrize("n,W,parts", [(300000, 2161, 3), (200000, 361, 4)])
def test_split_long_curve_matches_whole(umi, n, W, parts):
    """One long curve cut into halo-padded parts, as it would be spread over
    several GPUs, gives the whole-curve output: bit for bit where a part plans
    to the same kernel variant as the whole curve, else within the rounding
    of the lane-split sums."""
    from paper_2604_06602_gb300 import partition
    x = synth.random_curve(515 + W, n, nan_runs=3, run_len=(1, 3000))
    xd = torch.from_numpy(x).cuda()
    t0, d0 = umi.detrend(xd, W)
    torch.cuda.synchronize()
    t0, d0 = t0.cpu().numpy(), d0.cpu().numpy()
    whole = umi.get_plan(W, n)["variant"]
    kinds = set()
    for a, b, lo, hi in partition.split_curve(n, W, parts):
        t, d = umi.detrend(xd[lo:hi].contiguous(), W)
        torch.cuda.synchronize()
        t, d = t.cpu().numpy()[a - lo:b - lo], d.cpu().numpy()[a - lo:b - lo]
        if umi.get_plan(W, hi - lo)["variant"] == whole:
            kinds.add("same")
            assert np.array_equal(t, t0[a:b], equal_nan=True)
            assert np.array_equal(d, d0[a:b], equal_nan=True)
        else:
            kinds.add("differ")
            compare_trend(t, t0[a:b].astype(np.float64), what="part %d" % a)
            compare_detr(d, d0[a:b].astype(np.float64), what="part %d" % a)
    assert kinds == ({"same"} if W == 2161 else {"differ"})


@pytest.mark.parametrize("W", [7, 25, 61, 129, 361, 721, 2161])
def test_random_parameters(umi, W):
    """Seeded random estimator parameters (alpha on both sides of 1, c, the
    iteration count, min_valid, both scale modes) on gappy curves, against
    the oracle."""
    rng = np.random.default_rng(4000 + W)
    for trial in range(3):
        alpha = float(np.exp(rng.uniform(np.log(0.3), np.log(12.0))))
        c = float(rng.uniform(1.5, 8.0))
        iters = int(rng.integers(0, 10))
        min_valid = int(rng.choice([-1, 0, W // 2, W]))
        mad = bool(trial == 2)
        n = int(rng.integers(2 * W + 50, 4 * W + 500))
        x = synth.random_curve(5000 + 10 * W + trial, n, nan_frac=0.03, nan_runs=2, run_len=(1, W),
                               ties=bool(trial == 1))
        p = umi.params(alpha=alpha, c=c, iters=iters, min_valid=min_valid,
                       scale_mode=umi.SCALE_MAD if mad else umi.SCALE_UPPER_RMS)
        ref = oracle.detrend(x, W, alpha=alpha, c=c, iters=iters, min_valid=min_valid,
                             scale_mode=oracle.SCALE_MAD if mad else oracle.SCALE_UPPER_RMS)
        compare_diag(run_diag(umi, x, W, p), ref, c=c,
                     what="W=%d alpha=%.3g c=%.3g iters=%d min_valid=%d mad=%d"
                     % (W, alpha, c, iters, min_valid, mad))
