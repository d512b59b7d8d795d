"""Continuous-batching server on the GPU: each result is the same alone and in
a mix (the batches here stay small enough that every band plans to the same
kernel variant as the curve alone, so bit for bit), admission respects the
memory budget, errors are reported per request, and injected host-side
failures fail only the affected requests."""
import time

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


def curves_mix(n=40):
    out = []
    for i in range(n):
        kind = i % 3
        if kind == 0:
            x = synth.random_curve(500 + i, 3000 + 97 * i, nan_runs=2)
            W = 361
        elif kind == 1:
            x = synth.random_curve(500 + i, 1500 + 31 * i, nan_frac=0.02)
            W = 25
        else:
            x = synth.random_curve(500 + i, 5000 + 11 * i)
            W = 2161
        out.append((x, W))
    return out


def alone(umi, x, W):
    xd = torch.from_numpy(x).cuda()
    t, d = umi.detrend(xd, W)
    torch.cuda.synchronize()
    return t.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("busy_poll", [1, 0])
def test_alone_equals_mix(umi, busy_poll):
    mix = curves_mix()
    with umi.Server(mem_budget_bytes=1 << 30, n_streams=3, max_batch_curves=8,
                    busy_poll=busy_poll) as srv:
        tickets = [srv.submit(x, W) for x, W in mix]
        for t in tickets:
            srv.wait(t, 120.0)
        for (x, W), t in zip(mix, tickets):
            tr, de = srv.copy_out(t, x.size)
            ta, da = alone(umi, x, W)
            assert np.array_equal(tr, ta, equal_nan=True)
            assert np.array_equal(de, da, equal_nan=True)
            res = srv.poll(t)
            assert res is not None and res[2] > 0
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == len(mix) and st["failed"] == 0
        assert st["batches_launched"] >= len(mix) // 8
        assert st["resident_bytes"] == 0


def test_device_inputs_and_poll_pointers(umi):
    x = synth.random_curve(3, 4000)
    xd = torch.from_numpy(x).cuda()
    with umi.Server(mem_budget_bytes=64 << 20) as srv:
        launches0 = umi.kernel_launch_count()
        t = srv.submit(xd, 361)
        srv.wait(t, 60.0)
        assert umi.kernel_launch_count() > launches0     # server kernels are counted too
        tr_ptr, de_ptr, lat = srv.poll(t)
        assert tr_ptr and de_ptr and lat > 0
        tl = srv.timeline(t)
        assert 0 <= tl["admit"] <= tl["launch"] <= tl["done"] and tl["done"] == lat
        tr, _ = srv.copy_out(t, x.size)
        ta, _ = alone(umi, x, 361)
        assert np.array_equal(tr, ta, equal_nan=True)
        srv.release(t)
        with pytest.raises(umi.UmiError):
            srv.timeline(t)                               # released: unknown ticket


def test_budget_backpressure(umi):
    """A budget that holds two curves: later requests wait for releases."""
    n = 20000
    per = 3 * ((4 * n + 255) // 256 * 256)
    xs = [synth.random_curve(70 + i, n) for i in range(6)]
    with umi.Server(mem_budget_bytes=2 * per + 1024, n_streams=2) as srv:
        tickets = [srv.submit(x, 361) for x in xs]
        srv.wait(tickets[0], 60.0)
        srv.wait(tickets[1], 60.0)
        time.sleep(0.05)
        assert srv.poll(tickets[2]) is None            # no memory yet
        st = srv.stats()
        assert st["queued_requests"] == 4 and st["peak_resident_bytes"] <= 2 * per
        for i, t in enumerate(tickets):
            srv.wait(t, 60.0)
            tr, _ = srv.copy_out(t, n)
            ta, _ = alone(umi, xs[i], 361)
            assert np.array_equal(tr, ta, equal_nan=True)
            srv.release(t)
        assert srv.stats()["peak_resident_bytes"] <= 2 * per


def test_withdraw_queued_requests(umi):
    """Queued requests released before admission never run; the queue moves on
    to the ones behind them once memory frees up."""
    n = 20000
    per = 3 * ((4 * n + 255) // 256 * 256)
    xs = [synth.random_curve(170 + i, n) for i in range(6)]
    with umi.Server(mem_budget_bytes=2 * per + 1024, n_streams=2) as srv:
        tickets = [srv.submit(x, 361) for x in xs]
        srv.wait(tickets[0], 60.0)
        srv.wait(tickets[1], 60.0)
        time.sleep(0.05)
        assert srv.poll(tickets[2]) is None              # still queued: no memory
        srv.release(tickets[3])                          # withdrawn while queued
        srv.release(tickets[4])
        for t in tickets[3:5]:
            with pytest.raises(umi.UmiError) as e:
                srv.poll(t)
            assert e.value.status == umi.UMI_ERR_UNKNOWN_TICKET
        for i in (0, 1):
            srv.release(tickets[i])
        for i in (2, 5):
            srv.wait(tickets[i], 60.0)
            tr, _ = srv.copy_out(tickets[i], n)
            ta, _ = alone(umi, xs[i], 361)
            assert np.array_equal(tr, ta, equal_nan=True)
            srv.release(tickets[i])
        st = srv.stats()
        assert st["completed"] == 4 and st["admitted"] == 4 and st["released"] == 6
        assert st["resident_bytes"] == 0 and st["queued_requests"] == 0


def test_errors(umi):
    with umi.Server(mem_budget_bytes=1 << 20) as srv:
        x = synth.random_curve(1, 1000)
        with pytest.raises(umi.UmiError) as e:
            srv.submit(x, 360)
        assert e.value.status == umi.UMI_ERR_INVALID_ARG
        with pytest.raises(umi.UmiError) as e:
            srv.submit(synth.random_curve(2, 200000), 361)   # can never fit 1 MiB
        assert e.value.status == umi.UMI_ERR_BUSY
        with pytest.raises(umi.UmiError) as e:
            srv.poll(12345)
        assert e.value.status == umi.UMI_ERR_UNKNOWN_TICKET
        t = srv.submit(x, 361)
        srv.wait(t, 60.0)
        srv.release(t)
        with pytest.raises(umi.UmiError) as e:
            srv.release(t)
        assert e.value.status == umi.UMI_ERR_UNKNOWN_TICKET
        assert srv.stats()["rejected"] == 1


@pytest.mark.parametrize("busy_poll", [1, 0])
def test_injected_failures_only_hit_their_requests(umi, busy_poll):
    mix = curves_mix(12)
    # max_wait_s holds a partial batch back, so the four requests of one
    # window length submitted together form one batch of max_batch_curves = 4.
    same = [m for m in mix if m[1] == 361][:4]
    mix = same + [m for m in mix if m[1] != 361]
    with umi.Server(mem_budget_bytes=1 << 30, n_streams=1, max_batch_curves=4,
                    max_wait_s=2.0, busy_poll=busy_poll) as srv:
        srv.inject_fault(1, 1)                        # the next batch fails to launch
        first = [srv.submit(x, W) for x, W in mix[:4]]
        for t in first:
            with pytest.raises(umi.UmiError) as e:
                srv.wait(t, 60.0)
            assert e.value.status == umi.UMI_ERR_FAILED
        srv.inject_fault(2, 2)                        # two admissions fail
        rest = [srv.submit(x, W) for x, W in mix[4:]]
        outcomes = []
        for t in rest:
            try:
                srv.wait(t, 60.0)
                outcomes.append("ok")
            except umi.UmiError as e:
                assert e.status == umi.UMI_ERR_FAILED
                outcomes.append("failed")
        assert outcomes.count("failed") == 2 and outcomes[:2] == ["failed", "failed"]
        for (x, W), t, o in zip(mix[4:], rest, outcomes):
            if o == "ok":
                tr, _ = srv.copy_out(t, x.size)
                ta, _ = alone(umi, x, W)
                assert np.array_equal(tr, ta, equal_nan=True)
        for t in first + rest:
            srv.release(t)
        assert srv.stats()["resident_bytes"] == 0


def test_wait_timeout_is_reported(umi):
    with umi.Server(mem_budget_bytes=64 << 20, n_streams=1) as srv:
        # A queued request that cannot be admitted (slots full) times out cleanly.
        pass
    with umi.Server(mem_budget_bytes=64 << 20, max_slots=1) as srv:
        a = srv.submit(synth.random_curve(1, 2000), 25)
        b = srv.submit(synth.random_curve(2, 2000), 25)
        srv.wait(a, 60.0)
        with pytest.raises(umi.UmiError) as e:
            srv.wait(b, 0.05)                            # a holds the only slot
        assert e.value.status == umi.UMI_ERR_TIMEOUT
        srv.release(a)
        srv.wait(b, 60.0)
        srv.release(b)


def test_mixed_scale_modes_and_params_in_one_batch(umi):
    """Requests with different parameters (including the MAD scale, which
    runs a different kernel build) share batches and still match their own
    single-curve results."""
    mix = curves_mix(18)
    presets = [umi.params(), umi.params(alpha=1.0, scale_mode=umi.SCALE_MAD),
               umi.params(alpha=10.0, c=2.5), umi.params(iters=2, min_valid=0)]
    with umi.Server(mem_budget_bytes=1 << 30, n_streams=1, max_batch_curves=64,
                    max_wait_s=0.5) as srv:
        tickets = [srv.submit(x, W, presets[i % len(presets)]) for i, (x, W) in enumerate(mix)]
        for t in tickets:
            srv.wait(t, 120.0)
        assert srv.stats()["batches_launched"] <= 3
        for i, ((x, W), t) in enumerate(zip(mix, tickets)):
            tr, _ = srv.copy_out(t, x.size)
            xd = torch.from_numpy(x).cuda()
            ta, _ = umi.detrend(xd, W, presets[i % len(presets)])
            torch.cuda.synchronize()
            assert np.array_equal(tr, ta.cpu().numpy(), equal_nan=True)
            srv.release(t)


@pytest.mark.parametrize("by_window,expected", [(1, 3), (0, 1)])
def test_batches_by_window_length(umi, by_window, expected):
    """Requests held together by max_wait_s: one batch per window length with
    batch_by_window (the default), one batch in arrival order otherwise;
    results are the same."""
    mix = curves_mix(12)
    with umi.Server(mem_budget_bytes=1 << 30, n_streams=4, max_batch_curves=64,
                    max_wait_s=0.5, batch_by_window=by_window) as srv:
        tickets = [srv.submit(x, W) for x, W in mix]
        for t in tickets:
            srv.wait(t, 60.0)
        assert srv.stats()["batches_launched"] == expected
        for (x, W), t in zip(mix, tickets):
            tr, _ = srv.copy_out(t, x.size)
            ta, _ = alone(umi, x, W)
            assert np.array_equal(tr, ta, equal_nan=True)
            srv.release(t)


@pytest.mark.parametrize("priority_window", [0, 1025, 26])
def test_stream_priorities(umi, priority_window):
    """Long windows on the low-priority half of the streams (the default
    threshold 1025, a threshold that sends W = 361 there too, and none):
    every result equals the curve alone, and no class starves."""
    mix = curves_mix(30)
    with umi.Server(mem_budget_bytes=1 << 30, n_streams=4, max_batch_curves=4,
                    priority_window=priority_window) as srv:
        tickets = [srv.submit(x, W) for x, W in mix]
        for t in tickets:
            srv.wait(t, 120.0)
        for (x, W), t in zip(mix, tickets):
            tr, _ = srv.copy_out(t, x.size)
            ta, _ = alone(umi, x, W)
            assert np.array_equal(tr, ta, equal_nan=True)
            srv.release(t)
        assert srv.stats()["completed"] == len(mix)


def test_priority_config_checks(umi):
    with pytest.raises(umi.UmiError):
        umi.Server(mem_budget_bytes=1 << 20, priority_window=-1)
    # Priorities need window-homogeneous batches and two streams; otherwise they are off.
    with umi.Server(mem_budget_bytes=1 << 20, n_streams=1) as srv:
        x = synth.random_curve(5, 500)
        t = srv.submit(x, 25)
        srv.wait(t, 60.0)
        srv.release(t)


def test_served_results_match_oracle_on_serving_mixture(umi):
    """The production library's server against the FP64 oracle on a sample of
    the serving mixture (TESS 2-min, Kepler 29.4-min with gaps, TESS 20-s at
    W = 2161): 300 host-buffer requests, each its own slice of a tape of its
    class, submitted on a Poisson schedule at 20k/s so that they batch and
    overlap on the GPU.  Sampled positions of every request are checked one by
    one against the oracle (1e-5 relative, identical NaN pattern)."""
    import oracle
    from tests.helpers import compare_detr, compare_trend
    st = synth.serving_stream(n_requests=300, tape_samples=(400_000, 800_000, 600_000))
    Wk = [umi.window_length(c) for c in st.cadences]
    W_req = np.array(Wk, np.int32)[st.kind]
    assert set(np.unique(st.kind).tolist()) == {0, 1, 2}
    arrivals = st.arrivals / 20000.0
    rng = np.random.default_rng(5)
    with umi.Server(mem_budget_bytes=4 << 30, n_streams=4, max_batch_curves=64) as srv:
        tickets = []
        t0 = time.perf_counter()
        for i in range(st.n.size):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            tickets.append(srv.submit(st.flux(i), int(W_req[i])))
        for t in tickets:
            srv.wait(t, 120.0)
        assert srv.stats()["batches_launched"] < len(tickets)      # requests were batched
        for i, t in enumerate(tickets):
            x = st.flux(i)
            tr, de = srv.copy_out(t, x.size)
            srv.release(t)
            n, W = x.size, int(W_req[i])
            h = (W - 1) // 2
            pos = np.unique(np.concatenate([[0, n - 1, h, n - 1 - h], rng.integers(0, n, 12)]))
            ref = oracle.detrend_positions(x, W, pos)
            compare_trend(tr[pos], ref["trend"], what="request %d" % i)
            compare_detr(de[pos], ref["detr"], what="request %d" % i)
