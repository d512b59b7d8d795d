"""Calls from several host threads at once: the batched entry point (graph
cache, pinned staging ring, planner) on per-thread streams, the host-buffer
pipeline (per-thread side streams), and server submitters.  Every result must
equal the same call made alone, bit for bit."""
import threading

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


def batches(k):
    out = []
    for i in range(k):
        lens = [3000 + 997 * i, 1, 12000 - 500 * i, 777]
        Ws = [361, 25, 361 if i % 2 else 2161, 25]
        xs = [synth.random_curve(900 + 10 * i + j, n, nan_runs=1, run_len=(1, 200)) for j, n in enumerate(lens)]
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        out.append((np.concatenate(xs).astype(np.float32), off, np.array(Ws, np.int32)))
    return out


def run_threads(fn, items):
    results = [None] * len(items)
    errors = []

    def work(i):
        try:
            results[i] = fn(items[i])
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    th = [threading.Thread(target=work, args=(i,)) for i in range(len(items))]
    for t in th:
        t.start()
    for t in th:
        t.join(120)
    assert not errors, errors
    return results


def test_batched_from_threads(umi):
    items = batches(6)

    def alone(item):
        flux, off, W = item
        tr, _ = umi.detrend_batched(torch.from_numpy(flux).cuda(), off, W)
        torch.cuda.synchronize()
        return tr.cpu().numpy()

    ref = [alone(it) for it in items]

    def threaded(item):
        s = torch.cuda.Stream()
        flux, off, W = item
        got = []
        with torch.cuda.stream(s):
            fd = torch.from_numpy(flux).cuda()
            for _ in range(5):                          # repeats replay cached graphs
                tr, _ = umi.detrend_batched(fd, off, W, stream=s)
                s.synchronize()
                got.append(tr.cpu().numpy())
        return got

    for r, outs in zip(ref, run_threads(threaded, items)):
        for g in outs:
            assert np.array_equal(g, r, equal_nan=True)


def test_host_pipeline_from_threads(umi):
    items = batches(4)
    ref = [umi.detrend_batched_host(f, o, w)[0] for f, o, w in items]
    got = run_threads(lambda it: umi.detrend_batched_host(*it)[0], items)
    for r, g in zip(ref, got):
        assert np.array_equal(g, r, equal_nan=True)


def test_server_submitters_from_threads(umi):
    curves = [(synth.random_curve(700 + i, 2000 + 313 * i), (361, 25, 2161)[i % 3]) for i in range(24)]
    with umi.Server(mem_budget_bytes=1 << 30, n_streams=3, max_batch_curves=8) as srv:
        def submit_all(chunk):
            out = []
            for x, W in chunk:
                t = srv.submit(x, W)
                srv.wait(t, 60.0)
                tr, _ = srv.copy_out(t, x.size)
                srv.release(t)
                out.append(tr)
            return out

        chunks = [curves[i::4] for i in range(4)]
        got = run_threads(submit_all, chunks)
        assert srv.stats()["completed"] == len(curves)
    for chunk, outs in zip(chunks, got):
        for (x, W), tr in zip(chunk, outs):
            xd = torch.from_numpy(x).cuda()
            ta, _ = umi.detrend(xd, W)
            torch.cuda.synchronize()
            assert np.array_equal(tr, ta.cpu().numpy(), equal_nan=True)
