"""Runs representative detrend calls through the checked build
(libumi_checked.so, every kernel checking its indices) and compares each
result with the oracle.  Invoked by test_checked_build.py in a subprocess,
because a process loads one libumi; prints one JSON line."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

import oracle  # noqa: E402
from paper_2604_06602_gb300 import build as _build  # noqa: E402
from paper_2604_06602_gb300 import synth  # noqa: E402
from tests.helpers import compare_diag, compare_trend  # noqa: E402


def main():
    _build.LIB = _build.build(checked=True)
    from paper_2604_06602_gb300 import umi
    umi.load()
    assert umi.checked_build()
    umi.check_flags(clear=True)
    cases = 0
    # Single curves at variant capacity edges, short and ragged lengths, gaps.
    for W in (1, 3, 25, 27, 63, 65, 191, 193, 361, 385, 769, 1537, 2161, 4095):
        for n in sorted({1, max(1, W - 1), W + 1, 3 * W + 17, 5000}):
            x = synth.random_curve(900 + W + n, n, nan_runs=2, run_len=(1, W))
            xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
            out = umi.detrend_diag(xd, W)
            torch.cuda.synchronize()
            got = {k: v.cpu().numpy() for k, v in out.items()}
            compare_diag(got, oracle.detrend(x, W), what="checked W=%d n=%d" % (W, n))
            cases += 1
    # A mixed batch (several bands, empty curves), the MAD scale, the host
    # pipeline, the segmented path, the no-allocation path and the server.
    lens = [0, 5, 3000, 1, 20000, 0, 777, 9000, 40000]
    Ws = [3, 361, 25, 1, 361, 7, 2161, 25, 361]
    xs = [synth.random_curve(50 + k, n, nan_runs=1, run_len=(1, 500)) for k, n in enumerate(lens)]
    flux = np.concatenate(xs).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    Wv = np.array(Ws, np.int32)
    fd = torch.from_numpy(flux).cuda()
    for p, mode in ((umi.params(), oracle.SCALE_UPPER_RMS),
                    (umi.params(alpha=1.0, scale_mode=umi.SCALE_MAD), oracle.SCALE_MAD)):
        tr, _ = umi.detrend_batched(fd, off, Wv, p)
        torch.cuda.synchronize()
        tr = tr.cpu().numpy()
        for k in range(len(lens)):
            if lens[k]:
                ref = oracle.detrend(xs[k], Ws[k], alpha=p.alpha, scale_mode=mode)["trend"]
                compare_trend(tr[off[k]:off[k + 1]], ref, what="checked batch %d" % k)
        cases += 1
    th, _ = umi.detrend_batched_host(flux, off, Wv)
    tn, _ = umi.detrend_batched_noalloc(fd, off, Wv)
    ts, _, _ = umi.detrend_segmented(fd, off, Wv)
    torch.cuda.synchronize()
    for k in range(len(lens)):
        if lens[k]:
            ref = oracle.detrend(xs[k], Ws[k])["trend"]
            s = slice(off[k], off[k + 1])
            compare_trend(th[s], ref, what="checked host %d" % k)
            compare_trend(tn.cpu().numpy()[s], ref, what="checked noalloc %d" % k)
            rs, _, _ = oracle.detrend_segmented(xs[k], Ws[k])
            compare_trend(ts.cpu().numpy()[s], rs, what="checked segmented %d" % k)
    cases += 3
    with umi.Server(mem_budget_bytes=1 << 30, n_streams=2, max_batch_curves=4) as srv:
        tickets = [srv.submit(x, W) for x, W in zip(xs, Ws) if x.size]
        for t in tickets:
            srv.wait(t, 60.0)
        for (x, W), t in zip([(x, W) for x, W in zip(xs, Ws) if x.size], tickets):
            tr, _ = srv.copy_out(t, x.size)
            compare_trend(tr, oracle.detrend(x, W)["trend"], what="checked server W=%d" % W)
            srv.release(t)
    cases += 1
    flags = umi.check_flags()
    print(json.dumps({"checked": True, "flags": flags, "cases": cases,
                      "launches": umi.kernel_launch_count()}))


if __name__ == "__main__":
    main()
