"""Command line for the library (every step runs in libumi's kernels).

    python -m paper_2604_06602_gb300 detrend IN.npz OUT.npz [options]
    python -m paper_2604_06602_gb300 plan W POSITIONS
    python -m paper_2604_06602_gb300 tune W POSITIONS [--save FILE]

`detrend` reads a CSR batch from IN (.npz with `flux` [total] and `offsets`
[B+1], plus either `W` [B] or `cadence` [B] in days; or a .npy of one curve,
which then needs --cadence or --W), detrends it on the GPU and writes `trend`
and `detr` (and `offsets`) to OUT.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def _load_batch(path, args, umi):
    if path.endswith(".npy"):
        flux = np.load(path).astype(np.float32).ravel()
        offsets = np.array([0, flux.size], np.int64)
        if args.W is not None:
            W = np.array([args.W], np.int32)
        elif args.cadence is not None:
            W = np.array([umi.window_length(args.cadence, args.window_days)], np.int32)
        else:
            raise SystemExit("a .npy input needs --W or --cadence")
        return flux, offsets, W
    z = np.load(path)
    flux = np.asarray(z["flux"], np.float32).ravel()
    offsets = np.asarray(z["offsets"], np.int64) if "offsets" in z else np.array([0, flux.size], np.int64)
    B = offsets.size - 1
    if "W" in z:
        W = np.asarray(z["W"], np.int32)
    elif "cadence" in z:
        W = np.array([umi.window_length(float(c), args.window_days) for c in np.asarray(z["cadence"]).ravel()],
                     np.int32)
    elif args.W is not None:
        W = np.full(B, args.W, np.int32)
    elif args.cadence is not None:
        W = np.full(B, umi.window_length(args.cadence, args.window_days), np.int32)
    else:
        raise SystemExit("the input needs W or cadence arrays, or --W / --cadence")
    if W.size != B:
        raise SystemExit("W has %d entries for %d curves" % (W.size, B))
    if np.any(W < 1):
        raise SystemExit("a cadence gave no valid window length")
    return flux, offsets, W


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2604_06602_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    d = sub.add_parser("detrend", help="detrend a CSR batch of light curves")
    d.add_argument("input")
    d.add_argument("output")
    d.add_argument("--W", type=int, default=None, help="window length for every curve")
    d.add_argument("--cadence", type=float, default=None, help="cadence in days for every curve")
    d.add_argument("--window-days", type=float, default=0.5)
    d.add_argument("--alpha", type=float, default=2.0)
    d.add_argument("--c", type=float, default=5.0)
    d.add_argument("--iters", type=int, default=5)
    d.add_argument("--min-valid", type=int, default=-1)
    d.add_argument("--mad", action="store_true", help="MAD scale instead of the upper RMS (Eq. 1)")
    d.add_argument("--segmented", action="store_true", help="split at gaps first (umi_detrend_segmented)")
    d.add_argument("--tuning", default=None, help="load kernel plans from this tuning file")
    p = sub.add_parser("plan", help="print the kernel plan for a window length and band size")
    p.add_argument("W", type=int)
    p.add_argument("positions", type=int)
    t = sub.add_parser("tune", help="autotune the plan for a window length and band size")
    t.add_argument("W", type=int)
    t.add_argument("positions", type=int)
    t.add_argument("--curve-len", type=int, default=None,
                   help="tune on curves of this many samples (positions / curve-len of them) "
                        "instead of one curve of `positions` samples")
    t.add_argument("--save", default=None, help="write the tuning table to this file")
    args = ap.parse_args(argv)

    from . import umi
    umi.load(build_if_missing=True)
    if args.cmd == "plan":
        print(json.dumps(umi.get_plan(args.W, args.positions)))
        return 0
    if args.cmd == "tune":
        if args.curve_len:
            plan, ms = umi.autotune_batch(args.W, [args.curve_len] * max(1, args.positions // args.curve_len))
        else:
            plan, ms = umi.autotune(args.W, positions=args.positions)
        print(json.dumps({"plan": plan, "ms": ms}))
        if args.save:
            umi.save_tuning(args.save)
        return 0

    import torch
    if args.tuning:
        umi.load_tuning(args.tuning)
    flux, offsets, W = _load_batch(args.input, args, umi)
    prm = umi.params(alpha=args.alpha, c=args.c, iters=args.iters, min_valid=args.min_valid,
                     scale_mode=umi.SCALE_MAD if args.mad else umi.SCALE_UPPER_RMS)
    out = {"offsets": offsets, "W": W}
    if args.segmented:
        tr, de, kept = umi.detrend_segmented(torch.from_numpy(flux).cuda(), offsets, W, prm)
        torch.cuda.synchronize()
        out.update(trend=tr.cpu().numpy(), detr=de.cpu().numpy(), segments=np.int64(kept))
    else:
        tr, de = umi.detrend_batched_host(flux, offsets, W, prm)
        out.update(trend=tr, detr=de)
    np.savez(args.output, **out)
    print(json.dumps({"curves": int(offsets.size - 1), "samples": int(flux.size),
                      "windows": sorted(set(int(w) for w in W))}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
