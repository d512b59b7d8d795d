#!/usr/bin/env python3
"""Benchmark of the UMI detrend path on GB300.

Headline workload: 1,000 TESS-like 2-min curves x 18,000 samples (W = 361,
alpha 2, c 5, 5 iterations), flux resident in HBM, one batched call per step
(the persistent work-queue kernel, replayed from the CUDA-graph cache).

Prints ONE JSON line (rank 0) with: value = window evaluations per second
(positions whose trend is produced), curves/s, the live roofline of the
kernel (ALU-issue bound), the end-to-end number through the host-buffer
entry point, the one-launch-per-curve form, and SM clocks sampled during the
timed region.  Beside the headline it measures the other workloads the same
way (``workloads``: one curve, the uneven 4,096-curve TESS/Kepler batch and
256 20-s curves at W = 2161; per-band roofline fractions and a sampled check
against the FP64 oracle), the continuous-batching server on 200,000
host-buffer requests drawn from the serving mixture (``serving``), and the
FP64 oracle on the host cores as a CPU baseline.

--impl reference runs the FP64 CPU oracle instead (a bounded sample of the
same workload per step, on the host cores) and prints the same kind of line.
Under torchrun each rank detrends its own batch (weak scaling, no collective
on the data path); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Lane-ops per valid window sample for one window evaluation: 5 iterations x
# 9 (residual, scale, two sign selects, fma, clamp, square, two sums) + 5 for
# the upper-RMS scale + 4 for one exact selection pass.
OPS_PER_SAMPLE = 54
LANES_PER_SM = 128

# DRAM bytes (read + write) of one launch of the batched kernel on the
# headline workload, from the ncu capture of that workload, valid only while
# the kernel's code (comments and blank lines removed) hashes to
# `kernel_sha256`.
MEASURED_TRAFFIC = {"bytes": 163.02e6,
                    "kernel_sha256": "006aa279044fa5dccee93fc0fde15514b0bfb5f854327c42d3daa2726affd0c7"}
KERNEL_SOURCE = os.path.join(ROOT, "paper_2604_06602_gb300", "csrc", "umi_kernel.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="umi", choices=["umi", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4"],
                    help="c2 (default): 1000 TESS-like curves x 18000; c1: one such curve; "
                         "c3: 4096 uneven TESS/Kepler curves; c4: 256 x 118000 at 20-s cadence")
    ap.add_argument("--curves", type=int, default=None)
    ap.add_argument("--n", type=int, default=18000)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the per-curve, serving, e2e and CPU-baseline legs")
    ap.add_argument("--serve-requests", type=int, default=200000,
                    help="requests of the serving stream run at each of the high offered rates")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the one-curve, uneven-batch and 20-s legs")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--tuning-file", default=None,
                    help="load kernel plans from this file instead of running the autotuner")
    ap.add_argument("--save-tuning", default=None, help="write the tuned plans to this file")
    ap.add_argument("--shard", default="own", choices=["own", "lpt"],
                    help="own (default): each rank detrends its own batch (weak scaling); "
                         "lpt: one batch split over the ranks by window work (strong scaling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def shard_seed(rank, config=1):
    """Each rank detrends its own batch: seeds differ per rank."""
    from paper_2604_06602_gb300 import synth
    return synth.BASE_SEED + config + 1000 * rank


def lpt_part(batch, W, rank, world):
    """This rank's part of one batch split over `world` ranks by window work
    (greedy longest-processing-time): (sub-batch, its W, the part's curve indices)."""
    from paper_2604_06602_gb300 import partition
    shards = partition.lpt_shards(partition.window_work(batch.lengths, W), world)
    idx = shards[rank]
    return batch.subset(idx), W[idx], idx


def tune_for_batch(umi, batch, W, flux):
    """The kernel plans the benchmark times: for each window length, tuned on
    the band's own curves (`flux`, the batch on the device; every k-th curve
    when they hold more than 2e7 positions, repeated when they hold fewer
    than 1e6: the best plan depends on the band's size, on how its curves end
    within tiles and on its data), and, where one curve alone is a
    latency-regime band, on a single synthetic curve of the median length."""
    import torch
    for w in sorted(set(W.tolist())):
        idx = np.flatnonzero(W == w)
        n_one = max(1, int(np.median(batch.lengths[idx])))
        pick = idx[::max(1, int(np.ceil(batch.lengths[idx].sum() / 20_000_000)))]
        reps = max(1, int(np.ceil(1_000_000 / batch.lengths[pick].sum())))
        parts = [flux[int(batch.offsets[i]):int(batch.offsets[i + 1])] for i in pick] * reps
        umi.autotune_batch(int(w), np.tile(batch.lengths[pick], reps), flux=torch.cat(parts))
        if umi.get_plan(int(w), n_one)["latency"]:
            umi.autotune(int(w), positions=n_one)


def make_workload(args, rank):
    """The synthetic batch of the chosen workload, and a one-line description.
    With --shard lpt every rank builds the same batch (rank 0's seed) and
    later keeps its own part of it."""
    from paper_2604_06602_gb300 import synth
    if getattr(args, "shard", "own") == "lpt":
        rank = 0
    if args.workload == "c1":
        b = synth.config1(seed=shard_seed(rank, 0))
        return b, "one TESS-like 2-min curve x 18000 samples, W=361"
    if args.workload == "c3":
        b = synth.config3(seed=shard_seed(rank, 2), n_curves=args.curves or 4096)
        return b, ("%d uneven curves: half TESS 2-min (N 5k-20k, W=361), half Kepler 29.4-min "
                   "(N 4k-70k, W=25, 3-day gaps)" % b.B)
    if args.workload == "c4":
        b = synth.config4(seed=shard_seed(rank, 3), n_curves=args.curves or 256)
        return b, "%d TESS 20-s curves x 118000 samples, W=2161, 1%% spikes" % b.B
    b = synth.config2(seed=shard_seed(rank, 1), n_curves=args.curves or 1000, n=args.n)
    return b, ("%d TESS-like 2-min curves x %d samples, W=361, alpha 2, c 5, 5 iters"
               % (b.B, args.n))


def window_work(flux, offsets, W, min_valid=None):
    """(produced positions, sum of valid samples over their windows)."""
    evals, samples = 0, 0
    for b in range(offsets.size - 1):
        x = flux[offsets[b]:offsets[b + 1]]
        w = int(W[b])
        h = (w - 1) // 2
        fin = np.isfinite(x)
        cs = np.concatenate([[0], np.cumsum(fin, dtype=np.int64)])
        n = x.size
        j = np.arange(n)
        lo = np.maximum(0, j - h)
        hi = np.minimum(n, j + h + 1)
        nv = cs[hi] - cs[lo]
        mv = w // 3 if min_valid is None or min_valid < 0 else min_valid
        prod = fin & (nv >= max(1, mv))
        evals += int(prod.sum())
        samples += int(nv[prod].sum())
    return evals, samples


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": float(max(power))}


def kernel_sha256():
    """sha256 of the kernel source's code: comments and blank lines removed,
    so that a comment edit does not invalidate a measurement."""
    import hashlib
    import re
    with open(KERNEL_SOURCE) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
    return hashlib.sha256(code.encode()).hexdigest()


def measured_traffic():
    """Traffic per launch if the kernel is unchanged since it was measured."""
    if MEASURED_TRAFFIC["bytes"] and MEASURED_TRAFFIC["kernel_sha256"] == kernel_sha256():
        return MEASURED_TRAFFIC["bytes"]
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}, "fallback"


def cpu_baseline(batch, W, budget_s=12.0):
    """FP64 oracle on the host cores over a bounded sample of the workload."""
    import oracle
    threads = os.cpu_count() or 1
    k = max(threads, 8)
    while True:
        idx = np.arange(min(k, batch.B))
        sub = batch.subset(idx)
        t0 = time.perf_counter()
        oracle.detrend_batch(sub.flux, sub.offsets, W[idx], nthreads=threads)
        dt = time.perf_counter() - t0
        if dt * threads >= budget_s or k >= batch.B:
            break
        k = min(batch.B, int(k * max(2.0, budget_s / max(dt * threads, 1e-3))))
    evals, _ = window_work(sub.flux, sub.offsets, W[idx])
    return {"value": evals / dt, "unit": "window-evals/s", "cores": threads, "kind": "oracle",
            "sample": "%d of the %d curves (FP64 C oracle, %d pthreads, %.1f s wall, %.0f core-s)"
                      % (idx.size, batch.B, threads, dt, dt * threads),
            "curves_per_s": idx.size / dt}


L2_NOTE = ("flushed between timed steps by writing a buffer of twice the L2 (at least 256 MB); "
           "the writes fall outside the per-step CUDA events")


def run_config(desc, global_curves, seq_len, world):
    """The workload description both arms print, so that their lines compare
    like for like."""
    return {"workload": desc, "global_batch": int(global_curves), "seq_len": int(seq_len),
            "parallelism": "dp%d" % world, "l2": L2_NOTE}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    batch, desc = make_workload(args, 0)
    W = np.array([oracle.window_length(c) for c in batch.cadence], np.int32)
    threads = os.cpu_count() or 1
    per_step = min(batch.B, max(threads, 16) if args.workload != "c4" else max(2, threads // 4))
    idx_all = np.arange(batch.B)
    t_steps = []
    evals = 0
    for s in range(args.warmup + args.steps):
        idx = idx_all[(s * per_step) % batch.B:][:per_step]
        sub = batch.subset(idx)
        t0 = time.perf_counter()
        oracle.detrend_batch(sub.flux, sub.offsets, W[idx], nthreads=threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            t_steps.append(dt)
            evals += window_work(sub.flux, sub.offsets, W[idx])[0]
    total = sum(t_steps)
    value = evals / total
    global_curves = batch.B if args.shard == "lpt" else batch.B * world
    line = {
        "impl": "reference", "metric": "window-evals/s", "value": value, "unit": "window-evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "strong" if args.shard == "lpt" else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": run_config(desc, global_curves, batch.lengths.max(), world),
        "cpu_baseline": {"value": value, "unit": "window-evals/s", "cores": threads, "kind": "oracle",
                         "sample": "%d curves of the workload per step (%d steps), FP64 C oracle over "
                                   "%d pthreads" % (per_step, args.steps, threads)},
        "e2e": {"value": value, "unit": "window-evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_umi(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)          # before NCCL init: one rank per GPU
    dev = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    from paper_2604_06602_gb300 import build as libbuild
    from paper_2604_06602_gb300 import synth, umi
    if rank == 0:
        libbuild.build()
    barrier(dist)
    umi.load()

    batch, desc = make_workload(args, rank)
    W = np.array([umi.window_length(c) for c in batch.cadence], np.int32)
    global_curves = batch.B * world
    seq_len = batch.lengths.max()
    if args.shard == "lpt":
        global_curves = batch.B
        batch, W, _ = lpt_part(batch, W, rank, world)
        desc += ", split over %d ranks by window work" % world
    evals, samples = window_work(batch.flux, batch.offsets, W)
    flux = torch.from_numpy(batch.flux).to(dev)
    trend = torch.empty_like(flux)
    detr = torch.empty_like(flux)
    flush = l2_flush_buffer(torch, dev)
    stream = torch.cuda.current_stream(dev)
    umi.set_graph_cache(True)
    # The library's autotuner picks the kernel plan for this window length
    # (outside the timed region, as a user would once per GPU).
    if args.tuning_file:
        umi.load_tuning(args.tuning_file)
    else:
        tune_for_batch(umi, batch, W, flux)
    tuned_plan = {int(w): umi.get_plan(int(w), int(batch.lengths[W == w].sum())) for w in sorted(set(W.tolist()))}
    if args.save_tuning and rank == 0:
        umi.save_tuning(args.save_tuning)

    for _ in range(args.warmup):
        umi.detrend_batched(flux, batch.offsets, W, trend=trend, detr=detr)
        flush.fill_(1.0)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = umi.kernel_launch_count()
    barrier(dist)
    torch.cuda.synchronize()
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for s in range(args.steps):
        flush.fill_(float(s))          # L2 flush between steps (inside the timed region)
        starts[s].record(stream)
        umi.detrend_batched(flux, batch.offsets, W, trend=trend, detr=detr)
        ends[s].record(stream)
    t_all1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    gpu_launches = umi.kernel_launch_count() - launches0
    clk = clocks.stop()
    region_ms = t_all0.elapsed_time(t_all1)       # includes the L2 flushes between steps
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    kernel_ms = float(np.mean(step_ms))
    # The K steps' own device time (the flush writes between them excluded),
    # the slowest rank's.
    elapsed_ms = max_over_ranks(dist, float(np.sum(step_ms)), dev)
    region_ms = max_over_ranks(dist, region_ms, dev)
    total_evals = sum_over_ranks(dist, evals, dev)
    value = total_evals * args.steps / (elapsed_ms / 1e3)

    peak_ops, peak_note = lane_op_peak(torch, dev)
    achieved = OPS_PER_SAMPLE * samples / (kernel_ms / 1e3) / 1e12
    traffic = measured_traffic() if args.workload == "c2" and args.curves is None else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Tlane-op/s",
                "frac": achieved / peak_ops, "traffic": traffic,
                "algorithmic_bytes": 12 * batch.flux.size,
                "note": "peak = %s; achieved = %d lane-ops x %.4g valid window samples / mean kernel "
                        "time %.3f ms" % (peak_note, OPS_PER_SAMPLE, samples, kernel_ms)}

    line = {
        "metric": "window-evals/s", "value": value, "unit": "window-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "strong" if args.shard == "lpt" else "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": run_config(desc, global_curves, seq_len, world),
        "timed_region_ms": region_ms,
        "plan": tuned_plan,
        "curves_per_s": global_curves * args.steps / (elapsed_ms / 1e3),
        "kernel_ms": kernel_ms,
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": gpu_launches,
    }

    if not args.no_extras and rank == 0:
        line["per_curve_launch"] = per_curve_leg(umi, torch, flux, batch, W, evals)
        line["e2e"] = e2e_leg(umi, torch, batch, W, evals, args)
        line["segmented"] = segmented_leg(umi, torch, flux, batch, W, evals)
        line["mad_biweight"] = mad_leg(umi, torch, flux, batch, W, evals)
        cpu = cpu_baseline(batch, W)
        del flux, trend, detr
        if args.workload == "c2" and args.curves is None and not args.no_workloads:
            line["workloads"] = {}
            for name in ("c1", "c3", "c4"):
                line["workloads"][name] = workload_leg(umi, torch, dev, flush, name, local)
                torch.cuda.empty_cache()
        if args.workload == "c2" and not args.no_serving:
            line["serving"] = serving_leg(umi, torch, dev, args)
        line["cpu_baseline"] = cpu
    elif rank == 0:
        line["e2e"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def l2_flush_buffer(torch, dev):
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    return torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device=dev)


def lane_op_peak(torch, dev):
    """(peak T lane-ops/s, how it was formed): SMs x 128 FP32/INT32 lanes x the
    measured maximum SM clock."""
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    return (sms * LANES_PER_SM * sm_max * 1e6 / 1e12,
            "%d SMs x 128 lanes x %.0f MHz (%s sm_max_mhz)" % (sms, sm_max, peak_src))


def timed_batched(umi, torch, flux, offsets, W, trend, detr, flush, steps, warmup=2):
    """Per-step kernel times [ms] of the batched call (CUDA events on the
    launching stream; the L2 is flushed before every step)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        umi.detrend_batched(flux, offsets, W, trend=trend, detr=detr)
        flush.fill_(1.0)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for s, (a, b) in enumerate(ev):
        flush.fill_(float(s))
        a.record(stream)
        umi.detrend_batched(flux, offsets, W, trend=trend, detr=detr)
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def sample_positions(x, W, rng, k=6):
    """Positions of one curve checked against the oracle: both ends, the
    first and last full windows, both sides of the first few gaps, and k
    random positions."""
    n = x.size
    h = (W - 1) // 2
    pos = [0, 1, n - 2, n - 1, h, n - 1 - h]
    miss = np.isnan(x)
    edges = np.flatnonzero(np.diff(miss.astype(np.int8)))
    for e in edges[:6]:
        pos += [e - 1, e, e + 1, e + 2]
    pos += list(rng.integers(0, n, k))
    pos = np.unique(np.array(pos, np.int64))
    return pos[(pos >= 0) & (pos < n)]


def sampled_parity(batch, W, trend, detr, seed=11, tol=1e-5):
    """The GPU outputs against the FP64 oracle evaluated one position at a
    time on sampled positions of every curve: NaN patterns must match and the
    trend and detrended flux agree within `tol` relative."""
    import oracle
    rng = np.random.default_rng(seed)
    worst_t, worst_d, count, nan_ok = 0.0, 0.0, 0, True
    for i in range(batch.B):
        x = batch.curve(i)
        pos = sample_positions(x, int(W[i]), rng)
        ref = oracle.detrend_positions(x, int(W[i]), pos)
        o = batch.offsets[i]
        for got, want, which in ((trend[o + pos], ref["trend"], "t"), (detr[o + pos], ref["detr"], "d")):
            g = got.astype(np.float64)
            nan_ok &= bool(np.array_equal(np.isnan(g), np.isnan(want)))
            ok = ~np.isnan(want)
            if ok.any():
                rel = float(np.max(np.abs(g[ok] - want[ok]) / np.abs(want[ok])))
                if which == "t":
                    worst_t = max(worst_t, rel)
                else:
                    worst_d = max(worst_d, rel)
        count += pos.size
    return {"positions": count, "curves": batch.B, "max_rel_err_trend": worst_t,
            "max_rel_err_detr": worst_d, "nan_pattern_equal": nan_ok,
            "ok": bool(nan_ok and worst_t <= tol and worst_d <= tol), "tolerance": tol,
            "reference": "FP64 C oracle, one position at a time"}


def workload_leg(umi, torch, dev, flush, name, local):
    """One more workload measured like the headline: batched kernel time,
    window-evals/s, curves/s, the one-launch-per-curve form, the roofline
    fraction of each window band (a band timed as its own batch plans and
    runs exactly as inside the mixed batch) and a sampled oracle check."""
    from types import SimpleNamespace
    batch, desc = make_workload(SimpleNamespace(workload=name, curves=None, n=18000, shard="own"), 0)
    W = np.array([umi.window_length(c) for c in batch.cadence], np.int32)
    steps = {"c1": 20, "c3": 5, "c4": 3}[name]
    evals, samples = window_work(batch.flux, batch.offsets, W)
    flux = torch.from_numpy(batch.flux).to(dev)
    tune_for_batch(umi, batch, W, flux)
    trend = torch.empty_like(flux)
    detr = torch.empty_like(flux)
    peak_ops, peak_note = lane_op_peak(torch, dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms = timed_batched(umi, torch, flux, batch.offsets, W, trend, detr, flush, steps)
    bands = []
    for w in sorted(set(W.tolist())):
        idx = np.flatnonzero(W == w)
        if idx.size == batch.B:
            sub, bms = batch, ms
        else:
            sub = batch.subset(idx)
            sf = torch.from_numpy(sub.flux).to(dev)
            bms = timed_batched(umi, torch, sf, sub.offsets, W[idx], torch.empty_like(sf),
                                torch.empty_like(sf), flush, steps)
            del sf
        _, bs = window_work(sub.flux, sub.offsets, W[idx])
        bk = float(np.mean(bms))
        plan = umi.get_plan(int(w), int(sub.lengths.sum()))
        bands.append({"W": int(w), "curves": int(idx.size), "positions": int(sub.lengths.sum()),
                      "valid_window_samples": int(bs), "kernel_ms": bk, "plan": plan,
                      "regime": "latency" if plan["latency"] else "throughput",
                      "roofline_frac": OPS_PER_SAMPLE * bs / (bk / 1e3) / 1e12 / peak_ops})
    clk = clocks.stop()
    per_curve = per_curve_leg(umi, torch, flux, batch, W, evals)
    torch.cuda.synchronize()
    kms = float(np.mean(ms))
    parity = sampled_parity(batch, W, trend.cpu().numpy(), detr.cpu().numpy())
    return {"workload": desc, "curves": batch.B, "samples": int(batch.flux.size), "steps": steps,
            "kernel_ms": kms, "kernel_ms_min": float(np.min(ms)),
            "window_evals_per_s": evals / (kms / 1e3), "curves_per_s": batch.B / (kms / 1e3),
            "valid_window_samples": int(samples),
            "roofline_frac": OPS_PER_SAMPLE * samples / (kms / 1e3) / 1e12 / peak_ops,
            "roofline_note": "ALU-issue bound; peak = %s" % peak_note,
            "bands": bands, "per_curve_launch": per_curve, "parity": parity, "clocks": clk,
            "l2": L2_NOTE}


def per_curve_leg(umi, torch, flux, batch, W, evals):
    """The plain form: one umi_detrend launch per curve on one stream."""
    trend = torch.empty_like(flux)
    detr = torch.empty_like(flux)
    views = [(flux[batch.offsets[b]:batch.offsets[b + 1]], trend[batch.offsets[b]:batch.offsets[b + 1]],
              detr[batch.offsets[b]:batch.offsets[b + 1]]) for b in range(batch.B)]
    for b, (x, t, d) in enumerate(views[:8]):
        umi.detrend(x, int(W[b]), trend=t, detr=d)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for b, (x, t, d) in enumerate(views):
        umi.detrend(x, int(W[b]), trend=t, detr=d)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": evals / (ms / 1e3), "unit": "window-evals/s", "curves_per_s": batch.B / (ms / 1e3),
            "ms": ms, "launches": batch.B}


def mad_leg(umi, torch, flux, batch, W, evals):
    """The paper's comparison estimator on the same batch: symmetric
    biweight (alpha 1) with the MAD scale, which needs a second exact
    selection per window."""
    p = umi.params(alpha=1.0, scale_mode=umi.SCALE_MAD)
    trend = torch.empty_like(flux)
    detr = torch.empty_like(flux)
    for _ in range(2):
        umi.detrend_batched(flux, batch.offsets, W, p, trend=trend, detr=detr)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 5
    e0.record()
    for _ in range(steps):
        umi.detrend_batched(flux, batch.offsets, W, p, trend=trend, detr=detr)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": evals / (ms / 1e3), "unit": "window-evals/s", "kernel_ms": ms,
            "params": "alpha 1, c 5, MAD scale"}


def segmented_leg(umi, torch, flux, batch, W, evals):
    """The same batch through umi_detrend_segmented (gap handling with the
    default split rules): bit-pack kernel, host segment scan, one batched
    launch per call."""
    trend = torch.empty_like(flux)
    detr = torch.empty_like(flux)
    for _ in range(2):
        _, _, kept = umi.detrend_segmented(flux, batch.offsets, W, trend=trend, detr=detr)
    torch.cuda.synchronize()
    steps = 5
    t0 = time.perf_counter()
    for _ in range(steps):
        umi.detrend_segmented(flux, batch.offsets, W, trend=trend, detr=detr)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    return {"value": evals / dt, "unit": "window-evals/s", "ms_per_call": dt * 1e3,
            "segments": kept, "curves_per_s": batch.B / dt}


def e2e_leg(umi, torch, batch, W, evals, args):
    """Same metric through the host-buffer entry point (copies inside)."""
    fh = torch.from_numpy(batch.flux).pin_memory()
    th = torch.empty(batch.flux.size, dtype=torch.float32).pin_memory()
    dh = torch.empty(batch.flux.size, dtype=torch.float32).pin_memory()
    for _ in range(2):
        umi.detrend_batched_host(fh, batch.offsets, W, trend=th, detr=dh)
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(steps):
        umi.detrend_batched_host(fh, batch.offsets, W, trend=th, detr=dh)
    dt = time.perf_counter() - t0
    nbytes = batch.flux.size * 4
    return {"value": evals * steps / dt, "unit": "window-evals/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": 2 * nbytes, "steps": steps,
            "curves_per_s": batch.B * steps / dt}


SERVE_BUDGET = 40 << 30
SERVE_STEADY_AFTER_S = 1.0


def serve_at_rate(srv, stream, W_req, rate, n):
    """Submits requests 0..n-1 of the stream from host buffers on its Poisson
    schedule at `rate`, polling for completions in between.  Returns per
    request its arrival time [s], latency [s] (submit to completion, the
    server's clock) and (admit, launch, done) timeline, the wall time and the
    submission rate actually achieved."""
    arrivals = stream.arrivals[:n] / rate
    lat = np.empty(n)
    phases = np.empty((n, 3))
    pending = []
    t0 = time.perf_counter()

    def finish(i, tt):
        tl = srv.timeline(tt)
        lat[i] = tl["done"]
        phases[i] = (tl["admit"], tl["launch"], tl["done"])
        srv.release(tt)

    for i in range(n):
        due = t0 + arrivals[i]
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            if due - now > 2e-4:
                time.sleep(min(1e-3, due - now - 1e-4))
        pending.append((i, srv.submit(stream.flux(i), int(W_req[i]))))
        while pending:
            if srv.poll(pending[0][1]) is None:
                break
            finish(*pending.pop(0))
    t_sub = time.perf_counter() - t0
    for i, tt in pending:
        srv.wait(tt, 300)
        finish(i, tt)
    return arrivals, lat, phases, time.perf_counter() - t0, n / t_sub


def serialized_at_rate(umi, torch, stream, tapes_pinned, W_req, rate, n, dev):
    """The same request stream served the plain way: per request one copy of
    its flux from pinned host memory and one umi_detrend launch, all on one
    stream in arrival order.  Latency runs from the launch call to the
    completion of an event recorded after the kernel."""
    s = torch.cuda.Stream()
    nmax = int(stream.n.max())
    dflux = torch.empty(nmax, device=dev)
    dtrend = torch.empty(nmax, device=dev)
    ddetr = torch.empty(nmax, device=dev)
    arrivals = stream.arrivals[:n] / rate
    lat = np.empty(n)
    pend = []
    t0 = time.perf_counter()
    t_sub = t0
    i = 0
    while i < n or pend:
        now = time.perf_counter()
        if i < n and now >= t0 + arrivals[i]:
            k, a, m = int(stream.kind[i]), int(stream.start[i]), int(stream.n[i])
            t_sub = time.perf_counter()
            with torch.cuda.stream(s):
                dflux[:m].copy_(tapes_pinned[k][a:a + m], non_blocking=True)
            umi.detrend(dflux[:m], int(W_req[i]), trend=dtrend[:m], detr=ddetr[:m], stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
            pend.append((i, ev, t_sub))
            i += 1
            continue
        if pend and pend[0][1].query():
            j, _, ts = pend.pop(0)
            lat[j] = time.perf_counter() - ts
            if i == n and not pend:
                break
    return arrivals, lat, time.perf_counter() - t0, n / max(t_sub - t0, 1e-9)


def latency_summary(arrivals, lat, wall, offered, rate, n):
    steady = arrivals >= SERVE_STEADY_AFTER_S
    if steady.sum() < 100:
        steady = np.ones_like(steady)
    return {"rate_hz": rate, "requests": n, "offered_hz": offered, "curves_per_s": n / wall,
            "p50_ms": float(np.percentile(lat[steady], 50) * 1e3),
            "p99_ms": float(np.percentile(lat[steady], 99) * 1e3),
            "steady_requests": int(steady.sum()),
            "p50_ms_all": float(np.percentile(lat, 50) * 1e3),
            "p99_ms_all": float(np.percentile(lat, 99) * 1e3)}


def serving_leg(umi, torch, dev, args):
    """Poisson arrivals into the continuous-batching server: host-buffer
    requests (the copy to the device is inside each latency) whose sizes and
    window lengths are drawn from the serving mixture, every request its own
    slice of a light-curve tape of its class.  The full stream runs at 20k/s
    and at 50k/s (past saturation), shorter ones at 1k/s and 5k/s; the same
    stream is also served by serialized per-curve copies and launches.
    Latency percentiles are taken over requests arriving after the first
    second (steady state)."""
    from paper_2604_06602_gb300 import synth
    R = args.serve_requests
    st = synth.serving_stream(n_requests=R)
    tapes_pinned = [torch.from_numpy(t).pin_memory() for t in st.tapes]
    st.tapes = [t.numpy() for t in tapes_pinned]          # requests are slices of pinned memory
    Wk = [umi.window_length(c) for c in st.cadences]
    W_req = np.array(Wk, np.int32)[st.kind]
    for k, w in enumerate(Wk):
        # Both regimes: large batches, tuned on the class's own first requests
        # (up to 450 of them, about a saturated batch, and 2e7 positions), and
        # a median request of this window length.
        idx = np.flatnonzero(st.kind == k)[:450]
        idx = idx[np.cumsum(st.n[idx]) <= 20_000_000]
        flux_k = torch.cat([torch.from_numpy(st.flux(int(i))) for i in idx]).to(dev)
        umi.autotune_batch(w, st.n[idx], flux=flux_k)
        del flux_k
        n_one = int(np.median(st.n[st.kind == k]))
        if umi.get_plan(w, n_one)["latency"]:
            umi.autotune(w, positions=n_one)
    torch.cuda.synchronize()
    out = {"mixture": "45%% TESS 2-min N 5k-20k W=%d, 45%% Kepler 29.4-min N 4k-70k W=%d (3-day gaps), "
                      "10%% TESS 20-s N 60k-118k W=%d (1%% spikes)" % tuple(Wk),
           "requests": R, "host_inputs": True,
           "inputs": "every request its own size and its own slice of a pinned host tape of its "
                     "class (%s samples per tape)" % [int(t.size) for t in st.tapes],
           "mean_samples": float(st.n.mean()), "budget_bytes": SERVE_BUDGET,
           "steady_state": "requests arriving after the first %.0f s" % SERVE_STEADY_AFTER_S,
           "rates": []}
    peak = 0
    for rate, n in ((1000.0, min(R, 3000)), (2000.0, min(R, 6000)), (5000.0, min(R, 10000)),
                    (10000.0, min(R, 50000)), (20000.0, R), (50000.0, R)):
        with umi.Server(mem_budget_bytes=SERVE_BUDGET, n_streams=4, max_batch_curves=512) as srv:
            t = srv.submit(st.flux(0), int(W_req[0]))
            srv.wait(t, 60)
            srv.release(t)
            arr, lat, ph, wall, offered = serve_at_rate(srv, st, W_req, rate, n)
            stats = srv.stats()
        r = latency_summary(arr, lat, wall, offered, rate, n)
        r["p50_phases_ms"] = {"queued": float(np.median(ph[:, 0]) * 1e3),
                              "batching": float(np.median(ph[:, 1] - ph[:, 0]) * 1e3),
                              "gpu": float(np.median(ph[:, 2] - ph[:, 1]) * 1e3)}
        r["peak_resident_bytes"] = int(stats["peak_resident_bytes"])
        r["mean_batch_curves"] = stats["mean_batch_curves"]
        r["batches"] = int(stats["batches_launched"])
        peak = max(peak, r["peak_resident_bytes"])
        out["rates"].append(r)
    out["policy"] = ("one window length per batch, windows >= 1025 on low-priority streams "
                     "(the defaults: batch_by_window = 1, priority_window = 1025), 4 streams, "
                     "batches of at most 512 curves")
    out["peak_resident_bytes"] = peak
    out["serialized_rates"] = []
    for rate, n in ((1000.0, min(R, 3000)), (10000.0, min(R, 50000)), (20000.0, R)):
        arr, lat, wall, offered = serialized_at_rate(umi, torch, st, tapes_pinned, W_req, rate, n, dev)
        out["serialized_rates"].append(latency_summary(arr, lat, wall, offered, rate, n))
    hi = [r for r in out["rates"] if r["rate_hz"] == 20000.0][0]
    out["p50_ms"], out["p99_ms"] = hi["p50_ms"], hi["p99_ms"]
    out["curves_per_s_at_20k"] = hi["curves_per_s"]
    out["saturation_curves_per_s"] = max(r["curves_per_s"] for r in out["rates"])
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_umi(args)


if __name__ == "__main__":
    sys.exit(main())
