"""Splitting a detrend batch over several GPUs (host logic only).

Every output position of the method depends on its own window and nothing
else (Section 2), so a batch splits over GPUs with no exchange step:

* ``lpt_shards`` assigns whole curves to ranks by greedy longest-processing-
  time on each curve's window work (the number of window samples the
  iterations visit), which keeps the slowest rank within 4/3 of the best
  possible split;
* ``split_curve`` cuts one long curve into position ranges.  A part reads its
  range plus (W-1)/2 samples of halo on each side (clipped to the curve) and
  detrends that slice as a curve of its own; the outputs of its range are
  exact, because every window of the range lies inside the slice, and the
  slice's edges coincide with the curve's edges wherever a window of the
  range is truncated by them.
"""
from __future__ import annotations

import heapq

import numpy as np


def window_work(n, W):
    """Window samples visited over a curve of n samples (no missing values):
    sum over positions of the truncated window's length,
    n*W - 2 * (h + (h-1) + ... + (h - min(h, n) + 1)) with h = (W-1)/2."""
    n = np.asarray(n, np.int64)
    W = np.asarray(W, np.int64)
    h = (W - 1) // 2
    k = np.minimum(h, n)
    tri = lambda x: x * (x + 1) // 2  # noqa: E731
    return n * W - 2 * (tri(h) - tri(h - k))


def lpt_shards(costs, world):
    """Curve indices per rank: the largest remaining cost goes to the least
    loaded rank (ties to the lower rank).  Each rank's list is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, np.int64)
    order = sorted(range(costs.size), key=lambda i: (-int(costs[i]), i))
    heap = [(0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + int(costs[i]), r))
    return [np.array(sorted(s), np.int64) for s in shards]


def split_curve(n, W, parts):
    """(a, b, lo, hi) per part: the part produces positions [a, b) by
    detrending samples [lo, hi) as a curve and keeping outputs a-lo .. b-lo."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    if W < 1 or W % 2 == 0:
        raise ValueError("W must be odd and >= 1")
    h = (W - 1) // 2
    cuts = [n * k // parts for k in range(parts + 1)]
    out = []
    for k in range(parts):
        a, b = cuts[k], cuts[k + 1]
        out.append((a, b, max(0, a - h), min(n, b + h)))
    return out


def take_curves(flux, offsets, idx):
    """The CSR sub-batch of curves `idx`: (flux, offsets)."""
    offsets = np.asarray(offsets, np.int64)
    idx = np.asarray(idx, np.int64)
    lens = offsets[idx + 1] - offsets[idx]
    sub_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    if idx.size == 0:
        return flux[:0], sub_off
    sub = np.concatenate([flux[offsets[i]:offsets[i + 1]] for i in idx])
    return sub, sub_off
