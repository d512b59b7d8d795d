"""Host logic for splitting a batch over GPUs (partition.py): window work
against brute force, the longest-processing-time assignment, and the halo
split of one long curve, which the oracle reproduces bit for bit (every
position depends on its own window only, Section 2)."""
import numpy as np
import pytest

import oracle
from paper_2604_06602_gb300 import partition, synth


def brute_work(n, W):
    h = (W - 1) // 2
    return sum(min(p + h, n - 1) - max(p - h, 0) + 1 for p in range(n))


@pytest.mark.parametrize("n", [0, 1, 2, 5, 17, 60, 61, 62, 200])
@pytest.mark.parametrize("W", [1, 3, 25, 61, 121])
def test_window_work_closed_form(n, W):
    assert int(partition.window_work(n, W)) == brute_work(n, W)


def test_window_work_vectorised():
    n = np.array([0, 10, 1000, 7])
    W = np.array([3, 3, 361, 25])
    assert partition.window_work(n, W).tolist() == [brute_work(a, b) for a, b in zip(n, W)]


def test_lpt_known_case():
    # 7 -> r0, 6 -> r1, 5 -> r1 (11), 4 -> r0 (11), 3 -> r0 (tie, lower rank): loads 14 / 11.
    shards = partition.lpt_shards([7, 6, 5, 4, 3], 2)
    assert [s.tolist() for s in shards] == [[0, 3, 4], [1, 2]]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_lpt_covers_and_balances(world):
    rng = np.random.default_rng(world)
    costs = rng.integers(1, 10**6, size=500)
    shards = partition.lpt_shards(costs, world)
    allidx = np.concatenate(shards)
    assert np.array_equal(np.sort(allidx), np.arange(costs.size))
    loads = np.array([costs[s].sum() for s in shards])
    # Any list schedule ends within the mean load plus the largest job.
    assert loads.max() <= costs.sum() / world + costs.max()


def test_lpt_more_ranks_than_curves():
    shards = partition.lpt_shards([5, 1], 4)
    assert sorted(len(s) for s in shards) == [0, 0, 1, 1]


@pytest.mark.parametrize("n,W,parts", [(3000, 61, 4), (100, 61, 5), (500, 25, 1), (37, 361, 3)])
def test_split_curve_is_exact_under_the_oracle(n, W, parts):
    x = synth.random_curve(300 + n + W, n, nan_runs=2, run_len=(1, 40))
    full = oracle.detrend(x, W)
    ranges = partition.split_curve(n, W, parts)
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(ranges[k][1] == ranges[k + 1][0] for k in range(parts - 1))
    for a, b, lo, hi in ranges:
        part = oracle.detrend(x[lo:hi], W)
        for key in ("trend", "detr"):
            np.testing.assert_array_equal(part[key][a - lo:b - lo], full[key][a:b])


def test_take_curves():
    flux = np.arange(10, dtype=np.float32)
    off = np.array([0, 3, 3, 7, 10])
    sub, so = partition.take_curves(flux, off, [3, 0])
    assert so.tolist() == [0, 3, 6] and sub.tolist() == [7, 8, 9, 0, 1, 2]
