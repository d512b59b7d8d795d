"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
gets its own shard of curves, no data-path collective, and the step time is
the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    r, w, _ = bench.dist_env()
    d = bench.init_dist(w, "gloo")
    local_time = 10.0 + 5.0 * r
    mx = bench.max_over_ranks(d, local_time)
    bench.barrier(d)
    out[r] = (mx, bench.shard_seed(r))
    d.destroy_process_group()


def test_two_rank_max_timing_and_shards():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] != out[1][1]


def test_window_work_counts():
    x = np.ones(10, np.float32)
    x[4] = np.nan
    ev, sm = bench.window_work(x, np.array([0, 10]), np.array([3], np.int32), min_valid=0)
    # positions 0..9 minus the NaN centre; valid samples per window
    # 2,3,3,2,(skip),2,3,3,3,2
    assert ev == 9
    assert sm == 2 + 3 + 3 + 2 + 2 + 3 + 3 + 3 + 2


def _lpt_worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    from types import SimpleNamespace

    from paper_2604_06602_gb300 import partition
    r, w, _ = bench.dist_env()
    d = bench.init_dist(w, "gloo")
    args = SimpleNamespace(workload="c3", curves=40, n=18000, shard="lpt")
    batch, _ = bench.make_workload(args, r)          # the same batch on every rank
    W = np.where(batch.cadence < 0.01, 361, 25).astype(np.int32)
    sub, Wr, idx = bench.lpt_part(batch, W, r, w)
    load = int(partition.window_work(sub.lengths, Wr).sum())
    gathered = [None] * w
    dist.all_gather_object(gathered, (idx.tolist(), load, float(batch.flux[:100].sum())))
    total = bench.sum_over_ranks(d, load)
    out[r] = (gathered, total, int(partition.window_work(batch.lengths, W).sum()),
              int(partition.window_work(batch.lengths, W).max()))
    d.destroy_process_group()


def test_two_rank_lpt_split_of_one_batch():
    """--shard lpt: every rank builds the same batch and keeps a disjoint part;
    the parts cover the batch and their window work is balanced."""
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_lpt_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    gathered, total, whole, biggest = out[0]
    assert out[1][0] == gathered
    (i0, l0, f0), (i1, l1, f1) = gathered
    assert f0 == f1                                   # same batch on both ranks
    assert sorted(i0 + i1) == list(range(40)) and not set(i0) & set(i1)
    assert total == l0 + l1 == whole
    assert max(l0, l1) <= whole / 2 + biggest
