"""The multi-GPU path of bench.py (independent replicas, no data-path collective),
run as two gloo ranks on the CPU: the timing barrier, the max over ranks, the
whole-job throughput and the per-rank noise streams."""
import os
import socket

import numpy as np
import pytest

import inputs
from oracle import noise as onoise


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_setup(None, backend="gloo")
    assert (r, w) == (rank, ws)
    bench.barrier(w)
    # rank r "took" 1 + r seconds: the job time is the slowest rank's
    t = bench.max_over_ranks(1.0 + r, w, device="cpu")
    wl = inputs.workload("tiny-8x8")
    seed = bench.replica_seed(wl, r)
    x = onoise.z2_noise(seed, 1, 0, 4, 32)
    out[rank] = (t, seed, x.tolist())
    dist.destroy_process_group()


def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True, start_method="spawn")
    times = [out[r][0] for r in range(ws)]
    assert times == [2.0, 2.0]                               # max over ranks, seen by every rank
    seeds = [out[r][1] for r in range(ws)]
    assert len(set(seeds)) == ws                             # independent noise per replica
    x0, x1 = (np.array(out[r][2]) for r in range(ws))
    assert not np.array_equal(x0, x1)
    import bench
    # whole-job throughput: both ranks' samples over the slowest rank's time
    assert bench.job_throughput(3 * 256, ws, times[0]) == pytest.approx(2 * 3 * 256 / 2.0)
