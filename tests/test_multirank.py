"""The multi-GPU path of bench.py (replicas: each rank evaluates its own walkers, no
collective on the data path) exercised on CPU with two gloo ranks: distinct walker
shards per rank, and the job value taken over the slowest rank."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "BENCH_BACKEND": "gloo"})
    import bench
    import workloads as W

    w, r, local = bench.dist_init()
    th = W.draw_walkers(16, bench.walker_seed(False, r), (5.0, 7.0))
    ms_local = 100.0 + 50.0 * r           # rank 1 is the slower one
    ms = bench.max_over_ranks(w, ms_local)
    value = bench.job_value(w, 16, 4, ms)
    bench.barrier(w)
    np.save(os.path.join(out, "rank%d.npy" % r), np.concatenate([th.ravel(), [ms, value]]))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_ranks_shard_walkers_and_time_the_slowest(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    th0, th1 = r0[:-2].reshape(16, 11), r1[:-2].reshape(16, 11)
    assert not np.allclose(th0, th1)             # each rank has its own walkers
    assert r0[-2] == r1[-2] == 150.0              # max over ranks
    assert r0[-1] == r1[-1] == pytest.approx(2 * 16 * 4 / 0.150)
