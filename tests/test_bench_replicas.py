"""The multi-GPU path of the bench is replicas only (every rank solves its own seeded problem of
the workload's shape; no collective on the data path).  Its host logic — the replica seeds, the
slowest rank's time taken by an all-reduce MAX, and the whole-job rate — runs here as two gloo
ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from workloads import load_config, make_particles  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(times[rank], dist, "cpu")
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_time_and_whole_job_rate():
    world = 2
    times = [1.25, 2.5]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), times, out), nprocs=world, start_method="spawn")
    assert out[0] == out[1] == max(times)
    n, steps = 513, 100
    rate = bench.whole_job_rate(n ** 3, steps, world, out[0])
    assert rate == pytest.approx(n ** 3 * steps * world / 2.5)
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0


def test_replicas_are_independent_problems_of_the_same_shape():
    cfg = load_config("c1_box64_n129")
    base = make_particles(cfg, seed=bench.replica_seed(0, int(cfg["index"])))
    assert np.array_equal(base.xyz, make_particles(cfg).xyz)          # rank 0: the workload itself
    others = [make_particles(cfg, seed=bench.replica_seed(r, int(cfg["index"]))) for r in (1, 2)]
    for o in others:
        assert o.xyz.shape == base.xyz.shape and not np.array_equal(o.xyz, base.xyz)
    assert not np.array_equal(others[0].xyz, others[1].xyz)
