"""Host-side logic of the multi-GPU benchmark path (one independent
trajectory per rank, no data-path collective), exercised with two gloo
ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.workload_of("water64", rank)
    my_ms = 100.0 + 50.0 * rank
    mx = bench.max_over_ranks(my_ms, dist, "cpu")
    seeds = [r.seed for r in w.replicas]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (mx, gathered, w.bead_atoms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_distinct_seeds():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    mx0, seeds0, ba = out[0]
    mx1, seeds1, _ = out[1]
    assert mx0 == mx1 == 150.0
    assert seeds0[0] != seeds0[1]          # each rank runs its own trajectory
    assert seeds0 == seeds1
    import bench
    v = bench.job_throughput(ba, world, 10, mx0)
    assert v == pytest.approx(world * ba * 10 / 0.150)


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.workload_of("fad", 0).replicas[0].seed == bench.workload_of("fad", 0).replicas[0].seed
    assert bench.workload_of("fad", 1).replicas[0].seed != bench.workload_of("fad", 0).replicas[0].seed
