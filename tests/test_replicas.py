"""The N-GPU path of the benchmark: independent replicas, one per rank, each
on its own problem instance (its own random streams), combined by the
slowest rank's time and the sum of the segments.  Exercised here with two
gloo ranks on CPU; the arithmetic of the method is not involved."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, seg = bench.combine_replicas(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world, "cpu")
        p, _ = bench.workload(rank, n_particles=1000)
        out[rank] = (ms, seg, p.instance, p.seed)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_combine_max_time_and_sum_of_segments():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, seg, inst, seed = out[r]
        assert ms == 15.0 and seg == 3000.0
        assert inst == r
    # same seed, different instance: the replicas draw different random streams
    assert out[0][3] == out[1][3]


def test_replica_instances_draw_different_streams():
    import oracle as O
    import bench
    p0, _ = bench.workload(0, n_particles=10)
    p1, _ = bench.workload(1, n_particles=10)
    u0 = O.draw(O.OracleProblem(p0), 12345, 7, 0)
    u1 = O.draw(O.OracleProblem(p1), 12345, 7, 0)
    assert u0 != u1 and 0.0 < u0 < 1.0 and 0.0 < u1 < 1.0


def test_single_rank_is_the_identity():
    import bench
    assert bench.combine_replicas(3.5, 42.0, 1, "cpu") == (3.5, 42.0)
