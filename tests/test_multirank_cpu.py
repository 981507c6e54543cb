"""The benchmark's multi-rank path on CPU: two gloo ranks, each with its own
instance (replicas, no data-path collective); the job time is the max over
ranks and the job throughput counts every rank's lattice updates."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_setup()
    assert (w, r, lr) == (world, rank, rank)
    t_local = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    t = bench.all_max(t_local, world, "cpu")
    bench.barrier(world)
    pb = bench.workload("chemotaxis_plume_512x256", rank)
    value = bench.job_mlups(pb.nodes, 100, 4, world, t)
    out[rank] = (t, value, float(pb.phi0[0].sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (t0, v0, s0), (t1, v1, s1) = out[0], out[1]
    assert t0 == t1 == 15.0                          # max over ranks
    nodes = 512 * 256
    assert v0 == v1 == pytest.approx(world * nodes * 100 * 4 / 15e-3 / 1e6)
    assert s0 != s1                                  # each rank draws its own instance (seed = rank)


def test_reference_arm_takes_the_first_instance_of_a_sweep():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    wl = bench.workload("batched_plume_sweep_64", 0)
    assert isinstance(wl, list) and len(wl) == 64
