"""The slab decomposition's host logic on CPU ranks (gloo): the row partition,
the halo exchange schedule between neighbouring ranks and the FP64 all-reduce of
paper_2101_03055_gb300.slab.

Each rank holds one slab of a lattice of 9 + 5m population planes and advances
it by the streaming part of the update (every node pulls population i from
x - c_i; half-way bounce-back at walls), exchanging its halo rows with
HaloExchange after every step.  Gathered, the slabs must equal the whole
lattice streamed alone, bit for bit: a wrong neighbour, direction, plane set or
row anywhere in the exchange changes values that the streaming carries into
the slabs.  (The GPU form of the same split, with the full collision, is checked
against the whole lattice in tests/test_split_gpu.py.)"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C9 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
OPP9 = [0, 3, 4, 1, 2, 7, 8, 5, 6]
C5 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1)]
OPP5 = [0, 3, 4, 1, 2]


def lattice_velocities(m):
    vel = [(cx, cy, OPP9[i]) for i, (cx, cy) in enumerate(C9)]
    for a in range(m):
        vel += [(cx, cy, 9 + 5 * a + OPP5[i]) for i, (cx, cy) in enumerate(C5)]
    return vel


def stream(F, lo, hi, periodic_y, vel):
    """Pull streaming of rows lo..hi-1 of F [planes][rows][nx] (x periodic); rows
    outside lo..hi keep their values.  A source row outside F is a wall (bounce-back
    from the node's opposite plane), or wraps when periodic_y."""
    ny = F.shape[1]
    G = F.copy()
    for k, (cx, cy, opp) in enumerate(vel):
        for y in range(lo, hi):
            sy = y - cy
            if periodic_y:
                sy %= ny
            if 0 <= sy < ny:
                G[k, y] = np.roll(F[k, sy], cx)
            else:
                G[k, y] = F[opp, y]
    return G


def whole_lattice(nx, ny, m, seed):
    # FP32 values, so the FP32 exchange buffers carry them exactly
    return np.random.default_rng(seed).normal(size=(9 + 5 * m, ny, nx)).astype(np.float32).astype(np.float64)


def _worker(rank, world, port, periodic, m, nx, ny, steps, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2101_03055_gb300 import slab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = slab.plan(ny, world, periodic)[rank]
    F = slab.local_rows(whole_lattice(nx, ny, m, 7), p, ny)
    lo, hi = p.halo & 1, (p.halo & 1) + p.rows
    up_planes, down_planes = slab.crossing_planes(m, True), slab.crossing_planes(m, False)

    def pack(side, buf):
        row, planes = (lo, down_planes) if side == 0 else (hi - 1, up_planes)
        buf.copy_(torch.from_numpy(F[planes, row].astype(np.float32).ravel()))

    def unpack(side, buf):
        row, planes = (0, up_planes) if side == 0 else (p.lny - 1, down_planes)
        F[planes, row] = buf.numpy().reshape(len(planes), nx)

    ex = slab.HaloExchange(rank, world, periodic, (3 + m) * nx, "cpu")
    vel = lattice_velocities(m)
    for _ in range(steps):
        # a slab's y axis is never periodic: its halo rows stand in for the neighbours
        F = stream(F, lo, hi, periodic_y=False, vel=vel)
        ex.exchange(pack, unpack)
    sums = slab.allreduce_sums(F[:, lo:hi].sum(axis=(1, 2)), "cpu")
    out[rank] = (p.y0, F[:, lo:hi].copy(), sums)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,periodic,m", [(2, False, 2), (2, True, 1), (3, True, 2), (3, False, 3)])
def test_slabs_over_gloo_equal_the_whole_lattice(world, periodic, m):
    nx, ny, steps = 12, 11, 9
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), periodic, m, nx, ny, steps, out), nprocs=world, join=True)
    W = whole_lattice(nx, ny, m, 7)
    vel = lattice_velocities(m)
    for _ in range(steps):
        W = stream(W, 0, ny, periodic, vel)
    got = np.empty_like(W)
    for r in range(world):
        y0, rows, _ = out[r]
        got[:, y0:y0 + rows.shape[1]] = rows
    np.testing.assert_array_equal(got, W)
    moved = sum(out[r][1].size for r in range(world))
    assert moved == W.size
    np.testing.assert_allclose(out[0][2], got.sum(axis=(1, 2)), rtol=1e-12)
    assert all(np.array_equal(out[0][2], out[r][2]) for r in range(world))


def test_plan_partitions_rows():
    from paper_2101_03055_gb300 import slab
    for ny, n, per in [(11, 2, False), (11, 3, True), (64, 4, True), (5, 5, False)]:
        ps = slab.plan(ny, n, per)
        assert sum(p.rows for p in ps) == ny and ps[0].y0 == 0
        assert all(ps[k + 1].y0 == ps[k].y0 + ps[k].rows for k in range(n - 1))
        assert max(p.rows for p in ps) - min(p.rows for p in ps) <= 1
        if not per:
            assert ps[0].halo & 1 == 0 and ps[-1].halo & 2 == 0
    with pytest.raises(ValueError):
        slab.plan(5, 3, True)  # a periodic slab needs two rows per slab
