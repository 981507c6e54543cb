"""A lattice split into slabs of rows along y, one slab per process.

The update of a node reads only the previous step's post-collision populations
of its nearest neighbours (Eqs. evolution12 and evolution3 with streaming,
Sec. 2 of the paper), so each process can advance its own slab of the lattice
once, before every step, its halo rows hold the populations that cross the cut
from the neighbouring slabs: per node of a cut, the three D2Q9 and the m D2Q5
populations whose velocity points across it ((3 + m) x nx values per cut and
direction).  The stop test's FP64 sums are added over the slabs with one
all-reduce.

`plan` is the row partition (the same as cdf_split's); `HaloExchange` is the
exchange schedule between neighbouring ranks of a torch.distributed group (CPU
tensors over gloo or CUDA tensors over NCCL); `SlabSolver` is one rank's slab on
its GPU, built on the C ABI's slab calls (cdf_options.halo_rows,
cdf_lb_halo_pack/unpack, cdf_lb_snapshot/cdf_lb_change_sums).
"""
from __future__ import annotations

from typing import List, NamedTuple, Optional

import numpy as np

from . import lib
from .inputs import Problem


class SlabPlan(NamedTuple):
    y0: int      # first row of the whole lattice the slab updates
    rows: int    # rows it updates
    halo: int    # bit 0: halo row below (local row 0); bit 1: halo row above (local row lny - 1)
    origin: int  # row of the whole lattice that local row 0 is (-1: wrapped)
    lny: int     # local rows, halo rows included


def plan(ny: int, nslabs: int, periodic: bool) -> List[SlabPlan]:
    """Nearly equal row counts (the first ny % nslabs slabs one row more); a walled
    axis has no halo row below the first slab or above the last."""
    if nslabs < 1 or nslabs > ny or (periodic and nslabs > 1 and ny < 2 * nslabs):
        raise ValueError("need 1 <= nslabs <= ny (ny >= 2 nslabs on a periodic axis)")
    out, y = [], 0
    for k in range(nslabs):
        r = ny // nslabs + (1 if k < ny % nslabs else 0)
        if nslabs == 1:
            hl = 0
        else:
            hl = 3 if periodic else ((1 if k > 0 else 0) | (2 if k < nslabs - 1 else 0))
        out.append(SlabPlan(y, r, hl, y - (hl & 1), r + (hl & 1) + (hl >> 1)))
        y += r
    return out


def crossing_planes(m: int, up: bool) -> List[int]:
    """Population planes (h_0..h_8, then f_{a,0..4}) whose velocity crosses a cut
    upwards (c_y = +1) or downwards (c_y = -1), in the order of a packed row."""
    return ([2, 5, 6] + [9 + 5 * a + 2 for a in range(m)]) if up else ([4, 7, 8] + [9 + 5 * a + 4 for a in range(m)])


def local_rows(field: np.ndarray, p: SlabPlan, ny: int) -> np.ndarray:
    """The slab's rows (halo rows included, wrapped on a periodic axis) of a field
    [..., ny, nx] of the whole lattice."""
    idx = (np.arange(p.lny) + p.origin) % ny
    return np.ascontiguousarray(field[..., idx, :])


class HaloExchange:
    """Halo exchange of one slab with the slabs of ranks rank - 1 (below) and
    rank + 1 (above), wrapping on a periodic axis.  Every exchange posts its sends
    and receives together (batch_isend_irecv), in an order in which each send meets
    its receive on the other side even when both neighbours are the same rank (two
    slabs on a periodic axis), and tags them by direction (0 up, 1 down)."""

    def __init__(self, rank: int, world: int, periodic: bool, nelem: int, device, group=None):
        import torch
        self.rank, self.world, self.group = rank, world, group
        self.up: Optional[int] = rank + 1 if rank + 1 < world else (0 if periodic and world > 1 else None)
        self.down: Optional[int] = rank - 1 if rank > 0 else (world - 1 if periodic and world > 1 else None)
        z = lambda: torch.zeros(nelem, dtype=torch.float32, device=device)  # noqa: E731
        self.send_up, self.send_down, self.recv_up, self.recv_down = z(), z(), z(), z()

    def exchange(self, pack, unpack):
        """pack(side, buf) fills buf with this slab's crossing row on side (0: the
        first row, sent down; 1: the last row, sent up); unpack(side, buf) writes a
        neighbour's row into the halo row on that side."""
        import torch.distributed as dist
        ops = []
        if self.up is not None:
            pack(1, self.send_up)
            ops.append(dist.P2POp(dist.isend, self.send_up, self.up, self.group, tag=0))
        if self.down is not None:
            ops.append(dist.P2POp(dist.irecv, self.recv_down, self.down, self.group, tag=0))
            pack(0, self.send_down)
            ops.append(dist.P2POp(dist.isend, self.send_down, self.down, self.group, tag=1))
        if self.up is not None:
            ops.append(dist.P2POp(dist.irecv, self.recv_up, self.up, self.group, tag=1))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        if self.down is not None:
            unpack(0, self.recv_down)
        if self.up is not None:
            unpack(1, self.recv_up)


def allreduce_sums(values: np.ndarray, device, group=None) -> np.ndarray:
    """FP64 sum over the ranks of per-slab sums (the whole lattice's sums)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(values, dtype=np.float64), device=device)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


class SlabSolver:
    """This rank's slab of the lattice `pb` on the current CUDA device, FP32
    populations, one step per launch, with the halo exchange after every step.
    The deviation references (phi_ref, p_ref_grad) are those of the whole lattice,
    so every node computes the bits it computes in the whole lattice."""

    def __init__(self, pb: Problem, rank: int, world: int, group=None, block=None):
        import torch
        self.pb, self.rank, self.world, self.group = pb, rank, world, group
        self.device = torch.device("cuda", torch.cuda.current_device())
        periodic = pb.south.kind == "periodic"
        self.plan = plan(pb.ny, world, periodic)[rank]
        p = self.plan
        sub = pb.replace(ny=p.lny, phi0=local_rows(pb.phi0, p, pb.ny), u0=local_rows(pb.u0, p, pb.ny),
                         p0=None if pb.p0 is None else local_rows(pb.p0, p, pb.ny))
        self.stream = torch.cuda.current_stream().cuda_stream
        grid, dif, src, frc, bc, opt = lib.structs_from_problem(
            sub, "fp32", self.stream, block, phi_ref=lib.default_phi_ref(pb), p_ref_grad=lib.default_p_ref_grad(pb),
            resident=-1, temporal=-1)
        opt.halo_rows, opt.origin_y, opt.ny_global = p.halo, (p.origin if p.halo else 0), (pb.ny if p.halo else 0)
        self.h = lib.cdf_lb_create(grid, pb.m, dif, pb.nu, src, frc, bc, opt)
        self.m, self.nx = pb.m, pb.nx
        lib.cdf_lb_init_moments(self.h, sub.phi0, sub.u0, sub.p0)
        self.ex = HaloExchange(rank, world, periodic, (3 + pb.m) * pb.nx, self.device, group)
        self.exchange()

    def close(self):
        if getattr(self, "h", None):
            lib.cdf_lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def exchange(self):
        self.ex.exchange(lambda side, buf: lib.cdf_lb_halo_pack(self.h, side, buf.data_ptr()),
                         lambda side, buf: lib.cdf_lb_halo_unpack(self.h, side, buf.data_ptr()))

    def step(self, n: int = 1):
        for _ in range(int(n)):
            lib.cdf_lb_step(self.h, 1)
            self.exchange()

    def moments(self) -> np.ndarray:
        """Moments of the rows this slab updates, [m+3][rows][nx]."""
        out = np.empty((self.m + 3, self.plan.lny, self.nx))
        lib.cdf_lb_moments(self.h, out)
        lo = self.plan.halo & 1
        return out[:, lo:lo + self.plan.rows]

    def mass(self) -> np.ndarray:
        out = np.empty(self.m)
        lib.cdf_lb_mass(self.h, out)
        return allreduce_sums(out, self.device, self.group)

    def run_to_steady(self, tol: float, check_every: int = 1000, max_steps: int = 10 ** 7):
        """The stop test of cdf_lb_run_to_steady on the whole lattice: every rank's
        FP64 change sums all-reduced before the test."""
        m, taken, R = self.m, 0, float("inf")
        q = np.empty(3 * m + 5)
        while taken < max_steps:
            lib.cdf_lb_snapshot(self.h)
            k = min(check_every, max_steps - taken)
            self.step(k)
            taken += k
            lib.cdf_lb_change_sums(self.h, q)
            tot = allreduce_sums(q, self.device, self.group)
            if tot[3 * m + 4] > 0:
                raise lib.CdfError(lib.CDF_EUNSTABLE, "non-finite moments in a slab")
            R = max(tot[m + f] / max(tot[2 * m + 2 + f], 1e-300) for f in range(m + 2))
            if k == check_every and R < tol:
                return True, taken, R
        return False, taken, R
