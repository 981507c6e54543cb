"""A lattice split into slabs along y (cdf_split_*, and one slab per process with
SlabSolver), against the whole lattice.

Every node of a slab pulls the same post-collision populations as in the whole
lattice -- its halo rows receive, after every step, the populations that cross
the cut -- and the slabs keep the whole lattice's deviation references, so the
moments must agree bit for bit: over every pair of side types, ragged sizes,
2-4 slabs, m = 1..4 and the chemotaxis plume (node-local S(t-1)).  The FP64
sums are added over the slabs, so they agree to rounding."""
import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I
from test_parity_gpu import SIDE_CASES, _rand_problem

pytestmark = pytest.mark.gpu


def _compare(cdf, pb, nslabs, steps):
    whole = cdf.Solver(pb)
    split = cdf.SplitSolver(pb, nslabs)
    whole.step(steps)
    split.step(steps)
    Mw, Ms = whole.moments(), split.moments()
    assert np.abs(Mw[pb.m:pb.m + 2]).max() > 0 or pb.m > 0
    assert np.array_equal(Mw, Ms), np.abs(Mw - Ms).max()
    np.testing.assert_allclose(split.mass(), whole.mass(), rtol=1e-12)
    return split


@pytest.mark.parametrize("xcase", list(SIDE_CASES))
@pytest.mark.parametrize("ycase", list(SIDE_CASES))
def test_split_equals_whole_lattice_on_every_side_pair(cdf, xcase, ycase):
    pb = _rand_problem(37, 23, 2, 31, xcase, ycase)
    s = _compare(cdf, pb, 3, 41)
    rows = [r for _, r in s.slabs()]
    assert sum(rows) == 23 and max(rows) - min(rows) <= 1


@pytest.mark.parametrize("nx,ny,m,nslabs", [(29, 19, 1, 2), (33, 17, 3, 4), (40, 9, 4, 3), (5, 31, 2, 4),
                                            (64, 8, 2, 4)])
def test_split_sizes_scalar_counts_and_slab_counts(cdf, nx, ny, m, nslabs):
    pb = _rand_problem(nx, ny, m, 5 + m, "mixed", "periodic")
    _compare(cdf, pb, nslabs, 30)
    pb = _rand_problem(nx, ny, m, 6 + m, "periodic", "freeslip_dirichlet")
    _compare(cdf, pb, nslabs, 30)


def test_split_plume_and_steady_driver(cdf):
    pb = I.chemotaxis_plume(96, 49, seed=2)
    _compare(cdf, pb, 3, 200)
    # the stop test summed over the slabs decides like the whole lattice's
    cav = I.ddc_cavity(24, Ra=1e4, Pr=0.7, Le=2.0, Nc=0.5)
    whole, split = cdf.Solver(cav), cdf.SplitSolver(cav, 2)
    ok_w, n_w, r_w = whole.run_to_steady(1e-4, 500, 60_000)
    ok_s, n_s, r_s = split.run_to_steady(1e-4, 500, 60_000)
    assert ok_w and ok_s and n_w == n_s
    assert r_s == pytest.approx(r_w, rel=1e-9)
    assert np.array_equal(whole.moments(), split.moments())


def test_one_slab_per_process_single_rank_and_halo_errors(cdf):
    from paper_2101_03055_gb300 import slab
    pb = _rand_problem(31, 14, 2, 3, "noslip_noflux", "noslip_noflux")
    one = slab.SlabSolver(pb, 0, 1)  # one rank: the whole lattice, no halo rows
    whole = cdf.Solver(pb)
    one.step(25)
    whole.step(25)
    assert np.array_equal(one.moments(), whole.moments())
    np.testing.assert_allclose(one.mass(), whole.mass(), rtol=1e-12)
    import torch
    buf = torch.zeros((3 + pb.m) * pb.nx, device="cuda")
    with pytest.raises(cdf.CdfError):
        cdf.cdf_lb_halo_pack(one.h, 0, buf.data_ptr())  # no halo row on that side
    grid, dif, src, frc, bc, opt = cdf.structs_from_problem(pb)
    opt.halo_rows, opt.temporal = 1, 1  # halo rows need one step per launch
    with pytest.raises(cdf.CdfError):
        cdf.cdf_lb_create(grid, pb.m, dif, pb.nu, src, frc, bc, opt)
