"""Two time steps per launch (cdf_options.temporal, step2_kernel).

Each CTA updates its tile plus a one-node halo from global memory into shared
memory, then the tile again from shared memory; every node runs the same pull
table and collision as the one-step kernel.  So every result (moments,
populations, S(t - 1)) must be bitwise equal to the one-step kernel's
(temporal = -1) for every boundary combination, tile shape, scalar count and
step count (odd counts end with one single step), and within the FP32 bound
of the FP64 oracle.
"""
import os

import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I

from test_parity_gpu import SIDE_CASES, _rand_problem, assert_parity

pytestmark = pytest.mark.gpu


def pair(cdf, pb, shape=None):
    a = cdf.Solver(pb, temporal=1, resident=-1, temporal_shape=shape)
    b = cdf.Solver(pb, temporal=-1, resident=-1, block=(128, 1))
    ia, ib = a.info(), b.info()
    assert ia.temporal == 1 and ib.temporal == 0
    if shape is not None:
        assert (ia.block_x, ia.block_y, ia.tile_x, ia.tile_y) == (shape[0], shape[1], shape[0] - 2, shape[2])
    return a, b


def assert_same(a, b):
    assert np.array_equal(a.moments(), b.moments())
    fa, ha, sa = a.populations()
    fb, hb, sb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb) and np.array_equal(sa, sb)
    assert a.t == b.t


@pytest.mark.parametrize("pb", [
    I.chemotaxis_plume(512, 256, seed=3),
    I.chemotaxis_plume(128, 64, seed=1),
    I.cross_diffusion_taylor_green(),
    I.ddc_cavity(128, Ra=1e5, Pr=0.7, Le=2.0, Nc=1.0, Df=0.1, Sr=0.1),
], ids=["plume512x256", "plume128x64", "taylor_green64", "cavity128"])
def test_two_step_launch_equals_one_step_kernel_bitwise(cdf, pb):
    a, b = pair(cdf, pb)
    for n in (1, 2, 37, 64, 100, 301):  # odd counts, short and long graph batches, remainders
        a.step(n)
        b.step(n)
    assert_same(a, b)


@pytest.mark.parametrize("shape", [(32, 8, 6), (32, 16, 30), (32, 17, 32), (64, 8, 14), (32, 32, 30), (64, 5, 9),
                                   (32, 8, 14)])
def test_tile_shapes_bitwise(cdf, shape):
    """CTA shapes with one, two and uneven passes of thread rows, halo regions of
    32 and 64 nodes, tiles that do not divide the lattice."""
    pb = I.chemotaxis_plume(200, 90, seed=6)
    a, b = pair(cdf, pb, shape)
    a.step(33)
    b.step(33)
    assert_same(a, b)


@pytest.mark.parametrize("xcase", list(SIDE_CASES))
@pytest.mark.parametrize("ycase", list(SIDE_CASES))
def test_boundaries_bitwise_and_oracle(cdf, oracle_mod, xcase, ycase):
    """Every pair of side types on a ragged 37 x 21 lattice: corners, free-slip
    images and anti-bounce-back links computed in the halo and in the tile."""
    pb = _rand_problem(37, 21, 2, 11, xcase, ycase)
    a, b = pair(cdf, pb, (32, 8, 6))
    a.step(60)
    b.step(60)
    assert_same(a, b)
    o = oracle_mod.OracleSim(pb)
    o.step(60)
    assert_parity(a, o, 2)


@pytest.mark.parametrize("m", [1, 2, 3, 4])
@pytest.mark.parametrize("xcase,ycase", [("periodic", "periodic"), ("mixed", "freeslip_dirichlet"),
                                         ("noslip_noflux", "periodic"), ("freeslip_dirichlet", "mixed")])
def test_fixed_shape_copy_bitwise(cdf, m, xcase, ycase):
    """The copy of the two-step kernel compiled for CTAs of 32 x 8 and tiles of
    30 x 14 (the autotuners' shape for large lattices and for the batched sweep;
    constant shared-memory strides) against one step per launch, on side pairs
    whose halo wraps or meets walls and corners, m = 1 .. 4."""
    pb = _rand_problem(71, 45, m, 20 + m, xcase, ycase)
    a, b = pair(cdf, pb, (32, 8, 14))
    a.step(29)
    b.step(29)
    assert_same(a, b)


@pytest.mark.parametrize("nx,ny,m", [(1, 1, 2), (9, 1, 2), (2, 30, 2), (130, 3, 2), (29, 19, 1), (29, 19, 3),
                                     (29, 19, 4), (70, 40, 4)])
def test_sizes_and_scalar_counts(cdf, nx, ny, m):
    """Walled lattices narrower than one tile, one-row lattices and m = 1 .. 4."""
    pb = _rand_problem(nx, ny, m, 5, "mixed", "noslip_noflux")
    a, b = pair(cdf, pb, (32, 4, 6) if m > 2 else (32, 8, 6))
    a.step(25)
    b.step(25)
    assert_same(a, b)


def test_periodic_wrap_and_consumption(cdf):
    """Periodic axes exactly as wide as the halo region (the wrapped halo node is
    the tile's own first column) with the consumption closure, whose S(t - 1)
    planes alternate between the launches."""
    pb = I.chemotaxis_plume(32, 40, seed=2)
    w = I.periodic_side(pb.m)
    pb = pb.replace(west=w, east=w)
    a, b = pair(cdf, pb, (32, 8, 38))
    a.step(41)
    b.step(41)
    assert_same(a, b)


def test_too_small_periodic_lattice_is_refused(cdf):
    pb = I.cross_diffusion_taylor_green(16, 16)
    with pytest.raises(cdf.CdfError) as e:
        cdf.Solver(pb, temporal=1, resident=-1, temporal_shape=(32, 8, 6))
    assert e.value.status == cdf.CDF_EINVAL


def test_checkpoint_and_run_to_steady(cdf, tmp_path):
    pb = I.ddc_cavity(64, Ra=1e4, Pr=0.7, Le=2.0, Nc=1.0, Df=0.1, Sr=0.1)
    a, b = pair(cdf, pb)
    a.step(51)
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    c = cdf.Solver(pb, temporal=1, resident=-1, init=False)
    c.load(path)
    b.step(51)
    c.step(77)
    b.step(77)
    assert_same(c, b)
    rc = c.run_to_steady(1e-30, check_every=41, max_steps=123)
    rb = b.run_to_steady(1e-30, check_every=41, max_steps=123)
    assert rc == rb and rc[1] == 123
    assert_same(c, b)


# ---------------------------------------------------------------------------
# 16-bit storage with two steps per launch
# ---------------------------------------------------------------------------
from test_parity_gpu import TOL16, developed_cavity, field_errors  # noqa: E402


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_16bit_two_step_launch_against_oracle(cdf, oracle_mod, storage):
    """The intermediate step stays in FP32 in shared memory, so the populations are
    rounded to 16 bits once per two steps.  Held to relative L2 1e-3 on every field
    and no worse than one step per launch by more than half."""
    for pb, steps in ((I.chemotaxis_plume(128, 64, seed=3), 2000), (developed_cavity(128), 2000)):
        a = cdf.Solver(pb, storage=storage, temporal=1, resident=-1)
        b = cdf.Solver(pb, storage=storage, temporal=-1, resident=-1)
        assert a.info().temporal == 1 and b.info().temporal == 0
        a.step(steps)
        b.step(steps)
        o = oracle_mod.OracleSim(pb)
        o.step(steps)
        ea = field_errors(a.moments(), o.moments(), 2)
        eb = field_errors(b.moments(), o.moments(), 2)
        print(storage, pb.name, "two-step", ea, "one-step", eb)
        for k, v in ea.items():
            assert v <= TOL16, (k, v)
        assert max(ea.values()) <= 1.5 * max(eb.values())


@pytest.mark.parametrize("xcase", list(SIDE_CASES))
@pytest.mark.parametrize("ycase", list(SIDE_CASES))
def test_16bit_two_step_boundaries_against_oracle(cdf, oracle_mod, xcase, ycase):
    pb = _rand_problem(37, 21, 2, 11, xcase, ycase)
    a = cdf.Solver(pb, storage="fp16", temporal=1, resident=-1, temporal_shape=(32, 8, 6))
    assert a.info().temporal == 1
    a.step(61)
    o = oracle_mod.OracleSim(pb)
    o.step(61)
    assert_parity(a, o, 2, tol=TOL16, populations=False)


@pytest.mark.parametrize("m", [1, 3, 4])
def test_16bit_two_step_scalar_counts(cdf, oracle_mod, m):
    pb = _rand_problem(45, 27, m, 9, "mixed", "noslip_noflux")
    a = cdf.Solver(pb, storage="fp16", temporal=1, resident=-1, temporal_shape=(32, 8, 6))
    a.step(40)
    o = oracle_mod.OracleSim(pb)
    o.step(40)
    assert_parity(a, o, m, tol=TOL16, populations=False)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("m,xcase,ycase", [(2, "periodic", "periodic"), (2, "mixed", "freeslip_dirichlet"),
                                           (1, "noslip_noflux", "periodic"), (3, "freeslip_dirichlet", "mixed"),
                                           (4, "periodic", "noslip_noflux")])
def test_16bit_two_step_fixed_copy_bitwise(cdf, storage, m, xcase, ycase):
    """A node's two steps do not depend on the tile it is computed in (a halo node
    is recomputed by each CTA with the same arithmetic), so the copy of the 16-bit
    two-step kernel compiled for CTAs of 32 x 8 and tiles of 30 x 14 must give the
    bits of the general kernel run with another shape."""
    pb = _rand_problem(71, 45, m, 30 + m, xcase, ycase)
    a = cdf.Solver(pb, storage=storage, temporal=1, resident=-1, temporal_shape=(32, 8, 14))
    b = cdf.Solver(pb, storage=storage, temporal=1, resident=-1, temporal_shape=(32, 4, 14))
    for n in (2, 31):
        a.step(n)
        b.step(n)
    assert_same(a, b)
