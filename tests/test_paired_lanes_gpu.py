"""Two steps per launch with two nodes per thread (cdf_options.temporal_lanes = 2,
step2_kernel_x2).

Each thread of the paired-lane kernel updates rows ly and ly + 8 of its column
together: the two nodes are pulled one after the other and collide as the two
lanes of paired FP32 instructions.  Each lane performs the operations of the
scalar node update in the same order with the same rounding, so every result
(moments, populations, S(t - 1)) must be bitwise equal to one step per launch
(temporal = -1) for every boundary combination, both tile heights, m = 1 and 2,
every closure branch (consumption, regularised cut-off, the Sherman-Morrison
quotient, constant sources, varphi = 1) and the batched solver's chains.
"""
import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I

from test_parity_gpu import SIDE_CASES, _rand_problem, assert_parity

pytestmark = pytest.mark.gpu


def pair(cdf, pb, th=14):
    a = cdf.Solver(pb, temporal=1, resident=-1, temporal_shape=(32, 8, th, 2))
    b = cdf.Solver(pb, temporal=-1, resident=-1, block=(128, 1))
    ia = a.info()
    assert ia.temporal == 1 and ia.lanes == 2 and (ia.block_x, ia.block_y, ia.tile_y) == (32, 8, th)
    assert b.info().temporal == 0
    return a, b


def assert_same(a, b):
    assert np.array_equal(a.moments(), b.moments())
    fa, ha, sa = a.populations()
    fb, hb, sb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb) and np.array_equal(sa, sb)
    assert a.t == b.t


@pytest.mark.parametrize("th", [14, 30])
@pytest.mark.parametrize("pb", [
    I.chemotaxis_plume(200, 90, seed=6),
    I.chemotaxis_plume(128, 64, seed=1),
    I.cross_diffusion_taylor_green(),
    I.ddc_cavity(96, Ra=1e5, Pr=0.7, Le=2.0, Nc=1.0, Df=0.1, Sr=0.1),
], ids=["plume200x90", "plume128x64", "taylor_green64", "cavity96"])
def test_paired_lanes_equal_one_step_kernel_bitwise(cdf, pb, th):
    a, b = pair(cdf, pb, th)
    for n in (1, 2, 37, 64, 101):  # odd counts end with one single step
        a.step(n)
        b.step(n)
    assert_same(a, b)


@pytest.mark.parametrize("xcase", list(SIDE_CASES))
@pytest.mark.parametrize("ycase", list(SIDE_CASES))
def test_boundaries_bitwise_and_oracle(cdf, oracle_mod, xcase, ycase):
    """Every pair of side types on a ragged 37 x 21 lattice: rows of R1 outside
    the lattice, paired rows past the tile, corners and free-slip images."""
    pb = _rand_problem(37, 21, 2, 11, xcase, ycase)
    a, b = pair(cdf, pb, 14)
    a.step(60)
    b.step(60)
    assert_same(a, b)
    o = oracle_mod.OracleSim(pb)
    o.step(60)
    assert_parity(a, o, 2)


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("th", [14, 30])
@pytest.mark.parametrize("xcase,ycase", [("periodic", "periodic"), ("mixed", "freeslip_dirichlet"),
                                         ("noslip_noflux", "periodic")])
def test_scalar_counts_and_tile_heights(cdf, m, th, xcase, ycase):
    pb = _rand_problem(71, 45, m, 20 + m, xcase, ycase)
    a, b = pair(cdf, pb, th)
    a.step(29)
    b.step(29)
    assert_same(a, b)


@pytest.mark.parametrize("name", ["regularised_const_source", "sherman_morrison_quotient", "varphi1"])
def test_closure_branches_bitwise(cdf, name):
    """The per-lane parts of the paired update: the regularised cut-off (one
    rsqrt per lane), the chemotaxis quotient 1 / (1 + delta omega_10) (a constant
    D with omega_10 != 0: one division per lane), constant sources and the
    second-order force term."""
    if name == "regularised_const_source":
        pb = I.chemotaxis_plume(80, 40, seed=2).replace(r_regularised=True, eps=0.05, c_star=0.97)
    elif name == "sherman_morrison_quotient":
        pb = I.chemotaxis_plume(80, 40, seed=4).replace(D=np.array([[0.05, 0.01], [0.02, 0.25]]))
    else:
        pb = _rand_problem(48, 33, 2, 9, "noslip_noflux", "mixed").replace(g=(3e-3, -1e-2), beta=np.full(2, 0.1),
                                                                           F0=0.05, varphi=1.0)
    a, b = pair(cdf, pb, 14)
    a.step(41)
    b.step(41)
    assert np.isfinite(a.moments()).all()
    assert_same(a, b)
    if name == "regularised_const_source":
        pc = _rand_problem(40, 30, 2, 3, "periodic", "noslip_noflux").replace(skind="const",
                                                                              S=np.array([1e-4, -2e-4]))
        a, b = pair(cdf, pc, 30)
        a.step(33)
        b.step(33)
        assert_same(a, b)


def test_periodic_wrap_as_wide_as_the_region(cdf):
    """Periodic axes exactly as wide as the halo region (32 columns; 16 rows for
    tile height 14) with the consumption closure."""
    pb = I.chemotaxis_plume(32, 16, seed=2)
    per = I.periodic_side(pb.m)
    pb = pb.replace(west=per, east=per, south=per, north=per)
    a, b = pair(cdf, pb, 14)
    a.step(41)
    b.step(41)
    assert_same(a, b)


def test_refused_shapes(cdf):
    pb = _rand_problem(40, 30, 3, 1, "mixed", "noslip_noflux")
    for shape, p in (((32, 8, 14, 2), pb), ((32, 8, 6, 2), I.chemotaxis_plume(64, 40, seed=1)),
                     ((64, 8, 14, 2), I.chemotaxis_plume(96, 40, seed=1))):
        with pytest.raises(cdf.CdfError) as e:
            cdf.Solver(p, temporal=1, resident=-1, temporal_shape=shape)
        assert e.value.status == cdf.CDF_EINVAL
    with pytest.raises(cdf.CdfError) as e:  # 16-bit storage has its own two-step kernel
        cdf.Solver(I.chemotaxis_plume(64, 40, seed=1), storage="fp16", temporal=1, resident=-1,
                   temporal_shape=(32, 8, 14, 2))
    assert e.value.status == cdf.CDF_EINVAL


@pytest.mark.parametrize("th", [14, 30])
def test_batched_chains_of_paired_lanes(cdf, th):
    """Mode 2 of the batched solver with the paired-lane kernel: every instance
    bitwise equal to its own single solver."""
    pbs = [I.chemotaxis_plume(nx, ny, seed=s) for s, (nx, ny) in enumerate([(97, 41), (128, 64), (60, 33), (150, 70)])]
    b = cdf.BatchSolver(pbs, tile=(32, 8), mode=2, chain_tile_y=th, chain_lanes=2)
    info = b.info()
    assert (info.mode, info.chain_block_x, info.chain_block_y, info.chain_tile_y, info.chain_lanes) == (2, 32, 8, th, 2)
    b.step(37)
    for k, pb in enumerate(pbs):
        s = cdf.Solver(pb, temporal=-1, resident=-1, block=(128, 1))
        s.step(37)
        assert np.array_equal(b.moments(k), s.moments()), k


# ---- one step per launch, flat launch with two nodes per thread (step_kernel_flat_x2)

def flat_pair(cdf, pb, width=128):
    a = cdf.Solver(pb, temporal=-1, resident=-1, block=(width, 0, 2))
    b = cdf.Solver(pb, temporal=-1, resident=-1, block=(128, 1))
    ia = a.info()
    assert (ia.temporal, ia.lanes, ia.block_x, ia.block_y) == (0, 2, width, 0)
    return a, b


@pytest.mark.parametrize("width", [64, 128, 256])
@pytest.mark.parametrize("pb", [
    I.chemotaxis_plume(512, 256, seed=3),
    I.cross_diffusion_taylor_green(),
    I.ddc_cavity(96, Ra=1e5, Pr=0.7, Le=2.0, Nc=1.0, Df=0.1, Sr=0.1),
], ids=["plume512x256", "taylor_green64", "cavity96"])
def test_flat_paired_lanes_equal_one_step_kernel_bitwise(cdf, pb, width):
    a, b = flat_pair(cdf, pb, width)
    for n in (1, 33, 64):
        a.step(n)
        b.step(n)
    assert_same(a, b)


@pytest.mark.parametrize("xcase", list(SIDE_CASES))
@pytest.mark.parametrize("ycase", list(SIDE_CASES))
def test_flat_boundaries_bitwise(cdf, xcase, ycase):
    pb = _rand_problem(37, 21, 2, 11, xcase, ycase)
    a, b = flat_pair(cdf, pb)
    a.step(40)
    b.step(40)
    assert_same(a, b)


@pytest.mark.parametrize("nx,ny,m", [(1, 1, 2), (9, 1, 2), (1, 9, 1), (33, 17, 1), (130, 3, 2), (29, 19, 2)])
def test_flat_odd_sizes_and_scalar_counts(cdf, nx, ny, m):
    """Node counts whose second half is short of a warp, odd counts, m = 1 and 2."""
    pb = _rand_problem(nx, ny, m, 5, "periodic" if nx < 3 else "mixed", "periodic" if ny < 3 else "noslip_noflux")
    a, b = flat_pair(cdf, pb, 64)
    a.step(25)
    b.step(25)
    assert_same(a, b)


@pytest.mark.parametrize("name", ["regularised_const_source", "sherman_morrison_quotient", "varphi1"])
def test_flat_closure_branches_bitwise(cdf, name):
    if name == "regularised_const_source":
        pb = I.chemotaxis_plume(80, 40, seed=2).replace(r_regularised=True, eps=0.05, c_star=0.97)
    elif name == "sherman_morrison_quotient":
        pb = I.chemotaxis_plume(80, 40, seed=4).replace(D=np.array([[0.05, 0.01], [0.02, 0.25]]))
    else:
        pb = _rand_problem(48, 33, 2, 9, "noslip_noflux", "mixed").replace(g=(3e-3, -1e-2), beta=np.full(2, 0.1),
                                                                           F0=0.05, varphi=1.0)
    a, b = flat_pair(cdf, pb)
    a.step(41)
    b.step(41)
    assert np.isfinite(a.moments()).all()
    assert_same(a, b)


def test_flat_paired_lanes_on_slabs(cdf):
    """Slabs of a split lattice: a lane whose node is a halo row repeats the
    other lane's node and is not stored."""
    pb = I.chemotaxis_plume(96, 49, seed=5)
    s = cdf.SplitSolver(pb, 3, block=(64, 0, 2))
    w = cdf.Solver(pb, temporal=-1, resident=-1, block=(128, 1))
    s.step(30)
    w.step(30)
    assert np.array_equal(s.moments(), w.moments())


def test_flat_refused(cdf):
    for kw in (dict(block=(128, 1, 2)), dict(block=(128, 0, 2), storage="bf16")):
        with pytest.raises(cdf.CdfError) as e:
            cdf.Solver(I.chemotaxis_plume(64, 40, seed=1), temporal=-1, resident=-1, **kw)
        assert e.value.status == cdf.CDF_EINVAL
    with pytest.raises(cdf.CdfError) as e:
        cdf.Solver(_rand_problem(40, 30, 3, 1, "mixed", "noslip_noflux"), temporal=-1, resident=-1, block=(128, 0, 2))
    assert e.value.status == cdf.CDF_EINVAL
