"""Case 1 of Sec. 2.1 on the GPU (cdf_options.prescribed_velocity): the
convection cross-diffusion equations alone in a steady prescribed velocity,
with the auxiliary source from the first-order time difference of phi u,
against the FP64 oracle's Case-1 mode.

Tolerance: relative L2 <= 1e-5 per scalar field (FP32 populations); the
reported velocity is the prescribed field rounded to FP32 and p is 0.
"""
import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I

from test_parity_gpu import SIDE_CASES, _rand_problem, rel_l2

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


def check(cdf, oracle_mod, pb, steps, block=None):
    s = cdf.Solver(pb, block=block)
    o = oracle_mod.OracleSim(pb)
    s.step(steps)
    o.step(steps)
    Mg, Mo = s.moments(), o.moments()
    m = pb.m
    errs = [rel_l2(Mg[a], Mo[a]) for a in range(m)]
    assert max(errs) <= TOL32, errs
    np.testing.assert_array_equal(Mg[m:m + 2], pb.u0.astype(np.float32).astype(np.float64))
    assert not Mg[m + 2].any()
    fg, _, _ = s.populations()
    fo, _ = o.post_collision()
    assert rel_l2(fg, fo) <= TOL32
    return s, errs


def cellular_u(nx, ny, U0=0.05):
    return I.cde_cellular(nx, ny, U0=U0).u0


def test_cellular_flow_with_walls(cdf, oracle_mod):
    _, errs = check(cdf, oracle_mod, I.cde_cellular(64, 48), 2000)
    print("cellular walls 64x48 x 2000:", errs)


def test_periodic_cellular_flow(cdf, oracle_mod):
    check(cdf, oracle_mod, I.cde_cellular(64, 64, walls=False, U0=0.08), 1000)


def test_uniform_advection_of_an_eigenmode(cdf, oracle_mod):
    pb = I.fourier_box(128, 4, 2, [[0.05, 0.01], [0.005, 0.03]], amp=(0.01, 0.02), u=(0.2, 0.05))
    check(cdf, oracle_mod, pb.replace(case1=True), 1500)


def test_chemotaxis_closures_in_a_prescribed_flow(cdf, oracle_mod):
    """Nonlinear D(phi) (Sherman-Morrison per node), consumption S(phi) and its
    time difference, Dirichlet oxygen at the top, in a cellular flow."""
    pb = I.chemotaxis_plume(48, 32, seed=2).replace(case1=True, g=(0.0, 0.0), u0=cellular_u(48, 32))
    s, _ = check(cdf, oracle_mod, pb.replace(r_regularised=True, eps=0.05), 800)
    # the step cut-off is decided in FP32 on the GPU: compare while c stays clear of c*
    s, _ = check(cdf, oracle_mod, pb, 200)
    assert np.abs(s.moments()[1] - pb.c_star).min() > 0.05


@pytest.mark.parametrize("xcase", ["periodic", "noslip_noflux", "freeslip_dirichlet", "mixed"])
@pytest.mark.parametrize("ycase", ["periodic", "mixed"])
def test_boundaries_on_a_ragged_lattice(cdf, oracle_mod, xcase, ycase):
    pb = _rand_problem(37, 21, 2, 13, xcase, ycase, force=False).replace(case1=True)
    check(cdf, oracle_mod, pb, 60)


@pytest.mark.parametrize("m", [1, 3, 4])
def test_other_scalar_counts(cdf, oracle_mod, m):
    pb = _rand_problem(29, 19, m, 3 + m, "mixed", "noslip_noflux", force=False).replace(case1=True)
    check(cdf, oracle_mod, pb, 40)


def test_block_shapes_restart_and_mass(cdf, tmp_path):
    pb = I.cde_cellular(80, 50, walls=False, U0=0.08)
    ref = None
    for blk in [(32, 4), (128, 1), (64, 2)]:
        s = cdf.Solver(pb, block=blk)
        m0 = s.mass()
        s.step(300)
        M = s.moments()
        if ref is None:
            ref = M
            assert np.abs(s.mass() / m0 - 1).max() < 1e-6  # periodic, divergence-free: conserved
        else:
            assert np.array_equal(M, ref), blk
    a = cdf.Solver(pb)
    a.step(100)
    path = str(tmp_path / "case1.ckpt")
    a.save(path)
    a.step(77)
    b = cdf.Solver(pb, init=False)
    b.load(path)
    b.step(77)
    assert np.array_equal(a.moments(), b.moments())


def test_case1_refusals(cdf):
    pb = I.cde_cellular(32, 16)
    with pytest.raises(RuntimeError):
        cdf.Solver(pb, storage="fp16")
    with pytest.raises(RuntimeError):
        cdf.Solver(pb.replace(g=(0.0, -1e-5)))
    with pytest.raises(RuntimeError):
        cdf.Solver(pb, resident=1)


def test_translation_invariance_bitwise(cdf):
    """A periodic Case-1 state (scalars and the prescribed velocity) rolled by
    (16, 3) nodes, stepped and rolled back equals the unrolled run bit for bit:
    no node's arithmetic depends on where it sits in its CTA or warp."""
    pb = I.cde_cellular(96, 40, walls=False, U0=0.08)
    a = cdf.Solver(pb, block=(32, 4))
    a.step(60)
    b = cdf.Solver(pb, block=(32, 4))
    sh, ax = (3, 16), (-2, -1)
    b.init_moments(np.roll(pb.phi0, sh, axis=ax), np.roll(pb.u0, sh, axis=ax))
    b.step(60)
    Ma, Mb = a.moments(), np.roll(b.moments(), (-3, -16), axis=ax)
    assert np.array_equal(Ma, Mb)


@pytest.mark.parametrize("shape", [None, (32, 8, 6), (64, 4, 9)])
def test_two_step_launch_equals_one_step_bitwise(cdf, tmp_path, shape):
    """Two Case-1 steps per launch (the scalar tiling of the two-step kernel;
    phi(t - 1) in two sets that alternate with the buffers) against one step per
    launch: bitwise equal on walls with Dirichlet sides, on a periodic box and on
    ragged side pairs, for odd step counts and across a checkpoint."""
    import os
    cases = [I.cde_cellular(64, 48), I.cde_cellular(96, 40, walls=False, U0=0.08)]
    cases += [_rand_problem(37, 21, 2, 11, xc, yc, force=False).replace(case1=True)
              for xc, yc in (("mixed", "freeslip_dirichlet"), ("noslip_noflux", "periodic"))]
    for pb in cases:
        a = cdf.Solver(pb, temporal=1, resident=-1, temporal_shape=shape)
        b = cdf.Solver(pb, temporal=-1, resident=-1, block=(128, 1))
        assert a.info().temporal == 1 and b.info().temporal == 0
        for n in (1, 2, 37, 64):
            a.step(n)
            b.step(n)
        assert np.array_equal(a.moments(), b.moments())
        fa, _, sa = a.populations()
        fb, _, sb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(sa, sb)
        path = os.path.join(tmp_path, "c1.bin")
        a.save(path)
        c = cdf.Solver(pb, temporal=1, resident=-1, temporal_shape=shape, init=False)
        c.load(path)
        c.step(33)
        b.step(33)
        assert np.array_equal(c.moments(), b.moments())
