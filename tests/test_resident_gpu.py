"""The tile-resident persistent step (cdf_options.resident).

It runs the same pull table and collision as the one-launch-per-step kernel,
with the tile's populations in shared memory and only the tile rings exchanged
through global memory, so every result must be bitwise equal to the global
kernel's (resident = -1), and within the FP32 bound of the FP64 oracle.  The
time-out path is exercised by a test hook that keeps one tile's step counter
from advancing: its neighbours' bounded waits run out and the host reports
CDF_ETIMEOUT with the context still usable.
"""
import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I

from test_parity_gpu import SIDE_CASES, _rand_problem, assert_parity

pytestmark = pytest.mark.gpu


def pair(cdf, pb, **kw):
    a = cdf.Solver(pb, resident=1, **kw)
    b = cdf.Solver(pb, resident=-1, block=(128, 1))
    assert a.info().resident == 1 and b.info().resident == 0
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
def test_resident_equals_global_kernel_bitwise(cdf, pb):
    a, b = pair(cdf, pb)
    for n in (1, 2, 37, 100):
        a.step(n)
        b.step(n)
    assert_same(a, b)
    info = a.info()
    assert info.tiles >= 1 and info.tile_x >= 1 and info.tile_y >= 1


@pytest.mark.parametrize("xcase", list(SIDE_CASES))
@pytest.mark.parametrize("ycase", ["periodic", "freeslip_dirichlet", "mixed"])
def test_resident_boundaries_bitwise_and_oracle(cdf, oracle_mod, xcase, ycase):
    pb = _rand_problem(37, 21, 2, 11, xcase, ycase)
    a, b = pair(cdf, pb)
    a.step(60)
    b.step(60)
    assert_same(a, b)
    o = oracle_mod.OracleSim(pb)
    o.step(60)
    assert_parity(a, o, 2)


@pytest.mark.parametrize("nx,ny,m", [(1, 1, 2), (9, 1, 2), (1, 9, 2), (2, 2, 2), (130, 3, 2), (29, 19, 1),
                                     (29, 19, 3), (29, 19, 4), (384, 384, 2)])
def test_resident_sizes_and_scalar_counts(cdf, nx, ny, m):
    pb = _rand_problem(nx, ny, m, 5, "periodic" if nx < 3 else "mixed", "periodic" if ny < 3 else "noslip_noflux")
    a, b = pair(cdf, pb)
    a.step(25)
    b.step(25)
    assert_same(a, b)


def test_resident_long_call_crosses_launches(cdf):
    """A call longer than one resident launch (4096 steps) continues bitwise."""
    pb = I.chemotaxis_plume(96, 48, seed=7)
    a, b = pair(cdf, pb)
    a.step(4096 + 5)
    b.step(4096 + 5)
    assert_same(a, b)


def test_resident_run_to_steady_and_restart(cdf, tmp_path):
    pb = I.ddc_cavity(48, Ra=1e4, Pr=0.7, Le=2.0, Nc=0.5, Df=0.1, Sr=0.1)
    a, b = pair(cdf, pb)
    ra = a.run_to_steady(1e-5, 1000, 200_000)
    rb = b.run_to_steady(1e-5, 1000, 200_000)
    assert ra == rb and ra[0]
    assert_same(a, b)
    path = str(tmp_path / "res.ckpt")
    a.save(path)
    a.step(50)
    b.step(50)
    c = cdf.Solver(pb, resident=1, init=False)
    c.load(path)
    c.step(50)
    assert np.array_equal(c.moments(), b.moments())


def test_resident_wait_timeout_is_reported(cdf):
    """One tile never publishes its step: the neighbours' waits (50 ms bound) run
    out, the next synchronising call returns CDF_ETIMEOUT, and the handle works
    again after a new initial state."""
    pb = I.chemotaxis_plume(128, 64, seed=1)
    s = cdf.Solver(pb, resident=1, wait_timeout_s=0.05, test_stall_tile=3)
    s.step(20)
    with pytest.raises(RuntimeError, match="timed out"):
        s.moments()
    ok = cdf.Solver(pb, resident=1)
    ok.step(20)
    ref = cdf.Solver(pb, resident=-1, block=(128, 1))
    ref.step(20)
    assert np.array_equal(ok.moments(), ref.moments())


def test_resident_refuses_what_does_not_fit(cdf):
    with pytest.raises(RuntimeError):
        cdf.Solver(I.periodic_box(1024, 1024), resident=1)
    with pytest.raises(RuntimeError):
        cdf.Solver(I.chemotaxis_plume(64, 32, seed=0), storage="fp16", resident=1)
