"""The batched persistent solver (many uneven lattices, one launch per
`steps_per_launch` steps, bounded grid barrier) against the single-lattice
solver and the oracle."""
import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def small_sweep(count=5, seed=3):
    return I.chemotaxis_plume_sweep(count, seed=seed, wmin=16, wmax=140, hmin=9, hmax=70)


@pytest.mark.parametrize("tile,spl,mode,th", [((64, 4), 32, 0, 0), ((32, 8), 7, 0, 0), ((128, 1), 1, 0, 0),
                                              ((128, 1), 0, 1, 0), ((64, 4), 0, 1, 0), ((32, 8), 0, 2, 14),
                                              ((32, 4), 0, 2, 6), ((64, 8), 0, 2, 30)])
def test_batch_equals_single_lattice_solver(cdf, tile, spl, mode, th):
    """Each instance of the batch follows exactly the single-lattice solver: the
    same per-node update, bit for bit, across launches, grid barriers (persistent
    mode), graph-captured kernel chains (chain mode) and chains of two-step
    launches with an odd remainder (mode 2; 70 = two graphs of 32 steps + 6,
    then 3 more steps)."""
    pbs = small_sweep()
    b = cdf.BatchSolver(pbs, tile=tile, steps_per_launch=spl, mode=mode, chain_tile_y=th)
    info = b.info()
    assert info.mode == mode
    if mode == 2:
        assert (info.chain_block_x, info.chain_block_y, info.chain_tile_y) == (tile[0], tile[1], th)
    b.step(67)
    b.step(3)
    assert b.info().t == 70
    for k, pb in enumerate(pbs):
        s = cdf.Solver(pb)
        s.step(70)
        np.testing.assert_array_equal(b.moments(k), s.moments())


def test_batch_vs_oracle(cdf, oracle_mod):
    pbs = small_sweep(3, seed=4)
    b = cdf.BatchSolver(pbs)
    b.step(150)
    for k, pb in enumerate(pbs):
        o = oracle_mod.OracleSim(pb)
        o.step(150)
        Mo, Mg = o.moments(), b.moments(k)
        for a in range(2):
            assert np.linalg.norm(Mg[a] - Mo[a]) / np.linalg.norm(Mo[a]) <= 1e-5
        assert np.linalg.norm(Mg[2:4] - Mo[2:4]) / np.linalg.norm(Mo[2:4]) <= 1e-5


def test_batch_barrier_timeout_is_reported(cdf):
    """A barrier that can never complete (test hook) makes every wait run out;
    the kernel returns, the host reports CDF_ETIMEOUT and the GPU stays usable."""
    pbs = small_sweep(2, seed=5)
    b = cdf.BatchSolver(pbs, tile=(64, 4), test_unreachable_barrier=True, barrier_timeout_s=0.002)
    with pytest.raises(cdf.CdfError) as e:
        b.step(4)
    assert e.value.status == cdf.CDF_ETIMEOUT
    b.close()
    s = cdf.Solver(pbs[0])
    s.step(5)
    assert np.isfinite(s.moments()).all()


def test_batch_autotuned_full_sweep_runs(cdf):
    pbs = I.chemotaxis_plume_sweep(256, seed=0)
    b = cdf.BatchSolver(pbs)
    info = b.info()
    assert info.count == 256 and info.nodes == sum(p.nodes for p in pbs)
    b.step(40)
    for k in (0, 77, 255):
        M = b.moments(k)
        assert np.isfinite(M).all()
        s = cdf.Solver(pbs[k])
        s.step(40)
        np.testing.assert_array_equal(M, s.moments())
