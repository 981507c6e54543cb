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


def test_batch_device_moment_calls_match_the_host_calls(cdf):
    """cdf_batch_init_moments_device / cdf_batch_moments_device, per instance and for
    all instances back to back (k = -1), give the bits of the host FP64 calls (which
    round the same values to FP32), before and after steps; bad arguments are refused."""
    import torch
    pbs = small_sweep(4, seed=8)
    m = pbs[0].m

    def stack(pb):
        return np.concatenate([pb.phi0.reshape(m, pb.ny, pb.nx), pb.u0.reshape(2, pb.ny, pb.nx),
                               pb.p0.reshape(1, pb.ny, pb.nx)]).astype(np.float32)

    host = cdf.BatchSolver(pbs, mode=2, tile=(32, 8))
    dev = cdf.BatchSolver(pbs, mode=2, tile=(32, 8), init=False)
    fields = torch.from_numpy(np.concatenate([stack(pb).ravel() for pb in pbs])).cuda()
    dev.init_moments_device(fields)
    out = torch.empty(dev.stack_floats(), dtype=torch.float32, device="cuda")
    for steps in (0, 23):
        host.step(steps)
        dev.step(steps)
        dev.moments_device(out)
        got, off = out.cpu().numpy(), 0
        for k, pb in enumerate(pbs):
            n = (m + 3) * pb.nx * pb.ny
            want = host.moments(k)
            assert np.array_equal(got[off:off + n].reshape(want.shape).astype(np.float64), want)
            one = torch.empty(n, dtype=torch.float32, device="cuda")
            dev.moments_device(one, k)
            assert np.array_equal(one.cpu().numpy(), got[off:off + n])
            off += n
    # one instance re-initialised alone from its own stack: it restarts like a fresh batch's,
    # the others keep their state
    k = 2
    dev.init_moments_device(torch.from_numpy(stack(pbs[k]).ravel()).cuda(), k)
    fresh = cdf.BatchSolver(pbs, mode=2, tile=(32, 8))
    assert np.array_equal(dev.moments(k), fresh.moments(k))
    for j in (0, 1, 3):
        assert np.array_equal(dev.moments(j), host.moments(j))
    for bad in (-2, len(pbs)):
        with pytest.raises(cdf.CdfError):
            cdf.cdf_batch_moments_device(dev.h, bad, out.data_ptr())
    with pytest.raises(cdf.CdfError):
        cdf.cdf_batch_init_moments_device(dev.h, 0, 0)
