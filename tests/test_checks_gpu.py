"""The checks build (libcdflb_checks.so, -DCDF_CHECKS): every population, moment
and shared-memory offset of the step kernels is tested before the access, and
every device buffer of a lattice or a batch lies between canary pads.

A child process loads the checks build (CDF_CHECKS=1) and runs every step-kernel
family -- one step per launch (2-D CTAs and the flat launch), two steps per
launch, the tile-resident step, FP16 and BF16 storage in both forms, Case 1 in
both forms, the batched solver in its three modes and a lattice split into
slabs -- over every pair of side types on ragged lattices and odd step counts.
No call may report CDF_ECHECK, and the moments must equal those of the normal
build bit for bit (the checks change no arithmetic).  The detectors themselves
are shown to fire by the library's self-test: an out-of-range offset routed
through the check on a 64-float buffer, and a byte written by the host into the
pad behind a buffer.  Nothing in these runs leaves its buffers: the check
replaces an out-of-range offset by an in-range one before the access."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_2101_03055_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

PAIRS = [("periodic", "periodic"), ("noslip_noflux", "freeslip_dirichlet"), ("mixed", "periodic"),
         ("freeslip_dirichlet", "mixed"), ("periodic", "noslip_noflux")]
STEPS = 23  # odd: the two-step paths end on a one-step launch


def run_cases(lib):
    """Moments of every case, in a fixed order, as a dict name -> array."""
    from test_parity_gpu import _rand_problem
    out = {}

    def solver(name, pb, **kw):
        s = lib.Solver(pb, **kw)
        s.step(STEPS - 10)
        s.step(10)
        out[name] = s.moments()

    for k, (xc, yc) in enumerate(PAIRS):
        pb = _rand_problem(37, 21, 2, 40 + k, xc, yc)
        solver(f"fp32_cta_{k}", pb, block=(32, 4), temporal=-1, resident=-1)
        solver(f"fp32_flat_{k}", pb, block=(64, 0), temporal=-1, resident=-1)
        solver(f"fp32_pair_{k}", pb, temporal=1, resident=-1, temporal_shape=(32, 8, 6))
        solver(f"fp32_resident_{k}", pb, resident=1)
        solver(f"fp16_cta_{k}", pb, storage="fp16", block=(32, 4), temporal=-1, resident=-1)
        solver(f"bf16_pair_{k}", pb, storage="bf16", temporal=1, resident=-1, temporal_shape=(32, 8, 6))
        c1 = _rand_problem(37, 21, 2, 60 + k, xc, yc, force=False).replace(case1=True)
        solver(f"case1_cta_{k}", c1, block=(32, 4), temporal=-1, resident=-1)
        solver(f"case1_pair_{k}", c1, temporal=1, resident=-1, temporal_shape=(32, 8, 6))
        sp = lib.SplitSolver(pb, 3)
        sp.step(STEPS)
        out[f"split_{k}"] = sp.moments()
    for m in (1, 3, 4):
        pb = _rand_problem(13, 7, m, 70 + m, "mixed", "noslip_noflux")
        solver(f"m{m}_cta", pb, block=(32, 2), temporal=-1, resident=-1)
        solver(f"m{m}_pair", pb, temporal=1, resident=-1, temporal_shape=(32, 4, 3))
    plume = I.chemotaxis_plume(41, 23, seed=3)
    solver("plume_pair", plume, temporal=1, resident=-1, temporal_shape=(32, 8, 6))
    solver("plume_fp16_pair", plume, storage="fp16", temporal=1, resident=-1, temporal_shape=(32, 8, 6))
    pbs = I.chemotaxis_plume_sweep(4, seed=9, wmin=16, wmax=90, hmin=9, hmax=50)
    for tile, mode, th in (((32, 8), 0, 0), ((64, 4), 1, 0), ((32, 8), 2, 6)):
        b = lib.BatchSolver(pbs, tile=tile, steps_per_launch=7 if mode == 0 else 0, mode=mode, chain_tile_y=th)
        b.step(STEPS)
        for j in range(len(pbs)):
            out[f"batch{mode}_{j}"] = b.moments(j)
    return out


def _child(path):
    import torch
    from paper_2101_03055_gb300 import lib
    torch.cuda.set_device(0)
    assert lib.CHECKS and lib.cdf_checks_enabled(), "the checks library was not loaded"
    st = lib.cdf_checks_selftest(0)
    msg0 = lib.cdf_lb_last_error()
    assert st == lib.CDF_ECHECK and "access site 99" in msg0, (st, msg0)
    st = lib.cdf_checks_selftest(1)
    msg1 = lib.cdf_lb_last_error()
    assert st == lib.CDF_ECHECK and "canary pad after" in msg1, (st, msg1)
    out = run_cases(lib)
    np.savez(path, **out)
    print(f"checks build: {len(out)} cases clean; self-test: {msg0} | {msg1}")


def test_checks_build_is_clean_and_bitwise_equal(cdf, tmp_path):
    from paper_2101_03055_gb300 import build
    build.build(checks=True)
    path = str(tmp_path / "checks.npz")
    env = dict(os.environ, CDF_CHECKS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), path], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    print(r.stdout.strip().splitlines()[-1])
    assert not cdf.CHECKS and cdf.cdf_checks_enabled() == 0
    assert cdf.cdf_checks_selftest(0) == cdf.CDF_EINVAL  # the normal build has no detectors
    got = np.load(path)
    want = run_cases(cdf)
    assert sorted(got.files) == sorted(want)
    for name, arr in want.items():
        assert np.array_equal(got[name], arr), name


if __name__ == "__main__":
    _child(sys.argv[1])
