"""The allocation-free entry point cdf_moment_sums_static.

Some callers cannot allocate device memory once they run (real-time loops,
plug-ins whose host owns all device memory through its own pool, processes
under a fixed memory quota).  cdf_moment_sums_static gives them the FP64
moment sums of cdf_lb_mass with its scratch in a static device array.  This
test calls it through the C ABI twice in a row, on two different states, and
checks each result against the existing entry point cdf_lb_mass, and that the
second call leaves the device's free memory unchanged (the first call may load
kernel code; that is the set-up the header asks callers to do at start-up).  It
lives in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_static_sums_match_existing_entry_point_twice(cdf):
    import torch
    pb = I.chemotaxis_plume(96, 48, seed=7)
    s = cdf.Solver(pb)
    m = pb.m
    fields = torch.empty((m + 3, pb.ny, pb.nx), dtype=torch.float32, device="cuda")
    out = torch.full((3 * m + 5,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        s.step(40 + 30 * call)
        s.moments_device(fields)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = cdf.cdf_moment_sums_static(fields.data_ptr(), 0, pb.nx, pb.ny, m, out.data_ptr(), 0)
        assert st == cdf.CDF_OK, cdf.cdf_lb_last_error()
        torch.cuda.synchronize()
        if call == 1:  # after the set-up of the first call nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:m], s.mass(), rtol=1e-12)  # same FP64 sums
        M = s.moments()
        np.testing.assert_allclose(got[2 * m + 2:3 * m + 4], np.abs(M[:m + 2]).reshape(m + 2, -1).sum(axis=1),
                                   rtol=1e-6)
        assert np.all(got[m:2 * m + 2] == 0.0) and got[3 * m + 4] == 0.0


def test_static_sums_residual_and_limits(cdf):
    import torch
    pb = I.chemotaxis_plume(64, 40, seed=8)
    s = cdf.Solver(pb)
    m = pb.m
    old = torch.empty((m + 3, pb.ny, pb.nx), dtype=torch.float32, device="cuda")
    new = torch.empty_like(old)
    out = torch.empty((3 * m + 5,), dtype=torch.float64, device="cuda")
    s.moments_device(old)
    s.step(25)
    s.moments_device(new)
    assert cdf.cdf_moment_sums_static(new.data_ptr(), old.data_ptr(), pb.nx, pb.ny, m, out.data_ptr(), 0) == 0
    torch.cuda.synchronize()
    diff = (new.double() - old.double()).abs()[: m + 2].reshape(m + 2, -1).sum(dim=1).cpu().numpy()
    np.testing.assert_allclose(out.cpu().numpy()[m:2 * m + 2], diff, rtol=1e-9)
    for bad_m, nx in ((5, pb.nx), (0, pb.nx), (m, 0)):
        st = cdf.cdf_moment_sums_static(new.data_ptr(), 0, nx, pb.ny, bad_m, out.data_ptr(), 0)
        assert st == cdf.CDF_EINVAL and cdf.cdf_lb_last_error()
