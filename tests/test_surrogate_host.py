"""Host-side pieces of the surrogate warm start (no GPU): the parameter draws, the
network's input planes, the map between the solver's moments and the network's
targets, the binomial filter, the hydrostatic pressure of a predicted state and the
resampling of a prediction to another lattice size.  Each is checked against a
property that fixes it exactly."""
import math

import numpy as np
import pytest

from paper_2101_03055_gb300 import surrogate as S


def test_parameter_draws_cover_the_stated_ranges_and_are_reproducible():
    prms = S.draw_parameters(400, 3)
    a = np.array([[math.log10(p["Ra"]), p["Nc"], p["Le"], p["Sr"], p["Df"]] for p in prms])
    lo, hi = np.array([4.0, -2.0, 1.0, 0.0, 0.0]), np.array([6.0, 2.0, 10.0, 0.5, 0.5])
    assert np.all(a >= lo) and np.all(a <= hi)
    # spread over the ranges (400 uniform draws reach within 3 % of each end)
    span = hi - lo
    assert np.all(a.min(axis=0) < lo + 0.03 * span) and np.all(a.max(axis=0) > hi - 0.03 * span)
    assert S.draw_parameters(400, 3) == prms
    assert S.draw_parameters(5, 4) != prms[:5]
    # a prefix of a longer draw is the shorter draw (counters 8k .. 8k + 4 per case)
    assert S.draw_parameters(7, 3) == prms[:7]


def test_input_planes_hold_the_scaled_parameters_and_cell_centres():
    prms = [dict(Ra=1e5, Nc=1.0, Le=5.5, Sr=0.25, Df=0.5), dict(Ra=1e4, Nc=-2.0, Le=10.0, Sr=0.0, Df=0.0)]
    n = 6
    x = S.input_planes(n, prms)
    assert x.shape == (2, n, n, S.IN_PAD) and x.dtype == np.float32
    np.testing.assert_allclose(x[0, 3, 2, :5], [0.0, 0.5, 0.0, 0.0, 1.0], atol=1e-7)
    np.testing.assert_allclose(x[1, 0, 5, :5], [-1.0, -1.0, 1.0, -1.0, -1.0], atol=1e-7)
    c = (np.arange(n) + 0.5) / n
    np.testing.assert_allclose(x[1, 4, :, 5], c, atol=1e-7)   # x varies along the row
    np.testing.assert_allclose(x[1, :, 4, 6], c, atol=1e-7)   # y along the column
    assert np.all(x[..., 7:] == 0.0)                          # padding channels


def test_targets_and_moments_are_inverse_maps():
    r = np.random.default_rng(0)
    n = 5
    M = np.zeros((5, n, n))
    M[0], M[1] = r.uniform(0, 1, (n, n)), r.uniform(0, 1, (n, n))
    M[2], M[3] = 0.02 * r.normal(size=(n, n)), 0.02 * r.normal(size=(n, n))
    y = S.targets_from_moments(M)
    assert y.shape == (n, n, 4)
    back = S.moments_from_prediction(y, velocity="raw")
    np.testing.assert_allclose(back[:4], M[:4], rtol=1e-6, atol=1e-7)  # float32 targets
    assert np.all(back[4] == 0.0)  # no problem given: no pressure
    assert np.all(S.moments_from_prediction(y)[2:4] == 0.0)  # default: fluid at rest
    np.testing.assert_array_equal(S.moments_from_prediction(y, velocity="filtered")[2:4],
                                  S.binomial_filter(back[2:4]))
    with pytest.raises(ValueError):
        S.moments_from_prediction(y, velocity="other")


def test_binomial_filter_keeps_linear_fields_and_removes_the_grid_scale_mode():
    n = 9
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lin = 0.3 * i - 0.7 * j + 2.0
    out = S.binomial_filter(lin[None])[0]
    np.testing.assert_allclose(out[1:-1, 1:-1], lin[1:-1, 1:-1], rtol=0, atol=1e-13)
    nyq = (-1.0) ** (i + j)
    assert np.abs(S.binomial_filter(nyq)[1:-1, 1:-1]).max() == 0.0
    const = np.full((2, n, n), 1.5)
    np.testing.assert_array_equal(S.binomial_filter(const), const)  # edges repeated: exact everywhere


def test_hydrostatic_pressure_of_a_prediction_balances_the_buoyancy():
    """p(j+1) - p(j) is the mean of F_y over the two rows (the discrete form of
    dp/dy = F_y between cell centres), and p has zero mean."""
    pb = S.cavity(12, dict(Ra=1e5, Nc=1.5, Le=2.0, Sr=0.1, Df=0.2))
    r = np.random.default_rng(1)
    y = np.zeros((12, 12, 4), np.float32)
    y[..., 2:] = r.uniform(-0.5, 0.5, (12, 12, 2))
    M = S.moments_from_prediction(y, pb)
    Fy = pb.g[1] * (pb.F0 + sum(pb.beta[a] * (M[a] - pb.phi_ref[a]) for a in range(2)))
    np.testing.assert_allclose(M[4][1:] - M[4][:-1], 0.5 * (Fy[1:] + Fy[:-1]), rtol=1e-12, atol=1e-15)
    assert abs(M[4].mean()) < 1e-15
    assert np.any(Fy != 0.0)


def test_resampling_a_prediction_reproduces_linear_fields_between_the_edge_cells():
    """Bilinear resampling between cell-centred grids is exact for fields linear in
    the cell-centre coordinates, wherever the fine cell centre lies between the
    coarse ones (the outermost fine cells are clamped to the edge value)."""
    pytest.importorskip("torch")
    m, n = 4, 12
    c = (np.arange(m) + 0.5) / m
    f = (np.arange(n) + 0.5) / n
    pred = np.zeros((1, m, m, 4), np.float32)
    pred[0, :, :, 0] = 1.0 + 2.0 * c[None, :]              # linear in x
    pred[0, :, :, 1] = -0.5 + 3.0 * c[:, None]             # linear in y
    pred[0, :, :, 2] = 0.25                                # constant
    pred[0, :, :, 3] = c[None, :] - c[:, None]             # linear in both
    up = S.upsample_prediction(pred, n)
    assert up.shape == (1, n, n, 4)
    inner = (f >= c[0]) & (f <= c[-1])
    ii = np.ix_(inner, inner)
    np.testing.assert_allclose(up[0, :, :, 0][ii], (1.0 + 2.0 * f[None, :] + 0 * f[:, None])[ii], atol=1e-6)
    np.testing.assert_allclose(up[0, :, :, 1][ii], (-0.5 + 3.0 * f[:, None] + 0 * f[None, :])[ii], atol=1e-6)
    np.testing.assert_allclose(up[0, :, :, 2], 0.25, atol=0)
    np.testing.assert_allclose(up[0, :, :, 3][ii], (f[None, :] - f[:, None])[ii], atol=1e-6)
