"""Nusselt and Sherwood numbers of the double-diffusive cavity (Sec. 3.2) from a
moment stack, on the CPU: the one-sided wall derivative through the wall value and
the first two cell centres (half and one and a half spacings from a half-way wall)
is exact for quadratic profiles, so fields sampled from known quadratics give the
wall fluxes in closed form on both walls, with the Soret / Dufour cross terms."""
import numpy as np
import pytest

from paper_2101_03055_gb300 import analysis as A


def stack(T_of_x, C_of_x, nx, ny, row_scale=None):
    x = (np.arange(nx) + 0.5) / nx
    s = np.ones(ny) if row_scale is None else row_scale
    M = np.zeros((5, ny, nx))
    M[0] = s[:, None] * T_of_x(x)[None, :]
    M[1] = s[:, None] * C_of_x(x)[None, :]
    return M


def test_wall_derivative_is_exact_for_quadratics():
    a, b, c, dx = 0.7, -1.3, 2.1, 0.05
    q = lambda x: a + b * x + c * x * x  # noqa: E731
    assert A.wall_derivative(q(dx / 2), q(3 * dx / 2), a, dx) == pytest.approx(b, rel=1e-12, abs=1e-12)


def test_linear_conduction_gives_unit_numbers_on_both_walls():
    M = stack(lambda x: 1 - x, lambda x: 1 - x, 40, 7)
    Nu, Sh, Nu_y, Sh_y = A.nusselt_sherwood(M, 0.0, 0.0)
    assert Nu == pytest.approx(1.0, rel=1e-12) and Sh == pytest.approx(1.0, rel=1e-12)
    assert Nu_y.shape == (7,)
    Nu_e, Sh_e, _, _ = A.nusselt_sherwood(M, 0.0, 0.0, T_wall=0.0, C_wall=0.0, east=True)
    assert Nu_e == pytest.approx(1.0, rel=1e-12) and Sh_e == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("D_CT,S_TC", [(0.0, 0.0), (0.2, -0.1), (-0.15, 0.3)])
def test_quadratic_profiles_with_cross_terms(D_CT, S_TC):
    """T = 1 - 1.5 x + 0.5 x^2, C = 1 - 0.4 x - 0.6 x^2: the flux in +x is
    Nu = -(T' + D_CT C'), Sh = -(S_TC T' + C') at x = 0 (west, walls T = C = 1) and
    at x = 1 (east, walls T(1), C(1)), averaged over rows scaled by s(y)."""
    T = lambda x: 1 - 1.5 * x + 0.5 * x * x  # noqa: E731
    C = lambda x: 1 - 0.4 * x - 0.6 * x * x  # noqa: E731
    s = np.array([0.5, 1.0, 1.5, 2.0])
    M = stack(T, C, 32, 4, row_scale=s)
    dT0, dC0, dT1, dC1 = -1.5, -0.4, -0.5, -1.6
    Nu, Sh, Nu_y, Sh_y = A.nusselt_sherwood(M, D_CT, S_TC, T_wall=1.0, C_wall=1.0)
    # rows scaled by s: wall values scale too only where s = 1, so compare row 1 exactly
    assert Nu_y[1] == pytest.approx(-(dT0 + D_CT * dC0), rel=1e-12)
    assert Sh_y[1] == pytest.approx(-(S_TC * dT0 + dC0), rel=1e-12)
    Me = stack(T, C, 32, 3)
    Nu, Sh, _, _ = A.nusselt_sherwood(Me, D_CT, S_TC)
    assert Nu == pytest.approx(-(dT0 + D_CT * dC0), rel=1e-12)
    assert Sh == pytest.approx(-(S_TC * dT0 + dC0), rel=1e-12)
    Nu_e, Sh_e, _, _ = A.nusselt_sherwood(Me, D_CT, S_TC, T_wall=T(1.0), C_wall=C(1.0), east=True)
    assert Nu_e == pytest.approx(-(dT1 + D_CT * dC1), rel=1e-12)
    assert Sh_e == pytest.approx(-(S_TC * dT1 + dC1), rel=1e-12)


def test_average_is_the_mean_over_rows():
    s = np.array([1.0, 2.0, 3.0])
    M = stack(lambda x: -x, lambda x: -2 * x, 16, 3, row_scale=s)  # wall values 0 = s * 0
    Nu, Sh, Nu_y, Sh_y = A.nusselt_sherwood(M, 0.0, 0.0, T_wall=0.0, C_wall=0.0)
    np.testing.assert_allclose(Nu_y, s, rtol=1e-12)
    np.testing.assert_allclose(Sh_y, 2 * s, rtol=1e-12)
    assert Nu == pytest.approx(2.0, rel=1e-12) and Sh == pytest.approx(4.0, rel=1e-12)
