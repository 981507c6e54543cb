"""Pins of the 3-D FP64 oracle (oracle/cdf_oracle3d.c: D3Q7 scalars with
cs^2 = 1/4, D3Q19 fluid with cs^2 = 1/3), each against what the paper and the
mathematics fix rather than against the oracle's own formulas:

* the moment conditions the Taylor expansion of the model needs (Eq. moment,
  Eq. momentNS) for f^eq, h^eq, F_i and G on the D3Q7/D3Q19 lattices;
* Eq. omega-D read back: (omega^-1 - I/2) cs_s^2 = D;
* the continuum limit of an eigenmode of D on a diagonal wave vector: decay at
  eig(D) |k|^2 with second-order convergence;
* exact scalar mass conservation in a periodic box and in a walled box;
* plane Poiseuille flow, exact with half-way bounce-back at tau = 1/2 + sqrt(3/16),
  along two different axes; a z-dependent shear wave decaying at nu k^2;
* the steady linear profile between two anti-bounce-back Dirichlet walls;
and a planted-mistake test that every pin set catches.
"""
import math

import numpy as np
import pytest

from oracle import oracle3d as O3
from paper_2101_03055_gb300 import inputs as I


@pytest.fixture(scope="module")
def o3():
    O3.build()
    return O3


def c7():
    return np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, 0, 0], [0, -1, 0], [0, 0, -1]], float)


def c19():
    c = [[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
    c += [[1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [-1, 0, 1], [1, 0, -1],
          [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]]
    return np.array(c, float)


# ---------------------------------------------------------------------------
# moment conditions
# ---------------------------------------------------------------------------
def test_scalar_equilibrium_moments(o3):
    """sum f^eq = phi, sum c f^eq = phi u, sum c c f^eq = phi cs_s^2 I (lambda = I,
    vartheta = 0) with cs_s^2 = 1/4 on D3Q7."""
    c = c7()
    for phi, u in [(1.3, (0.02, -0.01, 0.03)), (0.7, (0.0, 0.05, -0.04))]:
        f = o3.feq_scalar(phi, u)
        assert f.sum() == pytest.approx(phi, abs=1e-15)
        np.testing.assert_allclose(c.T @ f, phi * np.array(u), atol=1e-16)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", f, c, c), phi * 0.25 * np.eye(3), atol=1e-15)


def test_fluid_equilibrium_moments(o3):
    """He-Luo incompressible h^eq (Eq. heq) on D3Q19: sum = rho0, first moment u,
    second moment p I + u u (p the lattice pressure)."""
    c = c19()
    for p, u in [(0.013, (0.02, -0.01, 0.03)), (-0.2, (0.05, 0.0, -0.02))]:
        h = o3.heq(p, u, 1.0)
        assert h.sum() == pytest.approx(1.0, abs=1e-15)
        np.testing.assert_allclose(c.T @ h, u, atol=1e-16)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", h, c, c), p * np.eye(3) + np.outer(u, u), atol=1e-15)


def test_force_population_moments(o3):
    c = c19()
    F = np.array([1e-4, -3e-4, 2e-4])
    Fi = o3.force_pop(F)
    assert abs(Fi.sum()) < 1e-19
    np.testing.assert_allclose(c.T @ Fi, F, atol=1e-19)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", Fi, c, c), 0.0, atol=1e-19)


def test_relaxation_and_auxiliary_source(o3):
    """(omega^-1 - I/2) cs_s^2 = D; sum_i G_{i,a} = 0 and sum_i c_i G_{i,a} =
    sum_b (delta_ab - omega_ab/2)(u S_b + phi_b F) (Eq. Gi)."""
    D = np.array([[0.05, 0.01], [0.005, 0.03]])
    om = o3.relaxation_matrix(D)
    np.testing.assert_allclose((np.linalg.inv(om) - 0.5 * np.eye(2)) * 0.25, D, atol=1e-15)
    phi, u, S, F = np.array([1.1, 0.9]), np.array([0.01, -0.02, 0.03]), np.array([1e-3, -2e-3]), \
        np.array([2e-4, 1e-4, -3e-4])
    G = o3.aux_source(om, phi, u, S, F)
    np.testing.assert_allclose(G.sum(axis=1), 0.0, atol=1e-18)
    want = (np.eye(2) - 0.5 * om) @ (S[:, None] * u[None, :] + phi[:, None] * F[None, :])
    np.testing.assert_allclose(G @ c7(), want, atol=1e-18)


def _uniform_box(S=(1e-3, -2e-3), F=(2e-4, 1e-4, -3e-4), u=(0.01, -0.02, 0.03), phi=(1.1, 0.9), p=0.01):
    n = 2
    shape = (n, n, n)
    pb = I.periodic_box3d(n, u0=0.0)
    return pb.replace(skind="const", S=np.array(S), g=tuple(F), F0=1.0,
                      phi0=np.stack([np.full(shape, v) for v in phi]),
                      u0=np.stack([np.full(shape, v) for v in u]), p0=np.full(shape, p))


def test_initial_moments_reproduce_inputs(o3):
    """f = f^eq(phi0, u0), h = h^eq(u0, p0) - F_i/2: Eqs. sum-phi/u/p return
    (phi0, u0, p0) at t = 0 (with a body force and a source)."""
    pb = _uniform_box()
    M = o3.Sim(pb).moments()
    np.testing.assert_allclose(M[:2, 0, 0, 0], [1.1, 0.9], rtol=1e-15)
    np.testing.assert_allclose(M[2:5, 0, 0, 0], [0.01, -0.02, 0.03], atol=1e-17)
    assert M[5, 0, 0, 0] == pytest.approx(0.01, abs=1e-16)


def test_node_update_moments(o3):
    """The moment conditions through one whole node update from equilibrium:
    sum_i f*_{i,a} = phi_a + S_a and sum_i c_i f*_{i,a} = phi_a u + sum_b (delta_ab
    - omega_ab/2)(u S_b + phi_b F) (Eq. evolution12 with Eqs. source and Gi);
    sum_i c_i h*_i = u + F/2 (Eqs. evolution3 and force with sum-u)."""
    S, F, u, phi = np.array([1e-3, -2e-3]), np.array([2e-4, 1e-4, -3e-4]), np.array([0.01, -0.02, 0.03]), \
        np.array([1.1, 0.9])
    pb = _uniform_box(S, F, u, phi)
    f, h = o3.Sim(pb).post_collision()
    fz, hz = f[..., 0, 0, 0], h[:, 0, 0, 0]
    om = np.linalg.inv(pb.D / 0.25 + 0.5 * np.eye(2))
    np.testing.assert_allclose(fz.sum(axis=1), phi + S, rtol=1e-14)
    want = phi[:, None] * u[None, :] + (np.eye(2) - 0.5 * om) @ (S[:, None] * u[None, :] + phi[:, None] * F[None, :])
    np.testing.assert_allclose(fz @ c7(), want, atol=1e-17)
    np.testing.assert_allclose(c19().T @ hz, u + 0.5 * F, atol=1e-17)


# ---------------------------------------------------------------------------
# continuum limit of an eigenmode of D
# ---------------------------------------------------------------------------
def _diag_mode_rate(o3, N, j):
    D = np.array([[0.05, 0.01], [0.005, 0.03]])
    lam, V = np.linalg.eig(D)
    order = np.argsort(lam.real)
    lam, V = lam.real[order], V.real[:, order]
    left = np.linalg.inv(V)
    kv = 2 * math.pi / N * np.ones(3)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    th = kv[0] * x + kv[1] * y + kv[2] * z
    pb = I.periodic_box3d(N, u0=0.0, nu=0.1)
    pb = pb.replace(phi0=1.0 + 1e-3 * V[:, j][:, None, None, None] * np.cos(th)[None])
    s = o3.Sim(pb)
    amps, ts = [], []
    T1, T2 = N * N // 8, N * N // 2
    s.step(T1)
    for t in range(T1, T2 + 1, max(1, N * N // 32)):
        if t > T1:
            s.step(max(1, N * N // 32))
        M = s.moments()[:2]
        amps.append(abs(left[j] @ (M * np.cos(th)[None]).sum(axis=(1, 2, 3)) * 2 / N ** 3))
        ts.append(t)
    rate = -np.polyfit(ts, np.log(amps), 1)[0] / (kv @ kv)
    return lam[j], rate


def test_diagonal_mode_decays_with_eig_d(o3):
    for j in (0, 1):
        lam, r8 = _diag_mode_rate(o3, 8, j)
        _, r16 = _diag_mode_rate(o3, 16, j)
        e8, e16 = abs(r8 / lam - 1), abs(r16 / lam - 1)
        # consistent and at least second order: the error falls >= 3x per halving
        # of k (higher-order terms are still visible at N = 8)
        assert e16 < 3e-3, (j, e8, e16)
        assert e8 / e16 > 3.0, (j, e8, e16)


def test_scalar_mode_moves_with_the_fluid(o3):
    """A scalar Fourier mode in a uniform flow U (periodic, no force: the fluid stays
    uniform) travels at U along each axis in turn."""
    N = 32
    for axis in range(3):
        dims = [2, 2, 2]
        dims[axis] = N
        nz, ny, nx = dims[2], dims[1], dims[0]
        pb = I.periodic_box3d(nx, ny, nz, u0=0.0)
        coord = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")[2 - axis]
        k = 2 * math.pi / N
        u = np.zeros((3, nz, ny, nx))
        u[axis] = 0.1
        pb = pb.replace(u0=u, phi0=1.0 + 1e-3 * np.cos(k * coord)[None] * np.ones((2, 1, 1, 1)))
        s = o3.Sim(pb)
        ts, ph = [], []
        for t in range(0, 161, 20):
            if t:
                s.step(20)
            c = (s.moments()[0] * np.exp(-1j * k * coord)).sum()
            ts.append(t)
            ph.append(np.angle(c))
        speed = -np.polyfit(ts, np.unwrap(ph), 1)[0] / k
        assert speed == pytest.approx(0.1, rel=1e-3), (axis, speed)


# ---------------------------------------------------------------------------
# conservation, reduction to 2-D, Dirichlet walls
# ---------------------------------------------------------------------------
def test_mass_conservation(o3):
    pb = I.periodic_box3d(10, 8, 6, u0=0.03)
    s = o3.Sim(pb)
    a = s.moments()[:2].sum(axis=(1, 2, 3))
    s.step(150)
    assert np.abs(s.moments()[:2].sum(axis=(1, 2, 3)) / a - 1).max() < 1e-13
    walled = pb.replace(sides=[I.wall_side(2) for _ in range(6)])
    s = o3.Sim(walled)
    a = s.moments()[:2].sum(axis=(1, 2, 3))
    s.step(150)
    assert np.abs(s.moments()[:2].sum(axis=(1, 2, 3)) / a - 1).max() < 1e-13


def _poiseuille(o3, axis_wall, axis_flow, H=10, L=4):
    """Steady channel flow between no-slip walls normal to axis_wall, driven by a
    constant force along axis_flow, periodic elsewhere."""
    tau = 0.5 + math.sqrt(3.0 / 16.0)  # half-way bounce-back is exact for this tau
    nu = (tau - 0.5) / 3.0
    dims = [L, L, L]
    dims[axis_wall] = H
    nx, ny, nz = dims
    sides = [I.periodic_side(1) for _ in range(6)]
    sides[2 * axis_wall] = sides[2 * axis_wall + 1] = I.wall_side(1)
    g = [0.0, 0.0, 0.0]
    g[axis_flow] = 1.0
    F0 = 1e-6
    pb = I.Problem3D("channel", nx, ny, nz, 1, [[0.05]], nu, g=tuple(g), F0=F0, sides=sides)
    s = o3.Sim(pb)
    s.step(8000)
    M = s.moments()
    yw = np.arange(H) + 0.5
    want = F0 / (2 * nu) * yw * (H - yw)
    prof = np.moveaxis(M[1 + axis_flow], 2 - axis_wall, 0)  # [wall axis, ...]
    return prof, want, M


def test_channel_flow_is_the_exact_parabola(o3):
    """Plane Poiseuille flow with half-way bounce-back walls: at tau = 1/2 +
    sqrt(3/16) the steady lattice solution is the parabola F y (H - y) / (2 nu)
    with the walls half a spacing outside the first and last node, exactly;
    checked with the walls normal to y (flow along x) and normal to x (flow along z)."""
    for wall, flow in ((1, 0), (0, 2)):
        prof, want, M = _poiseuille(o3, wall, flow)
        np.testing.assert_allclose(prof, np.broadcast_to(want[:, None, None], prof.shape), rtol=1e-9)
        others = [1 + d for d in range(3) if d != flow]
        assert np.abs(M[others]).max() < 1e-15


def test_shear_wave_decays_with_nu(o3):
    """u_x = U sin(k z) with k = 2 pi / N (a z-dependent shear wave) decays at
    nu k^2, second order in k: the fluid couples along z with the D3Q19 weights."""
    errs = []
    for N in (16, 32):
        z = np.arange(N)
        u = np.zeros((3, N, 2, 2))
        u[0] = 1e-3 * np.sin(2 * math.pi * z / N)[:, None, None]
        pb = I.Problem3D("shear", 2, 2, N, 1, [[0.05]], 0.1, u0=u)
        s = o3.Sim(pb)
        T1, T2 = N * N // 16, N * N // 4
        s.step(T1)
        a1 = (s.moments()[1][:, 0, 0] * np.sin(2 * math.pi * z / N)).sum()
        s.step(T2 - T1)
        a2 = (s.moments()[1][:, 0, 0] * np.sin(2 * math.pi * z / N)).sum()
        rate = math.log(a1 / a2) / (T2 - T1) / (2 * math.pi / N) ** 2
        errs.append(abs(rate / 0.1 - 1))
    assert errs[1] < 3e-3 and 3.0 < errs[0] / errs[1] < 5.0, errs


def test_dirichlet_walls_give_the_linear_profile(o3):
    """Two anti-bounce-back walls (phi = 1 at x-, 0 at x+), no flow, no-flux y and
    z walls: the steady scalar is linear through the half-way walls,
    phi = 1 - (x + 1/2) / nx, to round-off (both scalars, cross-diffusion on)."""
    n = 9
    hot = I.wall_side(2, I.NOSLIP, [I.DIRICHLET] * 2, [1.0, 1.0])
    cold = I.wall_side(2, I.NOSLIP, [I.DIRICHLET] * 2, [0.0, 0.0])
    pb = I.periodic_box3d(n, 5, 4, u0=0.0).replace(sides=[hot, cold] + [I.wall_side(2) for _ in range(4)],
                                                    phi0=np.full((2, 4, 5, n), 0.5))
    s = o3.Sim(pb)
    s.step(6000)
    M = s.moments()
    want = 1.0 - (np.arange(n) + 0.5) / n
    np.testing.assert_allclose(M[0], np.broadcast_to(want, M[0].shape), atol=1e-11)
    np.testing.assert_allclose(M[1], np.broadcast_to(want, M[1].shape), atol=1e-11)


# ---------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------
PLANTED3D = [
    ("D3Q7 cs^2 of D2Q5", "static const double CS2S = 1.0 / 4.0;", "static const double CS2S = 1.0 / 3.0;"),
    ("drop G", "+ Si + G[a * 7 + i] +", "+ Si +"),
    ("transpose omega", "coll += omega[a * m + b] * (f[b * 7 + i]", "coll += omega[b * m + a] * (f[b * 7 + i]"),
    ("D3Q19 diagonal weight", "W19_2 = 1.0 / 36.0", "W19_2 = 1.0 / 30.0"),
    ("pressure without W0", "(nonrest - W19_0 * uu / (2.0 * CS2))", "(nonrest - uu / (2.0 * CS2))"),
    ("anti-bounce-back sign", "= -v + 2.0 * Q7_W[i] * P->value[side][a]", "= v + 2.0 * Q7_W[i] * P->value[side][a]"),
    ("fluid bounce-back keeps the direction", "s->hnew[node * 19 + io] = v;", "s->hnew[node * 19 + i] = v;"),
    ("no half force in u", "u[d] = j[d] + 0.5 * F[d];", "u[d] = j[d];"),
    ("scalars stream backwards", "T[d] = X[d] + Q7_C[i][d];", "T[d] = X[d] - Q7_C[i][d];"),
    ("D3Q7 z velocity dropped from f^eq", "double cu = Q7_C[i][0] * u[0] + Q7_C[i][1] * u[1] + Q7_C[i][2] * u[2];",
     "double cu = Q7_C[i][0] * u[0] + Q7_C[i][1] * u[1];"),
]


def _pins():
    import sys
    mod = sys.modules[__name__]
    return [getattr(mod, n) for n in dir(mod) if n.startswith("test_") and n != "test_planted_mistakes_3d"]


@pytest.mark.parametrize("name,old,new", PLANTED3D, ids=[p[0] for p in PLANTED3D])
def test_planted_mistakes_3d(o3, tmp_path, name, old, new):
    src = o3.source_text()
    assert src.count(old) == 1, name
    mutant = o3.Binding(o3.compile_source(src.replace(old, new), str(tmp_path / "mutant3d.so")))
    for pin in _pins():
        try:
            pin(mutant)
        except (AssertionError, FloatingPointError, ValueError, np.linalg.LinAlgError):
            return
    pytest.fail(f"no pin caught the planted mistake: {name}")
