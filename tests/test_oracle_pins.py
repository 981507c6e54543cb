"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here runs on the CPU.  None re-types the oracle's code: each compares
it with a closed form, a moment condition the paper states, an exact linear
theory built independently in Fourier space, a textbook special case written
separately, or an invariant.  Together they are chosen so that a dropped term,
a wrong sign or index, or a transposed operand anywhere in the oracle fails at
least one of them (test_planted_mistakes_are_caught checks that directly).
"""
import math

import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I

CS2 = 1.0 / 3.0
Q5 = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1)])
W5 = np.array([1 / 3, 1 / 6, 1 / 6, 1 / 6, 1 / 6])
Q9 = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------------------
# P1: moment conditions of a single node (Eq. moment, Eq. momentNS)
# ---------------------------------------------------------------------------
def test_scalar_equilibrium_moments(oracle_mod):
    """Eq. moment with lambda = I, vartheta = 0: sum f^eq = phi, sum c f^eq = phi u,
    sum c c f^eq = phi cs^2 I."""
    r = _rng(1)
    for _ in range(20):
        phi, ux, uy = r.uniform(0.1, 2.0), r.uniform(-0.1, 0.1), r.uniform(-0.1, 0.1)
        f = oracle_mod.feq_scalar(phi, ux, uy, 0.0)
        assert f.sum() == pytest.approx(phi, rel=1e-14)
        np.testing.assert_allclose(Q5.T @ f, [phi * ux, phi * uy], rtol=1e-13, atol=1e-16)
        second = np.einsum("ia,ib,i->ab", Q5, Q5, f)
        np.testing.assert_allclose(second, phi * CS2 * np.eye(2), rtol=1e-13, atol=1e-16)


def test_scalar_equilibrium_vartheta_on_d2q5_is_anisotropic(oracle_mod):
    """The vartheta phi uu term of Eq. feq-phi cannot be carried by D2Q5: its
    second moment is not phi cs^2 I + phi uu (why the experiments' linear f^eq,
    vartheta = 0, is the reading taken for the CUDA path)."""
    phi, ux, uy = 1.0, 0.1, 0.05
    f = oracle_mod.feq_scalar(phi, ux, uy, 1.0)
    second = np.einsum("ia,ib,i->ab", Q5, Q5, f)
    target = phi * CS2 * np.eye(2) + phi * np.outer([ux, uy], [ux, uy])
    assert np.abs(second - target).max() > 1e-3


def test_fluid_equilibrium_moments(oracle_mod):
    """Eq. momentNSh: sum h^eq = rho0, sum c h^eq = u, sum c c h^eq = p I + u u,
    third moment cs^2 (delta delta + ...) . u (D2Q9 isotropy)."""
    r = _rng(2)
    for _ in range(20):
        p, ux, uy, rho0 = r.uniform(-0.01, 0.01), r.uniform(-0.1, 0.1), r.uniform(-0.1, 0.1), r.uniform(0.5, 2)
        h = oracle_mod.heq(p, ux, uy, rho0)
        u = np.array([ux, uy])
        assert h.sum() == pytest.approx(rho0, rel=1e-14)
        np.testing.assert_allclose(Q9.T @ h, u, rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(np.einsum("ia,ib,i->ab", Q9, Q9, h), p * np.eye(2) + np.outer(u, u),
                                   rtol=1e-12, atol=1e-16)
        third = np.einsum("ia,ib,ic,i->abc", Q9, Q9, Q9, h)
        d = np.eye(2)
        expect = CS2 * (np.einsum("ab,c->abc", d, u) + np.einsum("bc,a->abc", d, u) + np.einsum("ac,b->abc", d, u))
        np.testing.assert_allclose(third, expect, rtol=1e-12, atol=1e-16)


def test_force_population_moments(oracle_mod):
    """Eq. momentNS with varphi = 0: sum F_i = 0, sum c F_i = F, sum c c F_i = 0."""
    F = np.array([3e-4, -7e-4])
    Fi = oracle_mod.force_pop(*F)
    assert abs(Fi.sum()) < 1e-18
    np.testing.assert_allclose(Q9.T @ Fi, F, rtol=1e-13)
    assert np.abs(np.einsum("ia,ib,i->ab", Q9, Q9, Fi)).max() < 1e-18


def test_force_population_moments_with_varphi(oracle_mod):
    """Eq. force with its second-order part (varphi = 1, Case 2 of the appendix):
    sum F_i = 0, sum c F_i = F, sum c c F_i = varphi (uF + Fu) (Eq. momentNS)."""
    r = np.random.default_rng(11)
    for varphi in (0.0, 1.0, 0.5):
        F, u = r.normal(size=2) * 1e-3, r.normal(size=2) * 0.05
        Fi = oracle_mod.force_pop_phi(F, u, varphi)
        assert abs(Fi.sum()) < 1e-17
        np.testing.assert_allclose(Q9.T @ Fi, F, rtol=1e-12)
        want = varphi * (np.outer(u, F) + np.outer(F, u))
        np.testing.assert_allclose(np.einsum("ia,ib,i->ab", Q9, Q9, Fi), want, atol=1e-18)


def _accelerated_box(oracle_mod, varphi, steps, F=(2e-4, 1e-4), nu=0.1):
    m, n = 1, 4
    side = I.periodic_side(m)
    pb = I.Problem("accelerated", n, n, m, np.array([[0.05]]), nu, g=F, beta=np.zeros(1), phi_ref=np.ones(1),
                   F0=1.0, west=side, east=side, south=side, north=side, phi0=np.ones((m, n, n)),
                   u0=np.zeros((2, n, n)), p0=np.zeros((n, n)), varphi=varphi)
    o = oracle_mod.OracleSim(pb)
    o.step(steps)
    return o


def test_uniform_acceleration_nonequilibrium_stress(oracle_mod):
    """The non-equilibrium momentum flux of Eq. cicihine-1 in a periodic box under a
    uniform force (grad u = 0, u grows by F every step): with varphi = 1 (Case 2)
    sum c c h^ne + (uF + Fu)/2 vanishes, with varphi = 0 (Case 1) sum c c h^ne =
    -(uF + Fu)/omega up to O(|F|^2), in the deviatoric components.  h^ne = h -
    h^eq(p, u) with u and p the moments of the pre-collision populations."""
    nu, F = 0.1, np.array([2e-4, 1e-4])
    w = oracle_mod.fluid_relaxation(nu)
    for steps in (50, 400):
        for varphi in (0.0, 1.0):
            o = _accelerated_box(oracle_mod, varphi, steps, tuple(F), nu)
            M = o.moments()
            _, h, _ = o.state()
            u, p = M[1:3, 0, 0], M[3, 0, 0]
            np.testing.assert_allclose(u, F * steps, rtol=1e-12)  # exact acceleration
            hne = h[:, 0, 0] - oracle_mod.heq(p, u[0], u[1], 1.0)
            Pi = np.einsum("ia,ib,i->ab", Q9, Q9, hne)
            uF = np.outer(u, F) + np.outer(F, u)
            R = Pi + 0.5 * varphi * uF - (varphi - 1.0) / w * uF
            # the deviatoric part (the isotropic part carries the box's O(Ma^2) pressure drift)
            resid = np.array([R[0, 1], R[0, 0] - R[1, 1]])
            bound = 1e-15 if varphi == 1.0 else 10 * float(F @ F)
            assert np.abs(resid).max() < bound, (varphi, steps, resid)
            assert np.abs(uF[0, 1]) > 100 * np.abs(resid).max()


def test_pressure_recovers_appendix_construction(oracle_mod):
    """The pressure of the appendix's derivation: populations built from its premises
    -- h = h^eq(p, u) + h^ne with sum_i h^ne_i = 0, h^ne_0 = (1/omega - 1/2) F_0 (the
    rest direction does not stream), sum_i c_i h^ne_i = -F/2 (Eq. sum-u) -- must
    return p and u exactly for varphi = 0 and 1.  The printed Eq. sum-p (opposite sign,
    no W_0) and the appendix's last line (no W_0) miss by O(u.F) when varphi = 1."""
    r = np.random.default_rng(5)
    nu = 0.07
    w = oracle_mod.fluid_relaxation(nu)
    side = I.periodic_side(1)
    for varphi in (0.0, 1.0):
        for _ in range(3):
            F = r.normal(size=2) * 1e-2
            u, p = r.normal(size=2) * 0.1, float(r.normal()) * 1e-2
            pb = I.Problem("node", 1, 1, 1, np.array([[0.05]]), nu, g=tuple(F), beta=np.zeros(1), phi_ref=np.ones(1),
                           F0=1.0, west=side, east=side, south=side, north=side, phi0=np.ones((1, 1, 1)),
                           u0=np.zeros((2, 1, 1)), p0=np.zeros((1, 1)), varphi=varphi)
            Fi = oracle_mod.force_pop_phi(F, u, varphi)
            ne = np.zeros(9)
            ne[0] = (1.0 / w - 0.5) * Fi[0]
            ne[1:] = r.normal(size=8) * 1e-3
            # impose sum_i ne_i = 0 and sum_i c_i ne_i = -F/2 with the axis directions 1..4
            ne[1:] += -(ne.sum()) / 8.0
            dj = -0.5 * F - Q9.T @ ne
            ne[1] += 0.5 * dj[0]
            ne[3] -= 0.5 * dj[0]
            ne[2] += 0.5 * dj[1]
            ne[4] -= 0.5 * dj[1]
            assert abs(ne.sum()) < 1e-15 and np.abs(Q9.T @ ne + 0.5 * F).max() < 1e-15
            h = oracle_mod.heq(p, u[0], u[1], 1.0) + ne
            f = oracle_mod.feq_scalar(1.0, u[0], u[1]).reshape(1, 5, 1, 1)
            o = oracle_mod.OracleSim(pb)
            o.set_state(f, h.reshape(9, 1, 1), np.zeros((1, 1, 1)))
            M = o.moments()
            np.testing.assert_allclose(M[1:3, 0, 0], u, rtol=0, atol=1e-15)
            assert abs(M[3, 0, 0] - p) < 1e-15, (varphi, M[3, 0, 0] - p)


def test_auxiliary_source_moments(oracle_mod):
    """Eq. moment + Case 2: sum_i G_i = 0 and sum_i c_i G_{i,a} = (I - omega/2)(u S + phi F)."""
    r = _rng(3)
    for m in (1, 2, 3):
        A = r.normal(size=(m, m)) * 0.05
        D = A @ A.T + 0.05 * np.eye(m) + 0.02 * r.normal(size=(m, m))  # non-symmetric
        omega = oracle_mod.relaxation_matrix(D)
        phi, S = r.uniform(0.5, 1.5, m), r.normal(size=m) * 1e-3
        u, F = r.normal(size=2) * 0.05, r.normal(size=2) * 1e-4
        G = oracle_mod.aux_source(omega, phi, u, S, F)
        np.testing.assert_allclose(G.sum(axis=1), 0.0, atol=1e-18)
        vec = np.outer(S, u) + np.outer(phi, F)  # (m, 2): u S_b + phi_b F
        expect = (np.eye(m) - 0.5 * omega) @ vec
        np.testing.assert_allclose(G @ Q5, expect, rtol=1e-12, atol=1e-20)


def test_relaxation_matrix_reproduces_diffusion(oracle_mod):
    """Eq. omega-D: D = (omega^-1 - I/2) cs^2 (lambda = I, dt = 1), checked through
    numpy's inverse; and the appendix nu = (1/omega - 1/2) cs^2."""
    r = _rng(4)
    for m in (1, 2, 4, 8):
        D = np.abs(r.normal(size=(m, m))) * 0.02 + np.diag(r.uniform(0.02, 0.5, m))
        omega = oracle_mod.relaxation_matrix(D)
        np.testing.assert_allclose((np.linalg.inv(omega) - 0.5 * np.eye(m)) * CS2, D, rtol=1e-12, atol=1e-15)
    for nu in (0.01, 0.1, 0.25, 2.0):
        w = oracle_mod.fluid_relaxation(nu)
        assert (1 / w - 0.5) * CS2 == pytest.approx(nu, rel=1e-14)


def test_cutoff_forms(oracle_mod):
    """r(c): step form (Sec. 3.1.3) and regularised form (Sec. 3.1.2)."""
    assert oracle_mod.cutoff(0.3, 0.3) == 1.0
    assert oracle_mod.cutoff(0.2999, 0.3) == 0.0
    assert oracle_mod.cutoff(0.3, 0.3, 0.02, True) == pytest.approx(0.5)
    assert oracle_mod.cutoff(1.0, 0.3, 0.02, True) == pytest.approx(1 - 0.5 * (0.02 / 0.7) ** 2 / 2, rel=1e-6)
    assert oracle_mod.cutoff(-1.0, 0.3, 0.02, True) < 1e-4


def test_chemotaxis_and_ddc_closures(oracle_mod):
    """Sec. 3.1: D = [[D_n, -chi n r(c)], [0, D_c]], S = (0, -k n r(c)), F = -g n y;
    Sec. 3.2: F = g (T + Nc C) y."""
    pb = I.chemotaxis_plume(64, 32)
    D, S, F = oracle_mod.closures(pb, np.array([1.3, 0.8]))
    np.testing.assert_allclose(D, [[0.05, -pb.chi * 1.3], [0.0, 0.25]], rtol=1e-15)
    np.testing.assert_allclose(S, [0.0, -pb.k * 1.3], rtol=1e-15)
    np.testing.assert_allclose(F, [0.0, -pb.beta[0] * 1.3], rtol=1e-15)
    D, S, F = oracle_mod.closures(pb, np.array([1.3, 0.2]))  # below c*: r = 0
    np.testing.assert_allclose(D, np.diag([0.05, 0.25]))
    assert S[1] == 0.0
    dd = I.ddc_cavity(64, Nc=-2.0)
    D, S, F = oracle_mod.closures(dd, np.array([0.7, 0.4]))
    np.testing.assert_allclose(F, [0.0, dd.beta[0] * (0.7 - 2.0 * 0.4)], rtol=1e-14)
    np.testing.assert_allclose(D, dd.D)


# ---------------------------------------------------------------------------
# P2: exact linear amplification of a Fourier mode, and its continuum limit
# ---------------------------------------------------------------------------
def _mode_map(z, m, kvec, omega, L, u, F):
    """One step of the scalar update for the Fourier amplitude of a mode
    e^{i k.x} on a periodic lattice with uniform velocity u and uniform force F,
    written in Fourier space from Eqs. evolution12, feq-phi, source, Gi and the
    backward difference of D S.  z = [a_{a,i} (m*5), S_prev (m)]."""
    a = z[: 5 * m].reshape(m, 5)
    sp = z[5 * m:]
    phi = a.sum(axis=1)
    S = L @ phi
    cu = Q5 @ u
    cF = Q5 @ F
    feq = np.outer(phi, W5 * (1 + cu / CS2))
    J = (np.eye(m) - 0.5 * omega)
    G = (J @ (np.outer(S, cu) + np.outer(phi, cF))) * W5 / CS2
    post = a - omega @ (a - feq) + np.outer(S, W5) + G + 0.5 * np.outer(S - sp, W5)
    shift = np.exp(-1j * (Q5 @ kvec))
    return np.concatenate([(post * shift).ravel(), S])


def _mode_amplitude(f, kvec):
    """Complex amplitude a of f = mean + Re[a e^{i k.x}] over the lattice."""
    ny, nx = f.shape[-2:]
    y, x = np.mgrid[0:ny, 0:nx]
    ph = np.exp(-1j * (kvec[0] * x + kvec[1] * y))
    return 2.0 * (f * ph).sum(axis=(-2, -1)) / (nx * ny)


@pytest.mark.parametrize("case", ["diffusion", "advection_source", "force"])
def test_fourier_mode_exact_amplification(oracle_mod, case):
    """The scheme is linear and translation invariant for constant D, uniform flow,
    a linear source and a uniform force, so a Fourier mode evolves exactly by the
    per-step amplification map; the oracle must follow it to round-off."""
    nx, ny, m = 16, 8, 2
    D = np.array([[0.05, 0.02], [0.004, 0.03]])  # non-symmetric on purpose
    kw = dict(mode=(1, 1), amp=(0.01, 0.02))
    if case == "diffusion":
        pb = I.fourier_box(nx, ny, m, D, **kw)
    elif case == "advection_source":
        pb = I.fourier_box(nx, ny, m, D, u=(0.03, -0.02), skind="consumption", k=2e-3, **kw)
    else:
        pb = I.fourier_box(nx, ny, m, D, u=(0.01, 0.02), skind="consumption", k=2e-3,
                           g=(0.6, -0.8), F0=2e-5, **kw)
    s = oracle_mod.OracleSim(pb)
    kvec = 2 * math.pi * np.array([1 / nx, 1 / ny])
    omega = np.linalg.inv(D / CS2 + 0.5 * np.eye(m))
    L = np.zeros((m, m))
    if pb.skind == "consumption":
        L[1, 0] = -pb.k  # S_1 = -k phi_0 (r = 1: c stays near 1)
    u0 = np.array([pb.u0[0, 0, 0], pb.u0[1, 0, 0]])
    F = np.array(pb.g) * pb.F0
    amp = np.array([0.01, 0.02])
    a0 = np.outer(amp, W5 * (1 + (Q5 @ u0) / CS2))
    z = np.concatenate([a0.ravel(), L @ amp]).astype(complex)
    steps = 40
    for t in range(steps):
        z = _mode_map(z, m, kvec, omega, L, u0 + F * t, F)
    s.step(steps)
    f, h, sp = s.state()
    got = _mode_amplitude(f.reshape(m * 5, ny, nx), kvec)
    np.testing.assert_allclose(got, z[: 5 * m], rtol=0, atol=1e-15)
    np.testing.assert_allclose(_mode_amplitude(sp, kvec), z[5 * m:], rtol=0, atol=1e-16)
    # the uniform fluid accelerates exactly by F per step
    M = s.moments()
    np.testing.assert_allclose(M[m:m + 2].reshape(2, -1).mean(axis=1), u0 + F * steps, rtol=1e-12, atol=1e-17)


def test_fourier_mode_continuum_limit(oracle_mod):
    """Continuum limit: a mode along an eigenvector v_j of D decays at rate
    lambda_j |k|^2 (Eq. CDE with u = 0, S = 0), with O(k^2) relative error."""
    D = np.array([[0.05, 0.01], [0.005, 0.03]])
    lam, V = np.linalg.eig(D)  # real spectrum for this D
    lam, V = lam.real, V.real
    Winv = np.linalg.inv(V)
    errs = []
    for nx in (32, 64):
        k = 2 * math.pi / nx
        rates = []
        for j in range(2):
            phi0 = 1.0 + 0.01 * V[:, j][:, None, None] * np.cos(k * np.arange(nx))[None, None, :]
            pb = I.fourier_box(nx, 1, 2, D).replace(phi0=phi0)
            s = oracle_mod.OracleSim(pb)
            n = int(0.5 / (lam[j] * k * k))
            s.step(n)
            ph = _mode_amplitude(s.moments()[:2], np.array([k, 0.0]))
            proj = np.real(Winv @ ph)[j] / 0.01
            rates.append(-math.log(proj) / (n * k * k))
        errs.append((np.abs(np.array(rates) - lam) / lam).max())
    assert errs[1] < 3e-3  # measured 2.3e-3 at k = 2 pi / 64
    assert 3.8 < errs[0] / errs[1] < 4.2  # second order in k


# ---------------------------------------------------------------------------
# P3: Taylor-Green vortex decay (fluid part)
# ---------------------------------------------------------------------------
def test_taylor_green_decay(oracle_mod):
    """u(t) = u(0) exp(-nu (kx^2 + ky^2) t) for the incompressible NS equations
    the appendix recovers; 64^2, nu = 0.1, u0 = 0.02, 1000 steps."""
    pb = I.cross_diffusion_taylor_green()
    s = oracle_mod.OracleSim(pb)
    s.step(1000)
    M = s.moments()
    k2 = 2 * (2 * math.pi / 64) ** 2
    ue = pb.u0 * math.exp(-pb.nu * k2 * 1000)
    err = np.linalg.norm(M[2:4] - ue) / np.linalg.norm(ue)
    assert err < 3e-3  # O(Ma^2) + O(k^2)
    rate = -math.log(np.sum(M[2:4] * pb.u0) / np.sum(pb.u0 ** 2)) / 1000
    assert rate == pytest.approx(pb.nu * k2, rel=2e-3)


# ---------------------------------------------------------------------------
# P4: steady chemotaxis closed form (Sec. 3.1.1)
# ---------------------------------------------------------------------------
def _run_to_rest(s, chunk, tol, max_chunks):
    prev = s.moments()
    for _ in range(max_chunks):
        s.step(chunk)
        cur = s.moments()
        if np.abs(cur - prev).max() <= tol * max(np.abs(cur).max(), 1e-300):
            return cur
        prev = cur
    raise AssertionError("no steady state")


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        return json.load(fh)


def test_chemotaxis_steady_closed_form(oracle_mod):
    """n^s = (delta A^2 / beta)(alpha/2) / cos^2(alpha A y / 2),
    c^s = 1 - (2/alpha) ln(cos(alpha A y/2) / cos(alpha A/2)), A = pi/20 for
    alpha = beta = 10, delta = 5, n0 = pi/40 (printed values, tests/golden);
    second-order convergence in H."""
    gd = _golden("chemotaxis_steady_sec3_1_1.json")
    al, be, de = gd["alpha"], gd["beta"], gd["delta"]
    A = eval(gd["A"], {"pi": math.pi})
    n0 = eval(gd["n0"], {"pi": math.pi})
    assert be * n0 == pytest.approx(de * A * math.tan(al * A / 2), rel=1e-14)  # Eq. A-relationship
    errs = []
    for ny in (25, 50):
        pb = I.chemotaxis_steady_strip(ny=ny, nx=1, Dn=0.2, alpha=al, beta=be, delta=de, n0=n0)
        s = oracle_mod.OracleSim(pb)
        M = _run_to_rest(s, 500, 1e-13, 400)
        y = (np.arange(ny) + 0.5) / ny
        ns = de * A * A / be * al / 2 / np.cos(al / 2 * A * y) ** 2
        cs = 1 - 2 / al * np.log(np.cos(al / 2 * A * y) / math.cos(al / 2 * A))
        en = np.linalg.norm(M[0, :, 0] - ns) / np.linalg.norm(ns)
        ec = np.linalg.norm(M[1, :, 0] - cs) / np.linalg.norm(cs)
        errs.append(max(en, ec))
        assert np.sum(M[0]) == pytest.approx(ny * n0, rel=1e-11)  # bacteria conserved
    assert errs[1] < 6e-4
    assert 3.5 < errs[0] / errs[1] < 4.5


# ---------------------------------------------------------------------------
# P5: exact mass conservation
# ---------------------------------------------------------------------------
def test_mass_conservation_periodic_and_walled(oracle_mod):
    pb = I.cross_diffusion_taylor_green(32, 32)
    s = oracle_mod.OracleSim(pb)
    m0 = s.moments()[:2].sum(axis=(1, 2))
    s.step(500)
    np.testing.assert_allclose(s.moments()[:2].sum(axis=(1, 2)), m0, rtol=1e-13)
    # closed no-flux box with chemotaxis, gravity and free slip; no source, no Dirichlet
    wb = I.chemotaxis_plume(24, 16)
    wb = wb.replace(skind="none", north=I.wall_side(2, I.FREESLIP), beta=np.array([1e-4, 0.0]))
    s = oracle_mod.OracleSim(wb)
    m0 = s.moments()[:2].sum(axis=(1, 2))
    s.step(500)
    np.testing.assert_allclose(s.moments()[:2].sum(axis=(1, 2)), m0, rtol=1e-13)


# ---------------------------------------------------------------------------
# P6: reductions to textbook cases
# ---------------------------------------------------------------------------
def test_single_scalar_is_textbook_bgk_advection_diffusion(oracle_mod):
    """m = 1, constant D: the D2Q5 BGK advection-diffusion scheme,
    f_i(x + c_i, t + 1) = f_i - (f_i - W_i phi (1 + 3 c_i.u)) / tau, tau = 3 D + 1/2,
    written here separately with numpy rolls on a periodic box."""
    nx, ny, Dv = 12, 10, 0.07
    u = np.array([0.04, -0.03])
    phi0 = 1 + 0.1 * (2 * I.uniform(5, np.arange(nx * ny)) - 1).reshape(1, ny, nx)
    pb = I.fourier_box(nx, ny, 1, [[Dv]], u=tuple(u)).replace(phi0=phi0)
    s = oracle_mod.OracleSim(pb)
    s.step(30)
    tau = 3 * Dv + 0.5
    f = W5[:, None, None] * phi0[0][None] * (1 + 3 * (Q5 @ u))[:, None, None]
    for _ in range(30):
        phi = f.sum(axis=0)
        feq = W5[:, None, None] * phi[None] * (1 + 3 * (Q5 @ u))[:, None, None]
        post = f - (f - feq) / tau
        f = np.stack([np.roll(post[i], shift=(Q5[i, 1], Q5[i, 0]), axis=(0, 1)) for i in range(5)])
    np.testing.assert_allclose(s.state()[0][0], f, rtol=1e-13, atol=1e-15)


def test_diagonal_d_decouples_and_permutation_permutes(oracle_mod):
    pb = I.cross_diffusion_taylor_green(16, 16, D=((0.05, 0.0), (0.0, 0.03)))
    s = oracle_mod.OracleSim(pb)
    s.step(50)
    M = s.moments()
    for a in range(2):
        single = I.Problem("one", 16, 16, 1, [[pb.D[a, a]]], pb.nu, phi0=pb.phi0[a:a + 1], u0=pb.u0, p0=pb.p0)
        s1 = oracle_mod.OracleSim(single)
        s1.step(50)
        M1 = s1.moments()
        assert np.array_equal(M1[0], M[a])  # bitwise: same arithmetic per scalar
        assert np.array_equal(M1[1:], M[2:])
    full = I.cross_diffusion_taylor_green(16, 16)
    perm = full.replace(D=full.D[::-1, ::-1].copy(), phi0=full.phi0[::-1].copy())
    sa, sb = oracle_mod.OracleSim(full), oracle_mod.OracleSim(perm)
    sa.step(50)
    sb.step(50)
    np.testing.assert_allclose(sb.moments()[:2][::-1], sa.moments()[:2], rtol=1e-13)


# ---------------------------------------------------------------------------
# Boundary closed forms: bounce-back, anti-bounce-back, free slip, pressure
# ---------------------------------------------------------------------------
NU_MAGIC = math.sqrt(3.0 / 16.0) / 3.0  # tau = 1/2 + sqrt(3/16): BGK bounce-back wall exactly half-way


def _channel(ny, nu, top):
    m = 2
    return I.Problem("channel", 1, ny, m, np.diag([0.1, 0.1]), nu, g=(1.0, 0.0), F0=1e-6,
                     south=I.wall_side(m), north=top)


def test_poiseuille_no_slip_bounce_back(oracle_mod):
    """Half-way bounce-back with the force term: u(y) = F y (H - y) / (2 nu), exact at
    the magic relaxation time and second-order convergent otherwise."""
    ny = 16
    s = oracle_mod.OracleSim(_channel(ny, NU_MAGIC, I.wall_side(2)))
    M = _run_to_rest(s, 500, 1e-14, 100)
    y = np.arange(ny) + 0.5
    ue = 1e-6 / (2 * NU_MAGIC) * y * (ny - y)
    np.testing.assert_allclose(M[2, :, 0], ue, rtol=1e-9)
    assert np.abs(M[3]).max() < 1e-16
    e = []
    for ny in (8, 16):
        s = oracle_mod.OracleSim(_channel(ny, 0.1, I.wall_side(2)))
        M = _run_to_rest(s, 500, 1e-14, 200)
        y = np.arange(ny) + 0.5
        ue = 1e-6 / 0.2 * y * (ny - y)
        e.append(np.linalg.norm(M[2, :, 0] - ue) / np.linalg.norm(ue))
    assert 3.8 < e[0] / e[1] < 4.2


def test_free_slip_half_channel(oracle_mod):
    """Specular reflection at the top: u(y) = F y (2H - y) / (2 nu), zero shear at the top."""
    ny = 16
    s = oracle_mod.OracleSim(_channel(ny, NU_MAGIC, I.wall_side(2, I.FREESLIP)))
    M = _run_to_rest(s, 1000, 1e-14, 100)
    y = np.arange(ny) + 0.5
    ue = 1e-6 / (2 * NU_MAGIC) * y * (2 * ny - y)
    np.testing.assert_allclose(M[2, :, 0], ue, rtol=1e-8)


def test_anti_bounce_back_linear_profile(oracle_mod):
    """Anti-bounce-back Dirichlet walls with cross diffusion: the steady solution of
    div(D grad phi) = 0 with phi = 1 at x = 0 and 0 at x = L is linear in each
    scalar and reproduced to round-off, walls half-way outside the end nodes."""
    nx, m = 12, 2
    hot = I.wall_side(m, I.NOSLIP, [I.DIRICHLET] * 2, [1.0, 1.0])
    cold = I.wall_side(m, I.NOSLIP, [I.DIRICHLET] * 2, [0.0, 0.0])
    pb = I.Problem("cond", nx, 1, m, np.array([[0.2, 0.05], [0.03, 0.1]]), 0.1, west=hot, east=cold,
                   phi0=np.zeros((2, 1, nx)))
    s = oracle_mod.OracleSim(pb)
    M = _run_to_rest(s, 500, 1e-15, 200)
    pe = 1 - (np.arange(nx) + 0.5) / nx
    np.testing.assert_allclose(M[0, 0], pe, atol=1e-13)
    np.testing.assert_allclose(M[1, 0], pe, atol=1e-13)


def test_hydrostatic_pressure(oracle_mod):
    """Closed box, uniform n, force -g n y: rest with dp/dy = F_y (Eq. sum-p)."""
    m, g = 2, 1e-5
    pb = I.Problem("hydro", 8, 16, m, np.diag([0.1, 0.1]), 0.1, g=(0.0, -1.0), beta=np.array([g, 0.0]),
                   west=I.wall_side(m), east=I.wall_side(m), south=I.wall_side(m),
                   north=I.wall_side(m, I.FREESLIP))
    s = oracle_mod.OracleSim(pb)
    M = _run_to_rest(s, 500, 1e-13, 100)
    assert np.abs(M[2:4]).max() < 1e-11
    dp = np.diff(M[4], axis=0)
    assert dp.mean() == pytest.approx(-g, rel=1e-6)
    np.testing.assert_allclose(dp, -g, rtol=1e-3)  # wall rows deviate by ~2e-4


# ---------------------------------------------------------------------------
# P7: symmetry of the double-diffusive cavity
# ---------------------------------------------------------------------------
def test_ddc_cavity_centro_symmetry(oracle_mod):
    """With T, C measured from the mean wall value (walls at +1/2 and -1/2, F =
    g (T + Nc C)), a 180-degree rotation with phi -> -phi, u -> -u maps every
    term of Eqs. evolution12/evolution3 (including G = phi F) and every boundary
    rule onto itself, so the solution stays centro-symmetric to round-off."""
    pb = I.ddc_cavity(24, Ra=1e4, Pr=0.7, Le=2.0, Nc=1.0, Df=0.1, Sr=0.1)
    hot = I.wall_side(2, I.NOSLIP, [I.DIRICHLET] * 2, [0.5, 0.5])
    cold = I.wall_side(2, I.NOSLIP, [I.DIRICHLET] * 2, [-0.5, -0.5])
    pb = pb.replace(west=hot, east=cold)
    s = oracle_mod.OracleSim(pb)
    s.step(3000)
    M = s.moments()
    rot = M[:, ::-1, ::-1]
    umax = np.abs(M[2:4]).max()
    assert umax > 1e-3  # the cavity convects
    np.testing.assert_allclose(M[:2], -rot[:2], atol=1e-12)
    np.testing.assert_allclose(M[2:4], -rot[2:4], atol=1e-11 * umax)
    np.testing.assert_allclose(M[4], rot[4], atol=1e-12)


def test_initial_moments_reproduce_inputs(oracle_mod):
    """Eq. heq read through Eq. sum-phi/u/p: the initial populations built from
    (phi0, u0, p0) return exactly those moments, with a density-dependent force."""
    pb = I.cross_diffusion_taylor_green(16, 12).replace(g=(0.3, -1.0), beta=np.array([2e-4, -1e-4]))
    s = oracle_mod.OracleSim(pb)
    M = s.moments()
    np.testing.assert_allclose(M[:2], pb.phi0, rtol=1e-15)
    np.testing.assert_allclose(M[2:4], pb.u0, atol=1e-17)
    np.testing.assert_allclose(M[4], pb.p0, atol=1e-17)


# ---------------------------------------------------------------------------
# P9: Case 1 of Sec. 2.1 -- convection cross-diffusion in a prescribed velocity
# ---------------------------------------------------------------------------
def _case1_mode_rates(oracle_mod, N, U, j):
    """Advect the j-th eigenmode of D, phi = 1 + 1e-3 v_j cos(k x), k = 2 pi / N, by
    a uniform prescribed velocity U along x; return (lambda_j, fitted decay rate
    / k^2, fitted phase speed) over steps 4N .. 24N."""
    D = np.array([[0.05, 0.01], [0.005, 0.03]])
    lam, V = np.linalg.eig(D)
    order = np.argsort(lam.real)
    lam, V = lam.real[order], V.real[:, order]
    left = np.linalg.inv(V)
    k = 2 * math.pi / N
    x = np.arange(N)
    phi0 = 1.0 + 1e-3 * V[:, j][:, None, None] * np.cos(k * x)[None, None, :]
    pb = I.fourier_box(N, 1, 2, D, u=(U, 0.0)).replace(case1=True, phi0=phi0)
    s = oracle_mod.OracleSim(pb)
    ts, cs = [], []
    s.step(4 * N)
    for t in range(4 * N, 24 * N + 1, N // 16):
        if t > 4 * N:
            s.step(N // 16)
        ph = (2.0 / N) * (s.moments()[:2, 0, :] * np.exp(-1j * k * x)[None, :]).sum(axis=1)
        ts.append(t)
        cs.append(left[j] @ ph)
    cs = np.array(cs)
    rate = -np.polyfit(ts, np.log(np.abs(cs)), 1)[0] / k ** 2
    speed = -np.polyfit(ts, np.unwrap(np.angle(cs)), 1)[0] / k
    return lam[j], rate, speed


def test_case1_advected_mode_decays_with_d(oracle_mod):
    """Case 1 with the auxiliary source G = (I - omega/2) W_i c_i.d_t(phi u)/cs^2:
    an eigenmode of D advected at U = 0.2 decays at eig(D) k^2 and moves at U,
    with second-order convergence (error ratio ~4 from N = 64 to 128).  Without G
    the scheme's convective numerical diffusion would lower the rate by
    (omega^-1 - 1/2) U^2, i.e. by 3 U^2 = 12 % here."""
    for j in (0, 1):
        lam, r64, c64 = _case1_mode_rates(oracle_mod, 64, 0.2, j)
        _, r128, c128 = _case1_mode_rates(oracle_mod, 128, 0.2, j)
        e64, e128 = abs(r64 / lam - 1), abs(r128 / lam - 1)
        assert e64 < 1.5e-3 and e128 < 4e-4, (j, e64, e128)
        assert 3.0 < e64 / e128 < 5.0, (j, e64, e128)
        assert abs(c64 / 0.2 - 1) < 5e-4 and abs(c128 / 0.2 - 1) < 2e-4


def test_case1_conserves_mass_in_cellular_flow(oracle_mod):
    """sum_i G_{i,a} = 0 and the collision conserves phi: in a periodic
    divergence-free cellular flow the scalar totals stay constant to round-off,
    and the reported velocity is the prescribed one."""
    pb = I.cde_cellular(32, 24, walls=False, U0=0.08)
    s = oracle_mod.OracleSim(pb)
    a = s.moments()[:2].sum(axis=(1, 2))
    s.step(400)
    M = s.moments()
    assert np.abs(M[:2].sum(axis=(1, 2)) / a - 1).max() < 1e-13
    np.testing.assert_array_equal(M[2:4], pb.u0)
    assert M[:2].std() < 0.5 * pb.phi0.std()  # it mixes


# ---------------------------------------------------------------------------
# The pins catch planted mistakes
# ---------------------------------------------------------------------------
PLANTED = [
    ("drop auxiliary source G", "+ Si + G[a * 5 + i] +", "+ Si +"),
    ("flip sign of omega/2 in G", "(a == b ? 1.0 : 0.0) - 0.5 * omega[a * m + b]",
     "(a == b ? 1.0 : 0.0) + 0.5 * omega[a * m + b]"),
    ("transpose omega in collision", "coll += omega[a * m + b] * (f[b * 5 + i]", "coll += omega[b * m + a] * (f[b * 5 + i]"),
    ("drop time-derivative of S", "+ 0.5 * (Si - Si_prev)", ""),
    ("never update S(t-1)", "for (int a = 0; a < m; ++a) sp[a] = S[a];", ";"),
    ("force weight (1 - omega/2) dropped", "(1.0 - 0.5 * omega_f) * Fi[i]", "Fi[i]"),
    ("no half force in velocity", "u[0] = jx + 0.5 * F[0];", "u[0] = jx;"),
    ("pressure W0 term dropped", "(sum_nonrest - Q9_W[0] * uu / (2.0 * CS2))", "(sum_nonrest - uu / (2.0 * CS2))"),
    ("omega from D without 1/cs^2", "D[a * m + b] / CS2 + (a == b ? 0.5 : 0.0)", "D[a * m + b] + (a == b ? 0.5 : 0.0)"),
    ("sigma_0 without 1/cs^2", "(Q9_W[0] - 1.0) * p / CS2 + rho0", "(Q9_W[0] - 1.0) * p + rho0"),
    ("f^eq velocity sign", "(phi + cu * phi / CS2", "(phi - cu * phi / CS2"),
    ("chemotaxis sign", "D[0 * m + 1] += -P->chi", "D[0 * m + 1] += P->chi"),
    ("consumption uses wrong scalar", "S[1] = -P->k * phi[0] * r", "S[1] = -P->k * phi[1] * r"),
    ("scalar streams backwards in y", "int tx = x + Q5_CX[i], ty = y + Q5_CY[i];",
     "int tx = x + Q5_CX[i], ty = y - Q5_CY[i];"),
    ("fluid relaxation from nu off", "1.0 / (nu / CS2 + 0.5)", "1.0 / (nu / CS2 + 1.0)"),
    ("anti-bounce-back sign", "= -v + 2.0 * Q5_W[i] * P->value[side][a]", "= v + 2.0 * Q5_W[i] * P->value[side][a]"),
    ("free slip reflects both components", "int j = q9_dir(Q9_CX[i], -Q9_CY[i]);", "int j = q9_dir(-Q9_CX[i], -Q9_CY[i]);"),
    ("no half force at initialisation", "heq[i] - 0.5 * Fi[i]", "heq[i]"),
    ("bounce-back of scalars lands on wrong direction", "s->fnew[(node * m + a) * 5 + io] = v;",
     "s->fnew[(node * m + a) * 5 + i] = v;"),
    ("Case 1: G from phi instead of its time difference", "double dphi = phi[b] - phi_prev[b];",
     "double dphi = phi[b];"),
    ("Case 1: phi(t-1) never updated", "for (int a = 0; a < m; ++a) s->phiprev[node * m + a] = phi[a];", ";"),
    ("Case 1: sign of omega/2 in G", "a == b ? 1.0 - 0.5 * omega[a * m + b] : -0.5 * omega[a * m + b]",
     "a == b ? 1.0 + 0.5 * omega[a * m + b] : 0.5 * omega[a * m + b]"),
    ("varphi part of the force dropped", "varphi * uFFu_cc / (2.0 * CS2 * CS2)", "0.0 * uFFu_cc"),
    ("varphi part of the force without its trace term", "2.0 * cu * cF - 2.0 * CS2 * (ux * Fx + uy * Fy)",
     "2.0 * cu * cF"),
    ("pressure varphi term with the sign of Eq. sum-p", "- Q9_W[0] * P->varphi * (1.0 / omega_f - 0.5)",
     "+ P->varphi * (1.0 / omega_f - 0.5)"),
    ("pressure varphi term without W_0", "- Q9_W[0] * P->varphi * (1.0 / omega_f - 0.5)",
     "- P->varphi * (1.0 / omega_f - 0.5)"),
    ("varphi force ignores the velocity", "orc_force_pop_phi(F[0], F[1], u[0], u[1], P->varphi, Fi);",
     "orc_force_pop_phi(F[0], F[1], 0.0, 0.0, P->varphi, Fi);"),
]


def _pin_calls():
    import sys
    mod = sys.modules[__name__]
    calls = [lambda o, c=c: test_fourier_mode_exact_amplification(o, c)
             for c in ("diffusion", "advection_source", "force")]
    names = [n for n in dir(mod) if n.startswith("test_") and n not in
             ("test_planted_mistakes_are_caught", "test_fourier_mode_exact_amplification")]
    calls += [getattr(mod, n) for n in names]
    return calls


@pytest.mark.parametrize("name,old,new", PLANTED, ids=[p[0] for p in PLANTED])
def test_planted_mistakes_are_caught(oracle_mod, tmp_path, name, old, new):
    """Build a copy of the oracle with one plausible mistake and check that at
    least one pin above fails on it."""
    src = oracle_mod.source_text()
    assert src.count(old) == 1, name
    path = oracle_mod.compile_source(src.replace(old, new), str(tmp_path / "mutant.so"))
    mutant = oracle_mod.Binding(path)
    for call in _pin_calls():
        try:
            call(mutant)
        except (AssertionError, FloatingPointError, ValueError, np.linalg.LinAlgError):
            return
    pytest.fail(f"no pin caught the planted mistake: {name}")
