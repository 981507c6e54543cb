"""Seeded synthetic inputs: problem descriptions and initial moment fields.

This module is shared by the CUDA path, the tests and the benchmark.  It holds
no lattice Boltzmann arithmetic: it only draws random numbers and states the
problems (grid, lattice-unit coefficients, boundary kinds, initial moments).
Each side (the CUDA library and the CPU oracle) turns a `Problem` into its own
parameters and its own initial populations.

Random numbers come from a counter-based generator, SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
value for (seed, index) is the SplitMix64 output function applied to
seed * G2 + (index + 1) * G1, G1 = 0x9E3779B97F4A7C15 (the golden-ratio
increment) and G2 = 0xD1B54A32D192ED03.  Uniforms use the top 53 bits; normals
use the Box-Muller transform on the uniform pair (2 idx, 2 idx + 1).

Problems (lattice units, dx = dt = 1; node (i, j) of a walled axis sits half a
spacing inside the wall):
  * `cross_diffusion_taylor_green` -- 2D periodic box, m = 2, constant D,
    Taylor-Green vortex, scalars 1 + 0.1 U(-1, 1).
  * `chemotaxis_plume`  -- bacteria n and oxygen c (Sec. 3.1): no-slip side and
    bottom walls, free-slip top with c = 1, chemotactic cross term
    D_01 = -chi n r(c), consumption S_c = -k n r(c), force -g n along y,
    n0 = 1 + 0.01 N(0, 1).
  * `ddc_cavity` -- double-diffusive convection with Soret and Dufour terms
    (Sec. 3.2): T = C = 1 on the west wall, 0 on the east wall, adiabatic top
    and bottom, no slip everywhere, D = alpha [[1, Df], [Sr/Le, 1/Le]],
    F = g (T + N C) along y.
  * `chemotaxis_plume_regularised` -- the Sec. 3.1.2 example: regularised
    cut-off, periodic sides, large Sc, n0 = 1 / 0.5 across a perturbed interface.
  * `chemotaxis_steady_strip` -- the x-homogeneous steady chemotaxis test of
    Sec. 3.1.1 on a periodic strip.
  * `fourier_box` -- periodic box with uniform flow and a single Fourier mode in
    the scalars, for the exact linear-amplification pins.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)
_G1 = np.uint64(0x9E3779B97F4A7C15)
_G2 = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index) -> np.ndarray:
    """SplitMix64 output for counters `index` (array-like of non-negative ints)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * _G2 + (idx + np.uint64(1)) * _G1
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, index) -> np.ndarray:
    """U[0, 1) doubles, one per counter."""
    return (splitmix64(seed, index) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, index) -> np.ndarray:
    """N(0, 1) doubles by Box-Muller on the uniform pair (2 idx, 2 idx + 1)."""
    idx = np.asarray(index, dtype=np.uint64)
    u1 = 1.0 - uniform(seed, idx * np.uint64(2))  # (0, 1]
    u2 = uniform(seed, idx * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# problem description
# ----------------------------------------------------------------------------
PERIODIC, WALL = "periodic", "wall"
NOSLIP, FREESLIP = "noslip", "freeslip"
NOFLUX, DIRICHLET = "noflux", "dirichlet"


@dataclass
class Side:
    kind: str = PERIODIC          # PERIODIC or WALL
    fluid: str = NOSLIP           # NOSLIP or FREESLIP (walls only)
    scalar: List[str] = field(default_factory=list)   # per scalar: NOFLUX / DIRICHLET
    value: List[float] = field(default_factory=list)  # per scalar Dirichlet value


def periodic_side(m: int) -> Side:
    return Side(PERIODIC, NOSLIP, [NOFLUX] * m, [0.0] * m)


def wall_side(m: int, fluid: str = NOSLIP, scalar=None, value=None) -> Side:
    return Side(WALL, fluid, list(scalar or [NOFLUX] * m), list(value or [0.0] * m))


@dataclass
class Problem:
    """A CDF problem in lattice units plus its initial moments."""
    name: str
    nx: int
    ny: int
    m: int
    D: np.ndarray                      # (m, m) constant part of the diffusion matrix
    nu: float
    dkind: str = "const"               # "const" | "chemotaxis"
    chi: float = 0.0                   # chemotaxis: D_01 += -chi phi_0 r(phi_1)
    c_star: float = 0.3
    eps: float = 0.0
    r_regularised: bool = False
    skind: str = "none"                # "none" | "const" | "consumption"
    S: np.ndarray = None               # (m,) constant source
    k: float = 0.0                     # consumption: S_1 = -k phi_0 r(phi_1)
    g: tuple = (0.0, 0.0)              # F = g (F0 + sum_a beta_a (phi_a - phi_ref_a))
    beta: np.ndarray = None
    phi_ref: np.ndarray = None
    F0: float = 0.0
    rho0: float = 1.0
    west: Side = None
    east: Side = None
    south: Side = None
    north: Side = None
    phi0: np.ndarray = None            # (m, ny, nx)
    u0: np.ndarray = None              # (2, ny, nx)
    p0: np.ndarray = None              # (ny, nx)
    steps: int = 0                     # nominal step count of the workload
    case1: bool = False                # Case 1 of Sec. 2.1: no fluid; u0 is a steady prescribed velocity
    varphi: float = 0.0                # second-order part of Eq. force (0: the paper's experiments, 1: Case 2)

    def __post_init__(self):
        m = self.m
        self.D = np.asarray(self.D, dtype=np.float64).reshape(m, m)
        self.S = np.zeros(m) if self.S is None else np.asarray(self.S, np.float64)
        self.beta = np.zeros(m) if self.beta is None else np.asarray(self.beta, np.float64)
        self.phi_ref = np.zeros(m) if self.phi_ref is None else np.asarray(self.phi_ref, np.float64)
        for s in ("west", "east", "south", "north"):
            if getattr(self, s) is None:
                setattr(self, s, periodic_side(m))
        if self.phi0 is None:
            self.phi0 = np.ones((m, self.ny, self.nx))
        if self.u0 is None:
            self.u0 = np.zeros((2, self.ny, self.nx))
        if self.p0 is None:
            self.p0 = np.zeros((self.ny, self.nx))

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def node_coords(n: int, walled: bool) -> np.ndarray:
    """Node positions along one axis in lattice units: i + 1/2 between walls, i if periodic."""
    return np.arange(n, dtype=np.float64) + (0.5 if walled else 0.0)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def cross_diffusion_taylor_green(nx: int = 64, ny: int = 64, seed: int = 0, u0: float = 0.02,
                                 D=((0.05, 0.01), (0.005, 0.03)), nu: float = 0.1,
                                 steps: int = 1000) -> Problem:
    """Periodic box, m = 2, constant cross-diffusion D, Taylor-Green vortex
    u = (-u0 cos(kx x) sin(ky y), v0 sin(kx x) cos(ky y)), v0 = u0 kx / ky,
    p = -(u0^2 cos(2 kx x) + v0^2 cos(2 ky y)) / 4,
    scalars phi_a = 1 + 0.1 U(-1, 1) with counter a*nx*ny + y*nx + x."""
    m = 2
    x = node_coords(nx, False)[None, :]
    y = node_coords(ny, False)[:, None]
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    v0 = u0 * kx / ky
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = v0 * np.sin(kx * x) * np.cos(ky * y)
    p = -0.25 * (u0 ** 2 * np.cos(2 * kx * x) + v0 ** 2 * np.cos(2 * ky * y))
    idx = np.arange(m * ny * nx, dtype=np.uint64)
    phi = 1.0 + 0.1 * (2.0 * uniform(seed, idx) - 1.0)
    return Problem("cross_diffusion_taylor_green", nx, ny, m, np.array(D), nu,
                   phi0=phi.reshape(m, ny, nx), u0=np.stack([ux, uy]), p0=p, steps=steps)


def chemotaxis_plume(nx: int = 512, ny: int = 256, seed: int = 0, chi: float = 0.5,
                     Dn: float = 0.05, Dc: float = 0.25, nu: float = 0.25,
                     beta: float = 20.0, gamma: float = 2000.0, gravity_scale: float = 1.0,
                     c_star: float = 0.3, steps: int = 200_000) -> Problem:
    """Bacteria-oxygen plume (Sec. 3.1.3 setup on a box): lattice D_n, D_c, nu;
    k = beta D_n / H^2 and g = Sc gamma D_n^2 / H^3 (Sc = nu / D_n) map the
    dimensionless beta, gamma of Sec. 3.1 to lattice units with H = ny."""
    m = 2
    H = float(ny)
    Sc = nu / Dn
    k = beta * Dn / H ** 2
    g = gravity_scale * Sc * gamma * Dn ** 2 / H ** 3
    idx = np.arange(ny * nx, dtype=np.uint64)
    n0 = 1.0 + 0.01 * normal(seed, idx).reshape(ny, nx)
    phi0 = np.stack([n0, np.ones((ny, nx))])
    side = wall_side(m)  # no slip, no flux
    top = wall_side(m, FREESLIP, [NOFLUX, DIRICHLET], [0.0, 1.0])
    return Problem("chemotaxis_plume", nx, ny, m, np.diag([Dn, Dc]), nu, dkind="chemotaxis",
                   chi=chi, c_star=c_star, skind="consumption", k=k, g=(0.0, -1.0),
                   beta=np.array([g, 0.0]), west=side, east=wall_side(m), south=wall_side(m),
                   north=top, phi0=phi0, steps=steps)


def chemotaxis_plume_regularised(nx: int = 512, ny: int = 256, alpha: float = 5.0, beta: float = 5.0,
                                 delta: float = 0.25, gamma: float = 418.0, Sc: float = 7700.0, nu: float = 0.5,
                                 c_star: float = 0.3, steps: int = 200_000) -> Problem:
    """The example of Sec. 3.1.2: alpha = 5, beta = 5, delta = 0.25, gamma = 418,
    Sc = 7700, the regularised cut-off r(c) = (1 + (c - c*)/sqrt((c - c*)^2 + eps^2))/2
    with eps = dx (= 1/H), periodic sides, no-flux no-slip bottom, free-slip top with
    c = 1; n0 = 1 above y = 0.501 - 0.01 sin((x - 0.5) pi), 0.5 below, c0 = 1, u0 = 0
    (x, y scaled by H).  Lattice: nu fixes D_n = nu / Sc (the paper's large Sc
    forces a small D_n, as its dt = 1e-8 does), D_c = delta D_n, chi = alpha D_n,
    k = beta D_n / H^2, g = Sc gamma D_n^2 / H^3 (the mapping of chemotaxis_plume)."""
    m = 2
    H = float(ny)
    Dn = nu / Sc
    k = beta * Dn / H ** 2
    g = Sc * gamma * Dn ** 2 / H ** 3
    x = (np.arange(nx) + 0.5) / H
    y = (np.arange(ny) + 0.5) / H
    X, Y = np.meshgrid(x, y)
    n0 = np.where(Y > 0.501 - 0.01 * np.sin((X - 0.5) * np.pi), 1.0, 0.5)
    phi0 = np.stack([n0, np.ones((ny, nx))])
    top = wall_side(m, FREESLIP, [NOFLUX, DIRICHLET], [0.0, 1.0])
    return Problem("chemotaxis_plume_regularised", nx, ny, m, np.diag([Dn, delta * Dn]), nu, dkind="chemotaxis",
                   chi=alpha * Dn, c_star=c_star, eps=1.0 / H, r_regularised=True, skind="consumption", k=k,
                   g=(0.0, -1.0), beta=np.array([g, 0.0]), west=periodic_side(m), east=periodic_side(m),
                   south=wall_side(m), north=top, phi0=phi0, steps=steps)


def chemotaxis_plume_sweep(count: int = 256, seed: int = 0, wmin: int = 128, wmax: int = 512,
                           hmin: int = 64, hmax: int = 256, steps: int = 50_000):
    """Parameter sweep of plume instances of uneven size: W ~ U{wmin..wmax},
    H ~ U{hmin..hmax}, chi ~ U[0.1, 0.5], D_c ~ U[0.1, 0.3], gravity scale ~
    U[0.5, 2]; instance k draws its parameters from counters 8k..8k+4 of `seed`
    and its initial noise from seed 1000 seed + k + 1."""
    out = []
    for k in range(count):
        u = uniform(seed, np.arange(8 * k, 8 * k + 5))
        nx = wmin + int(u[0] * (wmax - wmin + 1))
        ny = hmin + int(u[1] * (hmax - hmin + 1))
        chi = 0.1 + 0.4 * u[2]
        Dc = 0.1 + 0.2 * u[3]
        gs = 0.5 + 1.5 * u[4]
        out.append(chemotaxis_plume(nx, ny, seed=1000 * seed + k + 1, chi=chi, Dc=Dc, gravity_scale=gs,
                                    steps=steps).replace(name=f"chemotaxis_plume_sweep[{k}]"))
    return out


def ddc_lattice_parameters(L: int, Ra: float, Pr: float, Ma: float = 0.1):
    """Lattice mapping of the dimensionless DDC system (Sec. 3.2): buoyancy velocity
    U = Ma cs, alpha = U L / sqrt(Ra Pr), nu = Pr alpha, buoyancy g = U^2 / L."""
    U = Ma * math.sqrt(1.0 / 3.0)
    alpha = U * L / math.sqrt(Ra * Pr)
    return alpha, Pr * alpha, U * U / L


def ddc_cavity(n: int = 1024, Ra: float = 1e5, Pr: float = 0.7, Le: float = 2.0, Nc: float = 1.0,
               Df: float = 0.1, Sr: float = 0.1, ny: Optional[int] = None, steps: int = 0, Ma: float = 0.1) -> Problem:
    """Square (or n x ny) cavity; dimensionless D = [[1, D_CT], [S_TC/Le, 1/Le]]
    times alpha_lat; F = g (T + Nc C) y_hat; T = C = 0 and u = 0 at t = 0; Ma sets
    the buoyancy velocity of the lattice mapping (ddc_lattice_parameters)."""
    m = 2
    ny = n if ny is None else ny
    alpha, nu, g = ddc_lattice_parameters(n, Ra, Pr, Ma)
    D = alpha * np.array([[1.0, Df], [Sr / Le, 1.0 / Le]])
    hot = wall_side(m, NOSLIP, [DIRICHLET, DIRICHLET], [1.0, 1.0])
    cold = wall_side(m, NOSLIP, [DIRICHLET, DIRICHLET], [0.0, 0.0])
    return Problem("ddc_cavity", n, ny, m, D, nu, g=(0.0, 1.0), beta=np.array([g, g * Nc]),
                   west=hot, east=cold, south=wall_side(m), north=wall_side(m),
                   phi0=np.zeros((m, ny, n)), steps=steps)


def chemotaxis_steady_strip(ny: int = 50, nx: int = 4, alpha: float = 10.0, beta: float = 10.0,
                            delta: float = 5.0, Dn: float = 0.05, n0: float = math.pi / 40,
                            nu: float = 0.1) -> Problem:
    """Sec. 3.1.1: periodic in x, bottom no-flux wall, top with c = 1 and no flux for n,
    r = 1 (c stays above c* = 0.3), no force; dimensionless y in [0, 1] with H = ny.
    Lattice: D_n, D_c = delta D_n, chi = alpha D_n, k = beta D_n / H^2."""
    m = 2
    H = float(ny)
    phi0 = np.stack([np.full((ny, nx), n0), np.ones((ny, nx))])
    top = wall_side(m, FREESLIP, [NOFLUX, DIRICHLET], [0.0, 1.0])
    return Problem("chemotaxis_steady_strip", nx, ny, m, np.diag([Dn, delta * Dn]), nu,
                   dkind="chemotaxis", chi=alpha * Dn, c_star=0.3, skind="consumption",
                   k=beta * Dn / H ** 2, west=periodic_side(m), east=periodic_side(m),
                   south=wall_side(m), north=top, phi0=phi0)


def fourier_box(nx: int, ny: int, m: int, D, mode=(1, 0), amp=(0.01, 0.02), u=(0.0, 0.0),
                nu: float = 0.1, skind: str = "none", S=None, k: float = 0.0,
                g=(0.0, 0.0), F0: float = 0.0) -> Problem:
    """Periodic box with uniform velocity u, phi_a = 1 + amp_a cos(k.x) for the
    integer wave numbers `mode`; used by the linear-amplification pins."""
    x = node_coords(nx, False)[None, :]
    y = node_coords(ny, False)[:, None]
    th = 2 * math.pi * (mode[0] * x / nx + mode[1] * y / ny)
    phi0 = np.stack([1.0 + amp[a % len(amp)] * np.cos(th) for a in range(m)])
    u0 = np.stack([np.full((ny, nx), u[0]), np.full((ny, nx), u[1])])
    return Problem("fourier_box", nx, ny, m, np.asarray(D, np.float64), nu, skind=skind, S=S,
                   k=k, g=tuple(g), F0=F0, phi0=phi0, u0=u0)


def cde_cellular(nx: int, ny: int, m: int = 2, U0: float = 0.05, D=((0.05, 0.01), (0.005, 0.03)),
                 seed: int = 0, walls: bool = True, steps: int = 0) -> Problem:
    """Case 1 of Sec. 2.1 (convection cross-diffusion without the fluid solver) in a
    prescribed steady cellular flow.  Walls: stream function psi = A sin(pi x / W)
    sin(pi y / H) (no normal velocity at the four walls), scalars Dirichlet on
    the west (phi = 1.2) and east (phi = 0.8) walls, no flux on the others.
    Periodic: u = U0 (sin(2 pi x / W) cos(2 pi y / H), -(H/W) cos(2 pi x / W) sin(2 pi y / H)).
    phi_a = 1 + 0.1 U(-1, 1) (seed; counters a * nx * ny + y * nx + x)."""
    x = node_coords(nx, walls)[None, :]
    y = node_coords(ny, walls)[:, None]
    W, H = float(nx), float(ny)
    if walls:
        ux = U0 * np.sin(math.pi * x / W) * np.cos(math.pi * y / H)
        uy = -U0 * (H / W) * np.cos(math.pi * x / W) * np.sin(math.pi * y / H)
        hot = wall_side(m, NOSLIP, [DIRICHLET] * m, [1.2] * m)
        cold = wall_side(m, NOSLIP, [DIRICHLET] * m, [0.8] * m)
        sides = dict(west=hot, east=cold, south=wall_side(m), north=wall_side(m))
    else:
        ux = U0 * np.sin(2 * math.pi * x / W) * np.cos(2 * math.pi * y / H)
        uy = -U0 * (H / W) * np.cos(2 * math.pi * x / W) * np.sin(2 * math.pi * y / H)
        sides = {}
    u0 = np.stack([np.broadcast_to(ux, (ny, nx)), np.broadcast_to(uy, (ny, nx))]).astype(np.float64)
    phi0 = 1.0 + 0.1 * (2.0 * uniform(seed, np.arange(m * nx * ny)) - 1.0).reshape(m, ny, nx)
    return Problem("cde_cellular", nx, ny, m, np.asarray(D, np.float64)[:m, :m], 0.1, phi0=phi0, u0=u0,
                   steps=steps, case1=True, **sides)


def periodic_box(nx: int, ny: int, seed: int = 0, m: int = 2, u0: float = 0.02) -> Problem:
    """Large periodic cross-diffusion box (roofline grid): the Taylor-Green setup at any size."""
    return cross_diffusion_taylor_green(nx, ny, seed=seed, u0=u0).replace(name="periodic_box")


# ----------------------------------------------------------------------------
# three-dimensional problems (D3Q7 scalars, D3Q19 fluid)
# ----------------------------------------------------------------------------
@dataclass
class Problem3D:
    """A 3-D CDF problem in lattice units plus its initial moments.  Sides in the
    order x-, x+, y-, y+, z-, z+; walls are no slip for the fluid."""
    name: str
    nx: int
    ny: int
    nz: int
    m: int
    D: np.ndarray
    nu: float
    dkind: str = "const"
    chi: float = 0.0
    c_star: float = 0.3
    eps: float = 0.0
    r_regularised: bool = False
    skind: str = "none"
    S: np.ndarray = None
    k: float = 0.0
    g: tuple = (0.0, 0.0, 0.0)
    beta: np.ndarray = None
    phi_ref: np.ndarray = None
    F0: float = 0.0
    rho0: float = 1.0
    sides: List[Side] = None
    phi0: np.ndarray = None            # (m, nz, ny, nx)
    u0: np.ndarray = None              # (3, nz, ny, nx)
    p0: np.ndarray = None              # (nz, ny, nx)
    steps: int = 0

    def __post_init__(self):
        m = self.m
        self.D = np.asarray(self.D, dtype=np.float64).reshape(m, m)
        self.S = np.zeros(m) if self.S is None else np.asarray(self.S, np.float64)
        self.beta = np.zeros(m) if self.beta is None else np.asarray(self.beta, np.float64)
        self.phi_ref = np.zeros(m) if self.phi_ref is None else np.asarray(self.phi_ref, np.float64)
        if self.sides is None:
            self.sides = [periodic_side(m) for _ in range(6)]
        shape = (self.nz, self.ny, self.nx)
        if self.phi0 is None:
            self.phi0 = np.ones((m,) + shape)
        if self.u0 is None:
            self.u0 = np.zeros((3,) + shape)
        if self.p0 is None:
            self.p0 = np.zeros(shape)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Problem3D":
        return dataclasses.replace(self, **kw)


def periodic_box3d(nx: int, ny: int = None, nz: int = None, seed: int = 0, m: int = 2, u0: float = 0.02,
                   D=((0.05, 0.01), (0.005, 0.03)), nu: float = 0.1) -> Problem3D:
    """Periodic box, constant cross-diffusion D, the 3-D Taylor-Green initial velocity
    u = u0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0) (k = 2 pi / n per axis),
    scalars 1 + 0.1 U(-1, 1) from seed (counters a * N + node)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = 2 * math.pi * x / nx, 2 * math.pi * y / ny, 2 * math.pi * z / nz
    u = np.stack([u0 * np.sin(kx) * np.cos(ky) * np.cos(kz), -u0 * np.cos(kx) * np.sin(ky) * np.cos(kz),
                  np.zeros_like(kx)])
    n = nx * ny * nz
    phi0 = 1.0 + 0.1 * (2.0 * uniform(seed, np.arange(m * n)) - 1.0).reshape(m, nz, ny, nx)
    return Problem3D("periodic_box3d", nx, ny, nz, m, np.asarray(D, np.float64)[:m, :m], nu, phi0=phi0, u0=u)


def ddc_cavity3d(n: int, Ra: float = 1e4, Pr: float = 0.7, Le: float = 2.0, Nc: float = 1.0, Df: float = 0.1,
                 Sr: float = 0.1, seed: int = 0, ny: Optional[int] = None, nz: Optional[int] = None,
                 gravity_axis: int = 2, periodic_z: bool = False) -> Problem3D:
    """Double-diffusive cavity (the Sec. 3.2 setup in 3-D): T = C = 1 on the x- wall,
    0 on the x+ wall, the other walls adiabatic, gravity along +z (gravity_axis = 2)
    or +y (1) in the dimensionless form F = g (T + Nc C) e_g; the lattice mapping of
    the 2-D cavity with n nodes across; from rest with T = C = 0.  periodic_z makes a
    slab whose z-independent solution is the 2-D cavity's."""
    m = 2
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    alpha, nu, g = ddc_lattice_parameters(n, Ra, Pr)
    D = alpha * np.array([[1.0, Df], [Sr / Le, 1.0 / Le]])
    hot = wall_side(m, NOSLIP, [DIRICHLET, DIRICHLET], [1.0, 1.0])
    cold = wall_side(m, NOSLIP, [DIRICHLET, DIRICHLET], [0.0, 0.0])
    zs = [periodic_side(m), periodic_side(m)] if periodic_z else [wall_side(m), wall_side(m)]
    sides = [hot, cold, wall_side(m), wall_side(m)] + zs
    gv = [0.0, 0.0, 0.0]
    gv[gravity_axis] = 1.0
    return Problem3D("ddc_cavity3d", n, ny, nz, m, D, nu, g=tuple(gv), beta=np.array([g, g * Nc]),
                     sides=sides, phi0=np.zeros((m, nz, ny, n)))
