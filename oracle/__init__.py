"""Python access to the CPU FP64 oracle (`cdf_oracle.c`).

TEST INFRASTRUCTURE.  Only the tests, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` use this package; the CUDA library never does.
The oracle is the lattice Boltzmann model of Zhan, Chai & Shi
(arXiv:2101.03055), Eqs. evolution12/evolution3 with feq-phi, heq, force,
source, Gi, sum-phi/u/p and omega-D, in FP64, one node at a time.

Pinned (tests/test_oracle_pins.py) by: the moment identities of Eq. moment and
Eq. momentNS; the exact linear amplification of a Fourier mode and its
continuum limit (eigenvalues of D times |k|^2); Taylor-Green decay; exact mass
conservation; reduction to decoupled single-scalar runs and index permutation;
the closed-form steady chemotaxis profile of Sec. 3.1.1; and the centro-symmetry
of the double-diffusive cavity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdf_oracle.c")
_LIB = os.path.join(_HERE, "libcdforacle.so")
_lock = threading.Lock()
_lib = None

MAX_M = 8
_SIDES = ("west", "east", "south", "north")


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C99, -O2).  OpenMP is
    compiled in when the compiler has it, for the all-cores CPU baseline only: the
    oracle runs one thread unless set_threads asks for more, and its results do
    not depend on the thread count."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            base = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True)
            if r.returncode != 0:
                subprocess.run(base, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Threads of the oracle's node and row loops (n < 1: all cores); returns the
    count in use (1 if the oracle was built without OpenMP)."""
    return int(_load().orc_set_threads(int(n)))


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("m", ctypes.c_int),
        ("dkind", ctypes.c_int), ("D", ctypes.c_double * (MAX_M * MAX_M)),
        ("chi", ctypes.c_double), ("c_star", ctypes.c_double), ("eps", ctypes.c_double),
        ("r_regularised", ctypes.c_int),
        ("skind", ctypes.c_int), ("S", ctypes.c_double * MAX_M), ("k", ctypes.c_double),
        ("g", ctypes.c_double * 2), ("beta", ctypes.c_double * MAX_M),
        ("phi_ref", ctypes.c_double * MAX_M), ("F0", ctypes.c_double),
        ("nu", ctypes.c_double), ("rho0", ctypes.c_double), ("theta", ctypes.c_double),
        ("side_kind", ctypes.c_int * 4), ("fluid_bc", ctypes.c_int * 4),
        ("scalar_bc", (ctypes.c_int * MAX_M) * 4), ("value", (ctypes.c_double * MAX_M) * 4),
        ("case1", ctypes.c_int), ("varphi", ctypes.c_double),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def _bind(path):
    lib = ctypes.CDLL(path)
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [ctypes.POINTER(_Params)]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_time.restype = ctypes.c_long
    lib.orc_time.argtypes = [ctypes.c_void_p]
    lib.orc_init.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
    lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.orc_moments.argtypes = [ctypes.c_void_p, _DP]
    lib.orc_get_state.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
    lib.orc_set_state.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
    lib.orc_post_collision.argtypes = [ctypes.c_void_p, _DP, _DP]
    lib.orc_feq_scalar.argtypes = [ctypes.c_double] * 4 + [_DP]
    lib.orc_heq.argtypes = [ctypes.c_double] * 4 + [_DP]
    lib.orc_force_pop.argtypes = [ctypes.c_double] * 2 + [_DP]
    lib.orc_force_pop_phi.argtypes = [ctypes.c_double] * 5 + [_DP]
    lib.orc_relaxation_matrix.argtypes = [ctypes.c_int, _DP, _DP]
    lib.orc_fluid_relaxation.restype = ctypes.c_double
    lib.orc_fluid_relaxation.argtypes = [ctypes.c_double]
    lib.orc_aux_source.argtypes = [ctypes.c_int, _DP, _DP, ctypes.c_double, ctypes.c_double,
                                   _DP, ctypes.c_double, ctypes.c_double, _DP]
    lib.orc_aux_source_case1.argtypes = [ctypes.c_int, _DP, _DP, _DP, ctypes.c_double, ctypes.c_double, _DP]
    lib.orc_cutoff.restype = ctypes.c_double
    lib.orc_cutoff.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int]
    lib.orc_closures.argtypes = [ctypes.POINTER(_Params), _DP, _DP, _DP, _DP]
    lib.orc_set_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def params_from_problem(pb, theta: float = 0.0) -> _Params:
    P = _Params()
    m = pb.m
    if m > MAX_M:
        raise ValueError("m too large for the oracle")
    P.nx, P.ny, P.m = pb.nx, pb.ny, m
    P.dkind = {"const": 0, "chemotaxis": 1}[pb.dkind]
    for a in range(m):
        for b in range(m):
            P.D[a * m + b] = float(pb.D[a, b])
    P.chi, P.c_star, P.eps, P.r_regularised = pb.chi, pb.c_star, pb.eps, int(pb.r_regularised)
    P.skind = {"none": 0, "const": 1, "consumption": 2}[pb.skind]
    for a in range(m):
        P.S[a] = float(pb.S[a])
        P.beta[a] = float(pb.beta[a])
        P.phi_ref[a] = float(pb.phi_ref[a])
    P.k = pb.k
    P.g[0], P.g[1] = float(pb.g[0]), float(pb.g[1])
    P.F0, P.nu, P.rho0, P.theta = pb.F0, pb.nu, pb.rho0, theta
    P.case1 = int(getattr(pb, "case1", False))
    P.varphi = float(getattr(pb, "varphi", 0.0))
    for s, name in enumerate(_SIDES):
        side = getattr(pb, name)
        P.side_kind[s] = {"periodic": 0, "wall": 1}[side.kind]
        P.fluid_bc[s] = {"noslip": 0, "freeslip": 1}[side.fluid]
        for a in range(m):
            P.scalar_bc[s][a] = {"noflux": 0, "dirichlet": 1}[side.scalar[a]]
            P.value[s][a] = float(side.value[a])
    return P


class OracleSim:
    """One lattice advanced by the FP64 oracle."""

    def __init__(self, problem, theta: float = 0.0, init: bool = True, lib=None):
        self.lib = lib if lib is not None else _load()
        self.pb = problem
        self.m, self.nx, self.ny = problem.m, problem.nx, problem.ny
        self._P = params_from_problem(problem, theta)
        self.h = self.lib.orc_create(ctypes.byref(self._P))
        if not self.h:
            raise ValueError("oracle rejected the problem parameters")
        if init:
            self.init(problem.phi0, problem.u0, problem.p0)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_destroy(h)
            self.h = None

    def init(self, phi0, u0, p0=None):
        phi = np.ascontiguousarray(phi0, np.float64)
        u = np.ascontiguousarray(u0, np.float64)
        p = None if p0 is None else np.ascontiguousarray(p0, np.float64)
        self.lib.orc_init(self.h, _ptr(phi), _ptr(u), None if p is None else _ptr(p))

    @property
    def t(self) -> int:
        return self.lib.orc_time(self.h)

    def step(self, n: int = 1):
        if self.lib.orc_step(self.h, int(n)) != 0:
            raise FloatingPointError("singular relaxation matrix")

    def moments(self) -> np.ndarray:
        out = np.empty((self.m + 3, self.ny, self.nx))
        self.lib.orc_moments(self.h, _ptr(out))
        return out

    def state(self):
        f = np.empty((self.m, 5, self.ny, self.nx))
        h = np.empty((9, self.ny, self.nx))
        sp = np.empty((self.m, self.ny, self.nx))
        self.lib.orc_get_state(self.h, _ptr(f), _ptr(h), _ptr(sp))
        return f, h, sp

    def set_state(self, f, h, sprev=None):
        f = np.ascontiguousarray(f, np.float64)
        h = np.ascontiguousarray(h, np.float64)
        sp = None if sprev is None else np.ascontiguousarray(sprev, np.float64)
        self.lib.orc_set_state(self.h, _ptr(f), _ptr(h), None if sp is None else _ptr(sp))

    def post_collision(self):
        f = np.empty((self.m, 5, self.ny, self.nx))
        h = np.empty((9, self.ny, self.nx))
        if self.lib.orc_post_collision(self.h, _ptr(f), _ptr(h)) != 0:
            raise FloatingPointError("singular relaxation matrix")
        return f, h


# ---- single-node functions --------------------------------------------------------
def feq_scalar(phi, ux, uy, theta=0.0, lib=None):
    out = np.empty(5)
    (lib or _load()).orc_feq_scalar(phi, ux, uy, theta, _ptr(out))
    return out


def heq(p, ux, uy, rho0=1.0, lib=None):
    out = np.empty(9)
    (lib or _load()).orc_heq(p, ux, uy, rho0, _ptr(out))
    return out


def force_pop(Fx, Fy, lib=None):
    out = np.empty(9)
    (lib or _load()).orc_force_pop(Fx, Fy, _ptr(out))
    return out


def force_pop_phi(F, u, varphi, lib=None):
    """Eq. force with its second-order part: F_i = W_i [c_i.F/cs^2 + varphi (uF + Fu):(c_i c_i - cs^2 I)/(2 cs^4)]."""
    out = np.empty(9)
    (lib or _load()).orc_force_pop_phi(F[0], F[1], u[0], u[1], varphi, _ptr(out))
    return out


def relaxation_matrix(D, lib=None):
    D = np.ascontiguousarray(D, np.float64)
    m = D.shape[0]
    out = np.empty((m, m))
    if (lib or _load()).orc_relaxation_matrix(m, _ptr(D), _ptr(out)) != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def fluid_relaxation(nu, lib=None):
    return (lib or _load()).orc_fluid_relaxation(nu)


def aux_source(omega, phi, u, S, F, lib=None):
    omega = np.ascontiguousarray(omega, np.float64)
    m = omega.shape[0]
    phi = np.ascontiguousarray(phi, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    out = np.empty((m, 5))
    (lib or _load()).orc_aux_source(m, _ptr(omega), _ptr(phi), u[0], u[1], _ptr(S), F[0], F[1], _ptr(out))
    return out


def cutoff(c, c_star, eps=0.0, regularised=False, lib=None):
    return (lib or _load()).orc_cutoff(c, c_star, eps, int(regularised))


def closures(problem, phi, lib=None):
    P = params_from_problem(problem)
    m = problem.m
    phi = np.ascontiguousarray(phi, np.float64)
    D = np.empty((m, m))
    S = np.empty(m)
    F = np.empty(2)
    (lib or _load()).orc_closures(ctypes.byref(P), _ptr(phi), _ptr(D), _ptr(S), _ptr(F))
    return D, S, F


class Binding:
    """The oracle's Python API bound to one compiled library (the default build,
    or a copy built from edited source by the tests that check the pins)."""

    def __init__(self, path: str):
        self.lib = _bind(path)

    def OracleSim(self, problem, theta: float = 0.0, init: bool = True):
        return OracleSim(problem, theta, init, lib=self.lib)

    def __getattr__(self, name):
        fn = globals().get(name)
        if name in _NODE_FUNCS and fn is not None:
            return lambda *a, **k: fn(*a, lib=self.lib, **k)
        raise AttributeError(name)


_NODE_FUNCS = {"feq_scalar", "heq", "force_pop", "force_pop_phi", "relaxation_matrix", "fluid_relaxation",
               "aux_source", "cutoff", "closures"}


def compile_source(src_text: str, out_path: str) -> str:
    """Compile C source text of the oracle to `out_path` (used to build planted-mistake copies)."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", out_path, src, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()
