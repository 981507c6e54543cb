"""Python access to the 3-D CPU FP64 oracle (`cdf_oracle3d.c`: D3Q7 scalars,
D3Q19 fluid).

TEST INFRASTRUCTURE.  Only the tests, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` use it; the CUDA library never does.  Pinned in
tests/test_oracle3d_pins.py by the moment identities of the D3Q7/D3Q19
equilibria and sources, the continuum limit of an eigenmode of D on a
diagonal wave vector, exact mass conservation, exact plane Poiseuille flow along
two axes, the decay of a z-dependent shear wave and the anti-bounce-back linear
profile.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdf_oracle3d.c")
_LIB = os.path.join(_HERE, "libcdforacle3d.so")
_lock = threading.Lock()
_lib = None
MAX_M = 8


def build(force: bool = False) -> str:
    """Compile the 3-D oracle with the host C compiler (plain C99, -O2)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
            os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("m", ctypes.c_int),
        ("dkind", ctypes.c_int), ("D", ctypes.c_double * (MAX_M * MAX_M)),
        ("chi", ctypes.c_double), ("c_star", ctypes.c_double), ("eps", ctypes.c_double),
        ("r_regularised", ctypes.c_int), ("skind", ctypes.c_int), ("S", ctypes.c_double * MAX_M),
        ("k", ctypes.c_double), ("g", ctypes.c_double * 3), ("beta", ctypes.c_double * MAX_M),
        ("phi_ref", ctypes.c_double * MAX_M), ("F0", ctypes.c_double), ("nu", ctypes.c_double),
        ("rho0", ctypes.c_double), ("side_kind", ctypes.c_int * 6),
        ("scalar_bc", (ctypes.c_int * MAX_M) * 6), ("value", (ctypes.c_double * MAX_M) * 6),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def _bind(path):
    lib = ctypes.CDLL(path)
    lib.o3_create.restype = ctypes.c_void_p
    lib.o3_create.argtypes = [ctypes.POINTER(_Params)]
    lib.o3_destroy.argtypes = [ctypes.c_void_p]
    lib.o3_time.restype = ctypes.c_long
    lib.o3_time.argtypes = [ctypes.c_void_p]
    lib.o3_init.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
    lib.o3_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.o3_moments.argtypes = [ctypes.c_void_p, _DP]
    lib.o3_post_collision.argtypes = [ctypes.c_void_p, _DP, _DP]
    lib.o3_feq_scalar.argtypes = [ctypes.c_double, _DP, _DP]
    lib.o3_heq.argtypes = [ctypes.c_double, _DP, ctypes.c_double, _DP]
    lib.o3_force_pop.argtypes = [_DP, _DP]
    lib.o3_relaxation_matrix.argtypes = [ctypes.c_int, _DP, _DP]
    lib.o3_aux_source.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP, _DP, _DP]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


class Binding:
    """The 3-D oracle loaded from another shared object (the planted-mistake tests)."""

    def __init__(self, path: str):
        self.lib = _bind(path)

    def Sim(self, problem, init: bool = True):
        return Sim(problem, init, self.lib)

    def __getattr__(self, name):
        fn = globals()[name]
        return lambda *a, **k: fn(*a, lib=self.lib, **k)


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def compile_source(src_text: str, out_path: str) -> str:
    c_path = out_path + ".c"
    with open(c_path, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", out_path, c_path, "-lm"], check=True)
    return out_path


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def params_from_problem(pb) -> _Params:
    P = _Params()
    m = pb.m
    P.nx, P.ny, P.nz, P.m = pb.nx, pb.ny, pb.nz, m
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
    for d in range(3):
        P.g[d] = float(pb.g[d])
    P.F0, P.nu, P.rho0 = pb.F0, pb.nu, pb.rho0
    for s, side in enumerate(pb.sides):
        P.side_kind[s] = {"periodic": 0, "wall": 1}[side.kind]
        for a in range(m):
            P.scalar_bc[s][a] = {"noflux": 0, "dirichlet": 1}[side.scalar[a]]
            P.value[s][a] = float(side.value[a])
    return P


class Sim:
    """One 3-D lattice advanced by the FP64 oracle."""

    def __init__(self, problem, init: bool = True, lib=None):
        self.lib = lib if lib is not None else _load()
        self.pb = problem
        self.m, self.nx, self.ny, self.nz = problem.m, problem.nx, problem.ny, problem.nz
        self._P = params_from_problem(problem)
        self.h = self.lib.o3_create(ctypes.byref(self._P))
        if not self.h:
            raise ValueError("3-D oracle rejected the problem parameters")
        if init:
            self.init(problem.phi0, problem.u0, problem.p0)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.o3_destroy(h)
            self.h = None

    def init(self, phi0, u0, p0=None):
        phi = np.ascontiguousarray(phi0, np.float64)
        u = np.ascontiguousarray(u0, np.float64)
        p = None if p0 is None else np.ascontiguousarray(p0, np.float64)
        self.lib.o3_init(self.h, _ptr(phi), _ptr(u), None if p is None else _ptr(p))

    @property
    def t(self) -> int:
        return self.lib.o3_time(self.h)

    def step(self, n: int = 1):
        if self.lib.o3_step(self.h, int(n)) != 0:
            raise FloatingPointError("singular relaxation matrix")

    def moments(self) -> np.ndarray:
        out = np.empty((self.m + 4, self.nz, self.ny, self.nx))
        self.lib.o3_moments(self.h, _ptr(out))
        return out

    def post_collision(self):
        f = np.empty((self.m, 7, self.nz, self.ny, self.nx))
        h = np.empty((19, self.nz, self.ny, self.nx))
        if self.lib.o3_post_collision(self.h, _ptr(f), _ptr(h)) != 0:
            raise FloatingPointError("singular relaxation matrix")
        return f, h


# ---- single-node functions -------------------------------------------------------------
def feq_scalar(phi, u, lib=None):
    out = np.empty(7)
    (lib or _load()).o3_feq_scalar(phi, _ptr(np.ascontiguousarray(u, np.float64)), _ptr(out))
    return out


def heq(p, u, rho0=1.0, lib=None):
    out = np.empty(19)
    (lib or _load()).o3_heq(p, _ptr(np.ascontiguousarray(u, np.float64)), rho0, _ptr(out))
    return out


def force_pop(F, lib=None):
    out = np.empty(19)
    (lib or _load()).o3_force_pop(_ptr(np.ascontiguousarray(F, np.float64)), _ptr(out))
    return out


def relaxation_matrix(D, lib=None):
    D = np.ascontiguousarray(D, np.float64)
    m = D.shape[0]
    out = np.empty((m, m))
    if (lib or _load()).o3_relaxation_matrix(m, _ptr(D), _ptr(out)) != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def aux_source(omega, phi, u, S, F, lib=None):
    omega = np.ascontiguousarray(omega, np.float64)
    m = omega.shape[0]
    out = np.empty((m, 7))
    f64 = lambda a: np.ascontiguousarray(a, np.float64)  # noqa: E731
    (lib or _load()).o3_aux_source(m, _ptr(omega), _ptr(f64(phi)), _ptr(f64(u)), _ptr(f64(S)), _ptr(f64(F)),
                                   _ptr(out))
    return out
