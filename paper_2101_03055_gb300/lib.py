"""Thin ctypes binding of libcdflb (include/cdf_lb.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
The functions keep the C names (cdf_lb_create, cdf_lb_step, ...); `Solver`
wraps a handle for convenience.  PyTorch is used for device memory and streams
only (device tensors are passed as raw pointers).  There is no CPU fallback:
loading fails loudly when the library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .inputs import Problem

_PKG = os.path.dirname(os.path.abspath(__file__))
# CDF_CHECKS=1 in the environment selects the checks build (built by
# build.build(checks=True)): offset checks in the step kernels and canary pads
# around the device buffers, same results.
CHECKS = os.environ.get("CDF_CHECKS", "0") not in ("", "0")
LIB_PATH = os.path.join(_PKG, "libcdflb_checks.so" if CHECKS else "libcdflb.so")
MAX_M = 4

(CDF_OK, CDF_EINVAL, CDF_ENOMEM, CDF_ECUDA, CDF_ENOTCONVERGED, CDF_EUNSTABLE, CDF_ETIMEOUT, CDF_EIO,
 CDF_ECHECK) = range(9)
STATUS_NAMES = ["CDF_OK", "CDF_EINVAL", "CDF_ENOMEM", "CDF_ECUDA", "CDF_ENOTCONVERGED",
                "CDF_EUNSTABLE", "CDF_ETIMEOUT", "CDF_EIO", "CDF_ECHECK"]
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}


class CdfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class cdf_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int)]


class cdf_diffusion(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("D", ctypes.c_double * (MAX_M * MAX_M)),
                ("chi", ctypes.c_double), ("c_star", ctypes.c_double), ("eps", ctypes.c_double),
                ("r_regularised", ctypes.c_int)]


class cdf_source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("S", ctypes.c_double * MAX_M), ("k", ctypes.c_double)]


class cdf_force(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double * 2), ("beta", ctypes.c_double * MAX_M),
                ("phi_ref", ctypes.c_double * MAX_M), ("F0", ctypes.c_double), ("varphi", ctypes.c_double)]


class cdf_side(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("fluid", ctypes.c_int), ("scalar", ctypes.c_int * MAX_M),
                ("value", ctypes.c_double * MAX_M)]


class cdf_boundaries(ctypes.Structure):
    _fields_ = [("west", cdf_side), ("east", cdf_side), ("south", cdf_side), ("north", cdf_side)]


class cdf_options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("rho0", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("phi_ref", ctypes.c_double * MAX_M), ("p_ref_grad", ctypes.c_double * 2),
                ("block_x", ctypes.c_int), ("block_y", ctypes.c_int), ("resident", ctypes.c_int),
                ("wait_timeout_s", ctypes.c_double), ("test_stall_tile", ctypes.c_int),
                ("prescribed_velocity", ctypes.c_int), ("temporal", ctypes.c_int),
                ("temporal_block_x", ctypes.c_int), ("temporal_block_y", ctypes.c_int),
                ("temporal_tile_y", ctypes.c_int), ("halo_rows", ctypes.c_int), ("origin_y", ctypes.c_int),
                ("ny_global", ctypes.c_int), ("temporal_lanes", ctypes.c_int), ("block_lanes", ctypes.c_int)]


class cdf_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("m", ctypes.c_int), ("pitch", ctypes.c_int),
                ("storage", ctypes.c_int), ("planes", ctypes.c_int), ("sprev_planes", ctypes.c_int),
                ("block_x", ctypes.c_int), ("block_y", ctypes.c_int), ("resident", ctypes.c_int),
                ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("tiles", ctypes.c_int),
                ("bytes_per_lup", ctypes.c_double), ("t", ctypes.c_longlong), ("temporal", ctypes.c_int),
                ("lanes", ctypes.c_int)]


class cdf_batch_options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("rho0", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("steps_per_launch", ctypes.c_int),
                ("barrier_timeout_s", ctypes.c_double), ("test_unreachable_barrier", ctypes.c_int),
                ("mode", ctypes.c_int), ("chain_tile_y", ctypes.c_int), ("chain_lanes", ctypes.c_int)]


class cdf_batch_info(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("m", ctypes.c_int), ("nodes", ctypes.c_longlong),
                ("tiles", ctypes.c_longlong), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("grid_blocks", ctypes.c_int), ("steps_per_launch", ctypes.c_int),
                ("bytes_per_lup", ctypes.c_double), ("t", ctypes.c_longlong), ("mode", ctypes.c_int),
                ("chain_block_x", ctypes.c_int), ("chain_block_y", ctypes.c_int), ("chain_tile_y", ctypes.c_int),
                ("chain_lanes", ctypes.c_int)]


_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.c_void_p
_H = ctypes.c_void_p
_lib = None

# name -> (restype, argtypes); the C ABI of include/cdf_lb.h
class cdf_grid3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class cdf_force3(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double * 3), ("beta", ctypes.c_double * MAX_M), ("phi_ref", ctypes.c_double * MAX_M),
                ("F0", ctypes.c_double)]


class cdf_boundaries3(ctypes.Structure):
    _fields_ = [("side", cdf_side * 6)]


class cdf_options3(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_double), ("cuda_stream", ctypes.c_void_p), ("phi_ref", ctypes.c_double * MAX_M),
                ("p_ref_grad", ctypes.c_double * 3), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int)]


class cdf_info3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("m", ctypes.c_int),
                ("pitch", ctypes.c_int), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
                ("bytes_per_lup", ctypes.c_double), ("t", ctypes.c_longlong)]


SIGNATURES = {
    "cdf_lb_create": (ctypes.c_int, [ctypes.POINTER(cdf_grid), ctypes.c_int, ctypes.POINTER(cdf_diffusion),
                                     ctypes.c_double, ctypes.POINTER(cdf_source), ctypes.POINTER(cdf_force),
                                     ctypes.POINTER(cdf_boundaries), ctypes.POINTER(cdf_options),
                                     ctypes.POINTER(ctypes.c_void_p)]),
    "cdf_lb_init_moments": (ctypes.c_int, [_H, _DP, _DP, _DP]),
    "cdf_lb_init_moments_device": (ctypes.c_int, [_H, _FP]),
    "cdf_lb_step": (ctypes.c_int, [_H, ctypes.c_longlong]),
    "cdf_lb_run_to_steady": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_longlong, ctypes.c_longlong,
                                            ctypes.POINTER(ctypes.c_longlong), _DP]),
    "cdf_lb_moments": (ctypes.c_int, [_H, _DP]),
    "cdf_lb_moments_device": (ctypes.c_int, [_H, _FP]),
    "cdf_lb_mass": (ctypes.c_int, [_H, _DP]),
    "cdf_lb_populations": (ctypes.c_int, [_H, _DP, _DP, _DP]),
    "cdf_lb_save": (ctypes.c_int, [_H, ctypes.c_char_p]),
    "cdf_lb_load": (ctypes.c_int, [_H, ctypes.c_char_p]),
    "cdf_lb_get_info": (ctypes.c_int, [_H, ctypes.POINTER(cdf_info)]),
    "cdf_lb_stream": (ctypes.c_void_p, [_H]),
    "cdf_lb_destroy": (None, [_H]),
    "cdf_lb_last_error": (ctypes.c_char_p, []),
    "cdf_moment_sums_static": (ctypes.c_int, [_FP, _FP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _FP,
                                              ctypes.c_void_p]),
    "cdf_lb_wall_transfer": (ctypes.c_int, [_H, ctypes.c_int] + [ctypes.c_double] * 4 + [_DP]),
    "cdf_lb_halo_pack": (ctypes.c_int, [_H, ctypes.c_int, _FP]),
    "cdf_lb_halo_unpack": (ctypes.c_int, [_H, ctypes.c_int, _FP]),
    "cdf_lb_snapshot": (ctypes.c_int, [_H]),
    "cdf_lb_change_sums": (ctypes.c_int, [_H, _DP]),
    "cdf_split_create": (ctypes.c_int, [ctypes.POINTER(cdf_grid), ctypes.c_int, ctypes.POINTER(cdf_diffusion),
                                        ctypes.c_double, ctypes.POINTER(cdf_source), ctypes.POINTER(cdf_force),
                                        ctypes.POINTER(cdf_boundaries), ctypes.POINTER(cdf_options), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "cdf_split_init_moments": (ctypes.c_int, [_H, _DP, _DP, _DP]),
    "cdf_split_step": (ctypes.c_int, [_H, ctypes.c_longlong]),
    "cdf_split_moments": (ctypes.c_int, [_H, _DP]),
    "cdf_split_mass": (ctypes.c_int, [_H, _DP]),
    "cdf_split_run_to_steady": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_longlong, ctypes.c_longlong,
                                               ctypes.POINTER(ctypes.c_longlong), _DP]),
    "cdf_split_slab": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "cdf_split_destroy": (None, [_H]),
    "cdf_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(cdf_grid), ctypes.c_int,
                                        ctypes.POINTER(cdf_diffusion), _DP, ctypes.POINTER(cdf_source),
                                        ctypes.POINTER(cdf_force), ctypes.POINTER(cdf_boundaries), _DP, _DP,
                                        ctypes.POINTER(cdf_batch_options), ctypes.POINTER(ctypes.c_void_p)]),
    "cdf_batch_init_moments": (ctypes.c_int, [_H, ctypes.c_int, _DP, _DP, _DP]),
    "cdf_batch_step": (ctypes.c_int, [_H, ctypes.c_longlong]),
    "cdf_batch_moments": (ctypes.c_int, [_H, ctypes.c_int, _DP]),
    "cdf_batch_init_moments_device": (ctypes.c_int, [_H, ctypes.c_int, _FP]),
    "cdf_batch_moments_device": (ctypes.c_int, [_H, ctypes.c_int, _FP]),
    "cdf_batch_get_info": (ctypes.c_int, [_H, ctypes.POINTER(cdf_batch_info)]),
    "cdf_batch_snapshot": (ctypes.c_int, [_H]),
    "cdf_batch_residuals": (ctypes.c_int, [_H, _DP]),
    "cdf_batch_stream": (ctypes.c_void_p, [_H]),
    "cdf_batch_destroy": (None, [_H]),
    "cdf_lb3d_create": (ctypes.c_int, [ctypes.POINTER(cdf_grid3), ctypes.c_int, ctypes.POINTER(cdf_diffusion),
                                       ctypes.c_double, ctypes.POINTER(cdf_source), ctypes.POINTER(cdf_force3),
                                       ctypes.POINTER(cdf_boundaries3), ctypes.POINTER(cdf_options3),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "cdf_lb3d_init_moments": (ctypes.c_int, [_H, _DP, _DP, _DP]),
    "cdf_lb3d_step": (ctypes.c_int, [_H, ctypes.c_longlong]),
    "cdf_lb3d_run_to_steady": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_longlong, ctypes.c_longlong,
                                              ctypes.POINTER(ctypes.c_longlong), _DP]),
    "cdf_lb3d_moments": (ctypes.c_int, [_H, _DP]),
    "cdf_lb3d_mass": (ctypes.c_int, [_H, _DP]),
    "cdf_lb3d_populations": (ctypes.c_int, [_H, _DP, _DP]),
    "cdf_lb3d_get_info": (ctypes.c_int, [_H, ctypes.POINTER(cdf_info3)]),
    "cdf_lb3d_stream": (ctypes.c_void_p, [_H]),
    "cdf_lb3d_destroy": (None, [_H]),
    "cdf_checks_enabled": (ctypes.c_int, []),
    "cdf_checks_selftest": (ctypes.c_int, [ctypes.c_int]),
}


def load(path: str = LIB_PATH):
    """Load libcdflb; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            how = "build(checks=True)" if path.endswith("_checks.so") else "build()"
            raise RuntimeError(f"libcdflb not built: {path} is missing (run paper_2101_03055_gb300.build.{how})")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int):
    if status != CDF_OK:
        raise CdfError(status, load().cdf_lb_last_error().decode())


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


# ---- same-name wrappers -----------------------------------------------------------
def cdf_lb_create(grid, m, diffusion, nu, source, force, boundaries, options):
    h = ctypes.c_void_p()
    _check(load().cdf_lb_create(ctypes.byref(grid), m, ctypes.byref(diffusion), nu, ctypes.byref(source),
                                ctypes.byref(force), ctypes.byref(boundaries), ctypes.byref(options),
                                ctypes.byref(h)))
    return h


def cdf_lb_init_moments(h, phi, u, p=None):
    _check(load().cdf_lb_init_moments(h, _dptr(phi), _dptr(u), None if p is None else _dptr(p)))


def cdf_lb_init_moments_device(h, dev_ptr: int):
    _check(load().cdf_lb_init_moments_device(h, ctypes.c_void_p(dev_ptr)))


def cdf_lb_step(h, n: int):
    _check(load().cdf_lb_step(h, int(n)))


def cdf_lb_run_to_steady(h, tol, check_every, max_steps):
    steps = ctypes.c_longlong(0)
    res = ctypes.c_double(0.0)
    st = load().cdf_lb_run_to_steady(h, tol, int(check_every), int(max_steps), ctypes.byref(steps), ctypes.byref(res))
    return st, steps.value, res.value


def cdf_lb_moments(h, out: np.ndarray):
    _check(load().cdf_lb_moments(h, _dptr(out)))


def cdf_lb_moments_device(h, dev_ptr: int):
    _check(load().cdf_lb_moments_device(h, ctypes.c_void_p(dev_ptr)))


def cdf_lb_mass(h, out: np.ndarray):
    _check(load().cdf_lb_mass(h, _dptr(out)))


def cdf_lb_populations(h, f=None, hf=None, s_now=None):
    _check(load().cdf_lb_populations(h, None if f is None else _dptr(f), None if hf is None else _dptr(hf),
                                     None if s_now is None else _dptr(s_now)))


def cdf_lb_save(h, path: str):
    _check(load().cdf_lb_save(h, path.encode()))


def cdf_lb_load(h, path: str):
    _check(load().cdf_lb_load(h, path.encode()))


def cdf_lb_get_info(h) -> cdf_info:
    info = cdf_info()
    _check(load().cdf_lb_get_info(h, ctypes.byref(info)))
    return info


def cdf_lb_stream(h) -> int:
    return load().cdf_lb_stream(h) or 0


def cdf_lb_destroy(h):
    load().cdf_lb_destroy(h)


def cdf_lb_last_error() -> str:
    return load().cdf_lb_last_error().decode()


def cdf_checks_enabled() -> bool:
    return bool(load().cdf_checks_enabled())


def cdf_checks_selftest(which: int) -> int:
    """The checks build's detector self-test: CDF_ECHECK when it caught the planted
    access (0: an offset beyond a device buffer; 1: a byte of a canary pad)."""
    return int(load().cdf_checks_selftest(int(which)))


def cdf_moment_sums_static(dev_fields: int, dev_fields_old: int, nx: int, ny: int, m: int, dev_out: int,
                           stream: int = 0) -> int:
    """Allocation-free FP64 sums over a device moment stack (see include/cdf_lb.h);
    returns the status code without raising."""
    return load().cdf_moment_sums_static(ctypes.c_void_p(dev_fields or None), ctypes.c_void_p(dev_fields_old or None),
                                         nx, ny, m, ctypes.c_void_p(dev_out or None), ctypes.c_void_p(stream or None))


def cdf_lb_wall_transfer(h, side: int, D_CT: float, S_TC: float, T_wall: float, C_wall: float) -> np.ndarray:
    out = np.empty(2)
    _check(load().cdf_lb_wall_transfer(h, int(side), D_CT, S_TC, T_wall, C_wall, _dptr(out)))
    return out


def cdf_lb_halo_pack(h, side: int, dev_buf: int):
    _check(load().cdf_lb_halo_pack(h, int(side), ctypes.c_void_p(dev_buf)))


def cdf_lb_halo_unpack(h, side: int, dev_buf: int):
    _check(load().cdf_lb_halo_unpack(h, int(side), ctypes.c_void_p(dev_buf)))


def cdf_lb_snapshot(h):
    _check(load().cdf_lb_snapshot(h))


def cdf_lb_change_sums(h, out: np.ndarray):
    _check(load().cdf_lb_change_sums(h, _dptr(out)))


def cdf_split_create(grid, m, diffusion, nu, source, force, boundaries, options, nslabs):
    h = ctypes.c_void_p()
    _check(load().cdf_split_create(ctypes.byref(grid), m, ctypes.byref(diffusion), nu, ctypes.byref(source),
                                   ctypes.byref(force), ctypes.byref(boundaries), ctypes.byref(options), int(nslabs),
                                   ctypes.byref(h)))
    return h


def cdf_split_init_moments(h, phi, u, p=None):
    _check(load().cdf_split_init_moments(h, _dptr(phi), _dptr(u), None if p is None else _dptr(p)))


def cdf_split_step(h, n: int):
    _check(load().cdf_split_step(h, int(n)))


def cdf_split_moments(h, out: np.ndarray):
    _check(load().cdf_split_moments(h, _dptr(out)))


def cdf_split_mass(h, out: np.ndarray):
    _check(load().cdf_split_mass(h, _dptr(out)))


def cdf_split_run_to_steady(h, tol, check_every, max_steps):
    steps = ctypes.c_longlong(0)
    res = ctypes.c_double(0.0)
    st = load().cdf_split_run_to_steady(h, tol, int(check_every), int(max_steps), ctypes.byref(steps),
                                        ctypes.byref(res))
    return st, steps.value, res.value


def cdf_split_slab(h, k: int):
    slab, y0, rows = ctypes.c_void_p(), ctypes.c_int(), ctypes.c_int()
    _check(load().cdf_split_slab(h, int(k), ctypes.byref(slab), ctypes.byref(y0), ctypes.byref(rows)))
    return slab, y0.value, rows.value


def cdf_split_destroy(h):
    load().cdf_split_destroy(h)


# ---- problem description -> C structs ------------------------------------------------
def structs_from_problem(pb: Problem, storage: str = "fp32", stream: int = 0, block=None, phi_ref=None,
                         p_ref_grad=None, resident: int = 0, wait_timeout_s: float = 0.0, test_stall_tile: int = 0,
                         temporal: int = 0, temporal_shape=None):
    m = pb.m
    if m > MAX_M:
        raise ValueError(f"m = {m} > {MAX_M}")
    grid = cdf_grid(pb.nx, pb.ny)
    dif = cdf_diffusion()
    dif.kind = {"const": 0, "chemotaxis": 1}[pb.dkind]
    for a in range(m):
        for b in range(m):
            dif.D[a * m + b] = float(pb.D[a, b])
    dif.chi, dif.c_star, dif.eps, dif.r_regularised = pb.chi, pb.c_star, pb.eps, int(pb.r_regularised)
    src = cdf_source()
    src.kind = {"none": 0, "const": 1, "consumption": 2}[pb.skind]
    src.k = pb.k
    frc = cdf_force()
    frc.g[0], frc.g[1] = float(pb.g[0]), float(pb.g[1])
    frc.F0 = pb.F0
    frc.varphi = float(getattr(pb, "varphi", 0.0))
    for a in range(m):
        src.S[a] = float(pb.S[a])
        frc.beta[a] = float(pb.beta[a])
        frc.phi_ref[a] = float(pb.phi_ref[a])
    bc = cdf_boundaries()
    for name in ("west", "east", "south", "north"):
        side, cs = getattr(pb, name), getattr(bc, name)
        cs.kind = {"periodic": 0, "wall": 1}[side.kind]
        cs.fluid = {"noslip": 0, "freeslip": 1}[side.fluid]
        for a in range(m):
            cs.scalar[a] = {"noflux": 0, "dirichlet": 1}[side.scalar[a]]
            cs.value[a] = float(side.value[a])
    opt = cdf_options()
    opt.storage = STORAGE[storage]
    opt.rho0 = pb.rho0
    opt.cuda_stream = stream or None
    ref = phi_ref if phi_ref is not None else default_phi_ref(pb)
    for a in range(m):
        opt.phi_ref[a] = float(ref[a])
    grad = p_ref_grad if p_ref_grad is not None else default_p_ref_grad(pb)
    opt.p_ref_grad[0], opt.p_ref_grad[1] = float(grad[0]), float(grad[1])
    if block is not None:  # (block_x, block_y) or, for a flat launch, (block_x, 0, lanes)
        opt.block_x, opt.block_y = block[0], block[1]
        if len(block) > 2:
            opt.block_lanes = block[2]
    opt.resident, opt.wait_timeout_s, opt.test_stall_tile = int(resident), float(wait_timeout_s), int(test_stall_tile)
    opt.prescribed_velocity = int(getattr(pb, "case1", False))
    opt.temporal = int(temporal)
    if temporal_shape is not None:  # (block_x, block_y, tile_y) or (block_x, block_y, tile_y, lanes)
        ts = [int(v) for v in temporal_shape]
        opt.temporal_block_x, opt.temporal_block_y, opt.temporal_tile_y = ts[:3]
        if len(ts) > 3:
            opt.temporal_lanes = ts[3]
    return grid, dif, src, frc, bc, opt


def default_phi_ref(pb: Problem):
    """Reference scalar values of the deviation storage: the midpoint of the
    initial range of each scalar, widened to include its Dirichlet values."""
    ref = []
    for a in range(pb.m):
        lo, hi = float(pb.phi0[a].min()), float(pb.phi0[a].max())
        for name in ("west", "east", "south", "north"):
            side = getattr(pb, name)
            if side.kind == "wall" and side.scalar[a] == "dirichlet":
                lo, hi = min(lo, side.value[a]), max(hi, side.value[a])
        ref.append(0.5 * (lo + hi))
    return ref


def default_p_ref_grad(pb: Problem):
    """Reference pressure gradient of the fluid deviation storage: the hydrostatic
    gradient grad p = F of the force at the mean initial scalar values."""
    mag = pb.F0 + sum(float(pb.beta[a]) * (float(pb.phi0[a].mean()) - float(pb.phi_ref[a])) for a in range(pb.m))
    return (float(pb.g[0]) * mag, float(pb.g[1]) * mag)


class Solver:
    """One lattice on the GPU behind the C ABI."""

    def __init__(self, pb: Problem, storage: str = "fp32", stream: int = 0, block=None, init: bool = True,
                 phi_ref=None, p_ref_grad=None, resident: int = 0, wait_timeout_s: float = 0.0,
                 test_stall_tile: int = 0, temporal: int = 0, temporal_shape=None):
        """resident: 0 = the autotuner decides whether the tile-resident step is
        used, 1 = always, -1 = never (cdf_options.resident).  temporal: the
        same choice for two steps per launch (cdf_options.temporal);
        temporal_shape: (block_x, block_y, tile_y) of that kernel, or
        (block_x, block_y, tile_y, lanes) with lanes = 2 for the paired-lane
        kernel (cdf_options.temporal_lanes), or None."""
        self.pb = pb
        self.m, self.nx, self.ny = pb.m, pb.nx, pb.ny
        self.storage = storage
        self._structs = structs_from_problem(pb, storage, stream, block, phi_ref, p_ref_grad, resident,
                                             wait_timeout_s, test_stall_tile, temporal, temporal_shape)
        grid, dif, src, frc, bc, opt = self._structs
        self.h = cdf_lb_create(grid, pb.m, dif, pb.nu, src, frc, bc, opt)
        if init:
            self.init_moments(pb.phi0, pb.u0, pb.p0)

    def close(self):
        if getattr(self, "h", None):
            cdf_lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_moments(self, phi, u, p=None):
        cdf_lb_init_moments(self.h, np.ascontiguousarray(phi, np.float64), np.ascontiguousarray(u, np.float64),
                            None if p is None else np.ascontiguousarray(p, np.float64))

    def init_moments_device(self, fields):
        """fields: contiguous float32 CUDA tensor [m+3, ny, nx]."""
        assert fields.is_cuda and fields.dtype.itemsize == 4 and fields.is_contiguous()
        assert tuple(fields.shape) == (self.m + 3, self.ny, self.nx)
        cdf_lb_init_moments_device(self.h, fields.data_ptr())

    def step(self, n: int = 1):
        cdf_lb_step(self.h, n)

    def run_to_steady(self, tol: float, check_every: int = 1000, max_steps: int = 10 ** 7):
        st, steps, res = cdf_lb_run_to_steady(self.h, tol, check_every, max_steps)
        if st not in (CDF_OK, CDF_ENOTCONVERGED):
            _check(st)
        return st == CDF_OK, steps, res

    def moments(self) -> np.ndarray:
        out = np.empty((self.m + 3, self.ny, self.nx))
        cdf_lb_moments(self.h, out)
        return out

    def moments_device(self, out):
        assert out.is_cuda and out.is_contiguous() and out.dtype.itemsize == 4
        assert tuple(out.shape) == (self.m + 3, self.ny, self.nx)
        cdf_lb_moments_device(self.h, out.data_ptr())
        return out

    def mass(self) -> np.ndarray:
        out = np.empty(self.m)
        cdf_lb_mass(self.h, out)
        return out

    def populations(self):
        f = np.empty((self.m, 5, self.ny, self.nx))
        hf = np.empty((9, self.ny, self.nx))
        s = np.empty((self.m, self.ny, self.nx))
        cdf_lb_populations(self.h, f, hf, s)
        return f, hf, s

    def save(self, path: str):
        cdf_lb_save(self.h, path)

    def load(self, path: str):
        cdf_lb_load(self.h, path)

    def wall_transfer(self, side: int, D_CT: float, S_TC: float, T_wall: float, C_wall: float):
        """Average (Nu, Sh) through the west (0) or east (1) wall (cdf_lb_wall_transfer)."""
        Nu, Sh = cdf_lb_wall_transfer(self.h, side, D_CT, S_TC, T_wall, C_wall)
        return float(Nu), float(Sh)

    def info(self) -> cdf_info:
        return cdf_lb_get_info(self.h)

    @property
    def stream(self) -> int:
        return cdf_lb_stream(self.h)

    @property
    def t(self) -> int:
        return self.info().t


class SplitSolver:
    """One lattice split into `nslabs` slabs along y on the current device, with
    the halo exchange after every step (cdf_split_*); same results as Solver."""

    def __init__(self, pb: Problem, nslabs: int, stream: int = 0, block=None, init: bool = True):
        self.pb = pb
        self.m, self.nx, self.ny = pb.m, pb.nx, pb.ny
        grid, dif, src, frc, bc, opt = structs_from_problem(pb, "fp32", stream, block)
        self.h = cdf_split_create(grid, pb.m, dif, pb.nu, src, frc, bc, opt, nslabs)
        self.nslabs = nslabs
        if init:
            self.init_moments(pb.phi0, pb.u0, pb.p0)

    def close(self):
        if getattr(self, "h", None):
            cdf_split_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_moments(self, phi, u, p=None):
        cdf_split_init_moments(self.h, np.ascontiguousarray(phi, np.float64), np.ascontiguousarray(u, np.float64),
                               None if p is None else np.ascontiguousarray(p, np.float64))

    def step(self, n: int = 1):
        cdf_split_step(self.h, n)

    def moments(self) -> np.ndarray:
        out = np.empty((self.m + 3, self.ny, self.nx))
        cdf_split_moments(self.h, out)
        return out

    def mass(self) -> np.ndarray:
        out = np.empty(self.m)
        cdf_split_mass(self.h, out)
        return out

    def run_to_steady(self, tol: float, check_every: int = 1000, max_steps: int = 10 ** 7):
        st, steps, res = cdf_split_run_to_steady(self.h, tol, check_every, max_steps)
        if st not in (CDF_OK, CDF_ENOTCONVERGED):
            _check(st)
        return st == CDF_OK, steps, res

    def slabs(self):
        """[(y0, rows)] of the slabs."""
        return [cdf_split_slab(self.h, k)[1:] for k in range(self.nslabs)]


# ---- batched solver -------------------------------------------------------------------
def cdf_batch_create(count, grids, m, diffusion, nu, source, force, boundaries, phi_ref, p_ref_grad, options):
    h = ctypes.c_void_p()
    _check(load().cdf_batch_create(count, grids, m, diffusion, nu.ctypes.data_as(_DP), source, force, boundaries,
                                   phi_ref.ctypes.data_as(_DP), p_ref_grad.ctypes.data_as(_DP),
                                   ctypes.byref(options), ctypes.byref(h)))
    return h


def cdf_batch_init_moments(h, k, phi, u, p=None):
    _check(load().cdf_batch_init_moments(h, k, _dptr(phi), _dptr(u), None if p is None else _dptr(p)))


def cdf_batch_step(h, n):
    _check(load().cdf_batch_step(h, int(n)))


def cdf_batch_moments(h, k, out):
    _check(load().cdf_batch_moments(h, k, _dptr(out)))


def cdf_batch_init_moments_device(h, k: int, dev_ptr: int):
    _check(load().cdf_batch_init_moments_device(h, int(k), ctypes.c_void_p(dev_ptr)))


def cdf_batch_moments_device(h, k: int, dev_ptr: int):
    _check(load().cdf_batch_moments_device(h, int(k), ctypes.c_void_p(dev_ptr)))


def cdf_batch_snapshot(h):
    _check(load().cdf_batch_snapshot(h))


def cdf_batch_residuals(h, out: np.ndarray):
    _check(load().cdf_batch_residuals(h, _dptr(out)))


def cdf_batch_get_info(h) -> cdf_batch_info:
    info = cdf_batch_info()
    _check(load().cdf_batch_get_info(h, ctypes.byref(info)))
    return info


def cdf_batch_stream(h) -> int:
    return load().cdf_batch_stream(h) or 0


def cdf_batch_destroy(h):
    load().cdf_batch_destroy(h)


class BatchSolver:
    """Many lattices (same m and source kind, FP32) advanced by the persistent batched kernel."""

    def __init__(self, problems, stream: int = 0, tile=None, steps_per_launch: int = 0, barrier_timeout_s: float = 0.0,
                 test_unreachable_barrier: bool = False, init: bool = True, mode: int = 0, chain_tile_y: int = 0,
                 chain_lanes: int = 0):
        self.problems = list(problems)
        n = len(self.problems)
        m = self.problems[0].m
        grids = (cdf_grid * n)()
        dif = (cdf_diffusion * n)()
        src = (cdf_source * n)()
        frc = (cdf_force * n)()
        bcs = (cdf_boundaries * n)()
        nu = np.empty(n)
        phi_ref = np.empty((n, m))
        grad = np.empty((n, 2))
        for k, pb in enumerate(self.problems):
            if pb.m != m:
                raise ValueError("all instances need the same m")
            g, d, s_, f, b, o = structs_from_problem(pb)
            grids[k], dif[k], src[k], frc[k], bcs[k] = g, d, s_, f, b
            nu[k] = pb.nu
            phi_ref[k] = default_phi_ref(pb)
            grad[k] = default_p_ref_grad(pb)
        opt = cdf_batch_options()
        opt.storage, opt.rho0, opt.cuda_stream = 0, self.problems[0].rho0, stream or None
        if tile is not None:
            opt.tile_x, opt.tile_y = tile
        opt.steps_per_launch = steps_per_launch
        opt.barrier_timeout_s = barrier_timeout_s
        opt.test_unreachable_barrier = int(test_unreachable_barrier)
        opt.mode = mode
        opt.chain_tile_y = chain_tile_y
        opt.chain_lanes = chain_lanes
        self.h = cdf_batch_create(n, grids, m, dif, nu, src, frc, bcs, phi_ref, grad, opt)
        self.m = m
        if init:
            for k, pb in enumerate(self.problems):
                cdf_batch_init_moments(self.h, k, np.ascontiguousarray(pb.phi0, np.float64),
                                       np.ascontiguousarray(pb.u0, np.float64), np.ascontiguousarray(pb.p0, np.float64))

    def close(self):
        if getattr(self, "h", None):
            cdf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        cdf_batch_step(self.h, n)

    def moments(self, k: int) -> np.ndarray:
        pb = self.problems[k]
        out = np.empty((self.m + 3, pb.ny, pb.nx))
        cdf_batch_moments(self.h, k, out)
        return out

    def stack_floats(self, k: int = -1) -> int:
        """FP32 values of instance k's moment stack [m+3][ny][nx], or of all stacks
        back to back for k = -1 (the layout of the device moment calls)."""
        pbs = self.problems if k == -1 else [self.problems[k]]
        return sum((self.m + 3) * pb.nx * pb.ny for pb in pbs)

    def _check_device_buffer(self, t, k):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and t.numel() == self.stack_floats(k)):
            raise ValueError(f"expected a contiguous CUDA float32 tensor of {self.stack_floats(k)} values")

    def init_moments_device(self, fields, k: int = -1):
        """Initial state from device FP32 moment stacks (cdf_batch_init_moments_device)."""
        self._check_device_buffer(fields, k)
        cdf_batch_init_moments_device(self.h, k, fields.data_ptr())

    def moments_device(self, out, k: int = -1):
        """Current moments into device FP32 stacks (cdf_batch_moments_device)."""
        self._check_device_buffer(out, k)
        cdf_batch_moments_device(self.h, k, out.data_ptr())

    def info(self) -> cdf_batch_info:
        return cdf_batch_get_info(self.h)

    def residuals_after(self, n: int) -> np.ndarray:
        """Advance n steps and return each instance's residual over those steps."""
        cdf_batch_snapshot(self.h)
        self.step(n)
        out = np.empty(len(self.problems))
        cdf_batch_residuals(self.h, out)
        return out

    def run_to_steady(self, tol: float, check_every: int = 1000, max_steps: int = 10 ** 6):
        """Step all instances until every residual is below tol (or max_steps);
        returns (steps taken, residuals, step at which each instance first met tol)."""
        n = len(self.problems)
        first = np.full(n, -1, dtype=np.int64)
        taken = 0
        R = np.full(n, np.inf)
        while taken < max_steps:
            k = min(check_every, max_steps - taken)
            R = self.residuals_after(k)
            taken += k
            newly = (R < tol) & (first < 0)
            first[newly] = taken
            if (first >= 0).all():
                break
        return taken, R, first

    @property
    def stream(self) -> int:
        return cdf_batch_stream(self.h)


# ---- three-dimensional solver (include/cdf_lb3d.h) --------------------------------------------
def structs3_from_problem(pb, stream: int = 0, block=None, phi_ref=None, p_ref_grad=None):
    m = pb.m
    grid = cdf_grid3(pb.nx, pb.ny, pb.nz)
    dif = cdf_diffusion()
    dif.kind = {"const": 0, "chemotaxis": 1}[pb.dkind]
    for a in range(m):
        for b in range(m):
            dif.D[a * m + b] = float(pb.D[a, b])
    dif.chi, dif.c_star, dif.eps, dif.r_regularised = pb.chi, pb.c_star, pb.eps, int(pb.r_regularised)
    src = cdf_source()
    src.kind = {"none": 0, "const": 1, "consumption": 2}[pb.skind]
    src.k = pb.k
    frc = cdf_force3()
    for d in range(3):
        frc.g[d] = float(pb.g[d])
    frc.F0 = pb.F0
    for a in range(m):
        src.S[a] = float(pb.S[a])
        frc.beta[a] = float(pb.beta[a])
        frc.phi_ref[a] = float(pb.phi_ref[a])
    bc = cdf_boundaries3()
    for k, side in enumerate(pb.sides):
        cs = bc.side[k]
        cs.kind = {"periodic": 0, "wall": 1}[side.kind]
        cs.fluid = 0
        for a in range(m):
            cs.scalar[a] = {"noflux": 0, "dirichlet": 1}[side.scalar[a]]
            cs.value[a] = float(side.value[a])
    opt = cdf_options3()
    opt.rho0 = pb.rho0
    opt.cuda_stream = stream or None
    if phi_ref is None:
        phi_ref = []
        for a in range(m):
            lo, hi = float(pb.phi0[a].min()), float(pb.phi0[a].max())
            for side in pb.sides:
                if side.kind == "wall" and side.scalar[a] == "dirichlet":
                    lo, hi = min(lo, side.value[a]), max(hi, side.value[a])
            phi_ref.append(0.5 * (lo + hi))
    for a in range(m):
        opt.phi_ref[a] = float(phi_ref[a])
    if p_ref_grad is None:
        mag = pb.F0 + sum(float(pb.beta[a]) * (float(pb.phi0[a].mean()) - float(pb.phi_ref[a])) for a in range(m))
        p_ref_grad = [float(pb.g[d]) * mag for d in range(3)]
    for d in range(3):
        opt.p_ref_grad[d] = float(p_ref_grad[d])
    if block is not None:
        opt.block_x, opt.block_y = block
    return grid, dif, src, frc, bc, opt


class Solver3D:
    """One 3-D lattice (D3Q7 scalars, D3Q19 fluid) on the GPU behind include/cdf_lb3d.h."""

    def __init__(self, pb, stream: int = 0, block=None, init: bool = True):
        self.pb = pb
        self.m, self.nx, self.ny, self.nz = pb.m, pb.nx, pb.ny, pb.nz
        self._structs = structs3_from_problem(pb, stream, block)
        grid, dif, src, frc, bc, opt = self._structs
        h = ctypes.c_void_p()
        _check(load().cdf_lb3d_create(ctypes.byref(grid), pb.m, ctypes.byref(dif), pb.nu, ctypes.byref(src),
                                      ctypes.byref(frc), ctypes.byref(bc), ctypes.byref(opt), ctypes.byref(h)))
        self.h = h
        if init:
            self.init_moments(pb.phi0, pb.u0, pb.p0)

    def close(self):
        if getattr(self, "h", None):
            load().cdf_lb3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_moments(self, phi, u, p=None):
        f64 = lambda a: np.ascontiguousarray(a, np.float64)  # noqa: E731
        _check(load().cdf_lb3d_init_moments(self.h, _dptr(f64(phi)), _dptr(f64(u)),
                                            None if p is None else _dptr(f64(p))))

    def step(self, n: int = 1):
        _check(load().cdf_lb3d_step(self.h, int(n)))

    def run_to_steady(self, tol: float, check_every: int = 1000, max_steps: int = 10 ** 7):
        steps, res = ctypes.c_longlong(), ctypes.c_double()
        st = load().cdf_lb3d_run_to_steady(self.h, tol, check_every, max_steps, ctypes.byref(steps),
                                           ctypes.byref(res))
        if st not in (CDF_OK, CDF_ENOTCONVERGED):
            _check(st)
        return st == CDF_OK, steps.value, res.value

    def moments(self) -> np.ndarray:
        out = np.empty((self.m + 4, self.nz, self.ny, self.nx))
        _check(load().cdf_lb3d_moments(self.h, _dptr(out)))
        return out

    def mass(self) -> np.ndarray:
        out = np.empty(self.m)
        _check(load().cdf_lb3d_mass(self.h, _dptr(out)))
        return out

    def populations(self):
        f = np.empty((self.m, 7, self.nz, self.ny, self.nx))
        hf = np.empty((19, self.nz, self.ny, self.nx))
        _check(load().cdf_lb3d_populations(self.h, _dptr(f), _dptr(hf)))
        return f, hf

    def info(self) -> cdf_info3:
        out = cdf_info3()
        _check(load().cdf_lb3d_get_info(self.h, ctypes.byref(out)))
        return out

    @property
    def stream(self) -> int:
        return load().cdf_lb3d_stream(self.h)
