"""CPU checks of the C ABI: the library loads, exports every function that
include/cdf_lb.h declares, the ctypes structs match the C layout, and
cdf_lb_create rejects invalid parameter sets before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2101_03055_gb300 import build, inputs as I, lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


@pytest.fixture(scope="module")
def L():
    build.build()
    return lib.load()


def declared_functions():
    names = set()
    for hp in HEADERS:
        text = open(hp).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cdf_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_function(L):
    names = declared_functions()
    assert "cdf_lb_create" in names and "cdf_lb_step" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = names - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for n in names:
        assert hasattr(L, n)


def test_binding_covers_the_header():
    from paper_2101_03055_gb300 import surrogate
    bound = set(lib.SIGNATURES) | set(surrogate.NN_SIGNATURES) | {"cdf_lb_last_error", "cdf_nn_last_error"}
    assert declared_functions() <= bound, sorted(declared_functions() - bound)


def test_struct_layout_matches_c(tmp_path):
    structs = ["cdf_grid", "cdf_diffusion", "cdf_source", "cdf_force", "cdf_side", "cdf_boundaries",
               "cdf_options", "cdf_info", "cdf_grid3", "cdf_force3", "cdf_boundaries3", "cdf_options3", "cdf_info3",
               "cdf_batch_options", "cdf_batch_info"]
    src = tmp_path / "probe.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cdf_lb.h"', '#include "cdf_lb3d.h"',
             "int main(void){"]
    for s in structs:
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
    lines.append('printf("opt.cuda_stream %zu\\n", offsetof(cdf_options, cuda_stream));')
    lines.append('printf("info.bytes_per_lup %zu\\n", offsetof(cdf_info, bytes_per_lup));')
    lines.append('printf("opt.prescribed_velocity %zu\\n", offsetof(cdf_options, prescribed_velocity));')
    lines.append('printf("opt3.block_y %zu\\n", offsetof(cdf_options3, block_y));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for s in structs:
        assert int(got[s]) == ctypes.sizeof(getattr(lib, s)), s
    assert int(got["opt.cuda_stream"]) == lib.cdf_options.cuda_stream.offset
    assert int(got["info.bytes_per_lup"]) == lib.cdf_info.bytes_per_lup.offset
    assert int(got["opt.prescribed_velocity"]) == lib.cdf_options.prescribed_velocity.offset
    assert int(got["opt3.block_y"]) == lib.cdf_options3.block_y.offset


def _create_status(pb, **kw):
    grid, dif, src, frc, bc, opt = lib.structs_from_problem(pb)
    for k, v in kw.items():
        if "__" not in k:
            continue
        obj, field = k.split("__")
        target = {"grid": grid, "dif": dif, "src": src, "opt": opt}[obj]
        setattr(target, field, v)
    h = ctypes.c_void_p()
    m = kw.get("m", pb.m)
    st = lib.load().cdf_lb_create(ctypes.byref(grid), m, ctypes.byref(dif), kw.get("nu", pb.nu), ctypes.byref(src),
                                  ctypes.byref(frc), ctypes.byref(bc), ctypes.byref(opt), ctypes.byref(h))
    return st, h.value, lib.cdf_lb_last_error()


@pytest.mark.parametrize("case", ["nu", "m0", "m5", "grid", "D", "chemo_m1", "storage", "rho0", "block",
                                  "periodic_mismatch", "dirichlet_on_periodic", "eps", "temporal_lanes",
                                  "lanes_without_shape", "block_lanes", "block_lanes_not_flat", "block_lanes_m3"])
def test_create_rejects_invalid_parameters(L, case):
    pb = I.cross_diffusion_taylor_green(16, 16)
    if case == "nu":
        pb = pb.replace(nu=0.0)
    elif case == "D":
        pb = pb.replace(D=np.array([[-0.3, 0.0], [0.0, 0.1]]))
    elif case == "chemo_m1":
        pb = I.Problem("x", 8, 8, 1, [[0.1]], 0.1, dkind="chemotaxis", chi=0.1)
    elif case == "periodic_mismatch":
        pb = pb.replace(west=I.wall_side(2))
    elif case == "dirichlet_on_periodic":
        pb = pb.replace(west=I.Side("periodic", "noslip", ["dirichlet", "noflux"], [1.0, 0.0]))
    kw = {"m0": {"m": 0}, "m5": {"m": 5}, "grid": {"grid__nx": 0}, "storage": {"opt__storage": 7},
          "rho0": {"opt__rho0": 0.0}, "block": {"opt__block_x": 48, "opt__block_y": 2},
          "eps": {"dif__r_regularised": 1, "dif__eps": 0.0},
          # nodes per thread of the paired-lane kernels: 0, 1 or 2, and 2 only with a given shape
          "temporal_lanes": {"opt__temporal_lanes": 3},
          "lanes_without_shape": {"opt__temporal_lanes": 2},
          "block_lanes": {"opt__block_x": 128, "opt__block_y": 0, "opt__block_lanes": 3},
          "block_lanes_not_flat": {"opt__block_x": 128, "opt__block_y": 1, "opt__block_lanes": 2},
          "block_lanes_m3": {"m": 3, "opt__block_x": 128, "opt__block_y": 0, "opt__block_lanes": 2}}.get(case, {})
    if case == "nu":
        kw["nu"] = 0.0
    st, h, msg = _create_status(pb, **kw)
    assert st == lib.CDF_EINVAL, (case, st, msg)
    assert h is None
    assert msg
    if "lanes" in case:  # refused for that reason, before any device call
        assert "lanes" in msg, msg


def test_null_arguments(L):
    assert L.cdf_lb_step(None, 1) == lib.CDF_EINVAL
    assert L.cdf_lb_moments(None, None) == lib.CDF_EINVAL
    assert L.cdf_lb_get_info(None, None) == lib.CDF_EINVAL
    L.cdf_lb_destroy(None)
