"""Benchmark of the fused lattice Boltzmann step (MLUPS and HBM roofline fraction).

Workload (default): the batched parameter sweep, 256 chemotaxis-plume instances
of uneven size (W ~ U{128..512}, H ~ U{64..256}, 13.2 M nodes in all), each with
its own chi, oxygen diffusivity and gravity scale; m = 2 (bacteria n, oxygen c),
FP32 populations, no-slip side and bottom walls, free-slip top with c = 1,
chemotactic cross term D_01 = -chi n r(c) with the step cut-off, consumption
S_c = -k n r(c), buoyancy -g n, n0 = 1 + 0.01 N(0, 1).  The state (2.6 GB) is far
above L2, so the step is an HBM measurement.  One benchmark step = `--lb-steps`
lattice time steps of every instance (by default about 0.1 s of work); L2 is
flushed (a 256 MiB write) between benchmark steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

With N = 1 the same JSON line also carries `extra`: the single 512 x 256 plume
(state in L2; its roofline is an effective figure, not an HBM one) and the
1024 x 1024 double-diffusive cavity, each timed in the same run.

Under torchrun each rank advances its own independent sweep (seed = rank):
weak scaling with no data-path collective; the barrier and the max-over-ranks
timing are the only collectives.  Rank 0 prints one JSON line.

value   -- whole-job MLUPS from CUDA events on the library's stream over the
           timed region (inputs resident in HBM).
e2e     -- the same metric through the C ABI with host buffers: every step
           uploads the initial moments from host memory, advances, and reads
           the moments back.
roofline -- the dominant kernel: the bytes it must move per launch (the state
           read once and written once: bytes per lattice update x nodes, per
           launch whatever the number of time steps the launch performs) over
           its average launch time, against the measured HBM copy bandwidth.
           A two-step launch moves those bytes once per two updates.
cpu_baseline -- the FP64 oracle as it stands on a bounded sample of the same
           workload on the host cores, with all cores (OpenMP over nodes and
           rows) and with one thread (rank 0, N = 1 only).
copy_pass -- context for the roofline: one pass of a plain device copy of as
           many bytes as one lattice step reads and writes.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2101_03055_gb300 import inputs as I  # noqa: E402

L2_FLUSH_BYTES = 256 << 20


def workload(name: str, rank: int):
    if name == "chemotaxis_plume_512x256":
        return I.chemotaxis_plume(512, 256, seed=rank, chi=0.5)
    if name == "chemotaxis_plume_2048x1024":
        return I.chemotaxis_plume(2048, 1024, seed=rank, chi=0.5)
    if name == "chemotaxis_plume_regularised_512x256":
        return I.chemotaxis_plume_regularised(512, 256)
    if name == "ddc_cavity_1024":
        return I.ddc_cavity(1024, Df=0.5, Sr=0.5)
    if name == "periodic_4096":
        return I.periodic_box(4096, 4096, seed=rank)
    if name == "periodic_2048":
        return I.periodic_box(2048, 2048, seed=rank)
    if name == "periodic3d_256":
        return I.periodic_box3d(256, seed=rank)
    if name == "periodic3d_128":
        return I.periodic_box3d(128, seed=rank)
    if name == "ddc_cavity3d_128":
        return I.ddc_cavity3d(128)
    if name == "cde_cellular_4096":
        return I.cde_cellular(4096, 4096, seed=rank)
    if name == "cde_cellular_2048":
        return I.cde_cellular(2048, 2048, seed=rank)
    if name == "batched_plume_sweep_256":
        return I.chemotaxis_plume_sweep(256, seed=rank)
    if name == "batched_plume_sweep_64":
        return I.chemotaxis_plume_sweep(64, seed=rank)
    raise SystemExit(f"unknown workload {name}")


def describe(name: str) -> str:
    return {
        "chemotaxis_plume_512x256": "chemotaxis-fluid plume 512x256, m=2 (n, c), FP32, walls + free-slip top, "
                                    "chi=0.5 step cut-off, consumption, buoyancy; n0 = 1 + 0.01 N(0,1)",
        "chemotaxis_plume_2048x1024": "chemotaxis-fluid plume 2048x1024 (the sweep's closures on one lattice above "
                                      "L2, for profiling the sweep's kernel)",
        "chemotaxis_plume_regularised_512x256": "chemotaxis-fluid plume of Sec. 3.1.2, 512x256: alpha=5, beta=5, "
                                                "delta=0.25, gamma=418, Sc=7700, regularised cut-off (eps = dx), "
                                                "periodic sides, n0 = 1 / 0.5 across a perturbed interface",
        "ddc_cavity_1024": "double-diffusive cavity 1024x1024 with Soret/Dufour (Df=Sr=0.5), Ra=1e5, Pr=0.7, Le=2, N=1",
        "periodic_4096": "periodic 4096x4096 cross-diffusion box (roofline grid)",
        "periodic_2048": "periodic 2048x2048 cross-diffusion box (profiling grid above L2)",
        "periodic3d_256": "3-D periodic 256^3 cross-diffusion box, m=2, D3Q7 scalars + D3Q19 fluid "
                          "(Taylor-Green initial velocity)",
        "periodic3d_128": "3-D periodic 128^3 cross-diffusion box (profiling size, 0.55 GB state > L2)",
        "ddc_cavity3d_128": "3-D double-diffusive cube 128^3 (hot/cold x walls, Ra=1e4, Pr=0.7, Le=2, N=1), "
                            "D3Q7 + D3Q19",
        "cde_cellular_4096": "Case 1 of Sec. 2.1: convection cross-diffusion (m=2) in a prescribed steady cellular "
                             "flow, 4096x4096, Dirichlet west/east walls, no fluid populations",
        "cde_cellular_2048": "Case 1 cellular flow at 2048x2048 (profiling size above L2)",
        "batched_plume_sweep_64": "64 chemotaxis-plume instances of the 256-instance sweep (profiling size)",
        "batched_plume_sweep_256": "256 chemotaxis-plume instances, W~U{128..512} x H~U{64..256} (13.2 M nodes), "
                                   "per-instance chi, D_c, gravity; execution mode (persistent kernel or graph of per-instance "
                                   "chains of one- or two-step launches) and tiles picked by the autotuner",
    }[name]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES_2D = ("lb_kernels.cu", "lb_device.cuh", "lb_internal.h", "lb_resident.cu")
KERNEL_SOURCES_3D = ("lb3d.cu",)


def kernel_source_hash(files=KERNEL_SOURCES_2D) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2101_03055_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_profile(workload_name: str, kernel: str):
    """The dominant kernel's ncu record for this workload (DRAM bytes per launch,
    issue-active fraction) from profiles/step_kernel_traffic.json, if it was taken
    on the current kernel source and for this kernel; else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(workload_name)
    files = KERNEL_SOURCES_3D if "3d" in workload_name else KERNEL_SOURCES_2D
    if not e or e.get("kernel_hash") != kernel_source_hash(files) or not kernel.startswith(e.get("kernel", "?")):
        return None
    return e


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 5 + k and s[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def moment_stack(pb) -> np.ndarray:
    """A problem's initial moments as the FP32 stack [m+3][ny][nx] of the device
    moment calls (phi_0..phi_{m-1}, u_x, u_y, p; p = 0 when the problem gives none)."""
    p = np.zeros((1, pb.ny, pb.nx)) if pb.p0 is None else np.asarray(pb.p0).reshape(1, pb.ny, pb.nx)
    return np.concatenate([np.asarray(pb.phi0).reshape(pb.m, pb.ny, pb.nx),
                           np.asarray(pb.u0).reshape(2, pb.ny, pb.nx), p]).astype(np.float32)


class E2EBuffers:
    """Pinned host buffers for the end-to-end step: the inputs in FP32 (written once,
    before timing, as a user's data pipeline would hand them over), and the result
    read back; device buffers of the same size."""

    def __init__(self, host_in: np.ndarray, device):
        import torch
        self.h_in = torch.from_numpy(np.ascontiguousarray(host_in.ravel())).pin_memory()
        self.h_out = torch.empty_like(self.h_in).pin_memory()
        self.d_in = torch.empty(self.h_in.numel(), dtype=torch.float32, device=device)
        self.d_out = torch.empty_like(self.d_in)
        self.nbytes = self.h_in.numel() * 4

    def upload(self):
        self.d_in.copy_(self.h_in, non_blocking=True)

    def download(self):
        import torch
        self.h_out.copy_(self.d_out, non_blocking=True)
        torch.cuda.current_stream().synchronize()  # the host holds the step's result


class _Single:
    """Uniform view of the single-lattice solver for the timing loops."""

    def __init__(self, lib, pb, storage, resident=0, block=None, temporal=0, temporal_shape=None):
        self.lib, self.pb = lib, pb
        self.s = lib.Solver(pb, storage=storage, resident=resident, block=block, temporal=temporal,
                            temporal_shape=temporal_shape)
        info = self.s.info()
        self.nodes, self.bytes_per_lup, self.storage = pb.nodes, info.bytes_per_lup, info.storage
        self.block = [info.block_x, info.block_y]
        self.m = pb.m
        self.resident = bool(info.resident)
        self.pair = bool(info.temporal) and not self.resident
        if self.pair:
            kname = ((f"step2_kernel_x2<{pb.m}>" if info.lanes == 2 else f"step2_kernel<{pb.m}>") if info.storage == 0
                     else f"step2_kernel_mr<{pb.m},{ {1: '__half', 2: '__nv_bfloat16'}[info.storage]}>")
            lanes = ", two nodes per thread on paired FP32 lanes" if info.lanes == 2 else ""
            self.kernel = (f"{kname} (two time steps per launch, CTAs of {info.block_x}x{info.block_y} "
                           f"threads, output tiles {info.tile_x}x{info.tile_y}{lanes})")
        elif self.resident:
            self.block = [info.tile_x, info.tile_y]
            self.kernel = (f"resident_kernel<{pb.m}> (tile-resident persistent step, {info.tiles} CTAs of "
                           f"{info.tile_x}x{info.tile_y} nodes)")
        else:
            if info.storage != 0:
                self.kernel = f"step_kernel_mr<{pb.m},{ {1: '__half', 2: '__nv_bfloat16'}[info.storage]}>"
            elif info.block_y == 0:
                self.kernel = f"step_kernel_flat<{pb.m},float> (flat launch, {info.block_x} threads per CTA)"
            else:
                self.kernel = f"step_kernel<{pb.m},float>"
        if getattr(pb, "case1", False):
            self.kernel = (f"step2_kernel_case1<{pb.m}> (prescribed velocity, no fluid; two time steps per launch, "
                           f"CTAs of {info.block_x}x{info.block_y} threads, output tiles {info.tile_x}x{info.tile_y})"
                           if self.pair else f"step_kernel_case1<{pb.m}> (prescribed velocity, no fluid)")

    def steps_per_launch(self, n):
        """Lattice steps per kernel launch inside step(n)."""
        return min(n, RESIDENT_MAX_STEPS) if self.resident else (2 if self.pair and n >= 2 else 1)

    def updates_per_pass(self, n):
        """Lattice updates per read + write of the state in global memory."""
        return self.steps_per_launch(n)

    def launches(self, n):
        """Kernels of this package launched by step(n)."""
        if self.resident:
            return -(-n // RESIDENT_MAX_STEPS)
        return n // 2 + n % 2 if self.pair else n

    stream = property(lambda self: self.s.stream)

    def step(self, n):
        self.s.step(n)

    def e2e_step(self, n):
        """Pinned FP32 moments up, initialisation, n steps, moments down (device calls)."""
        pb = self.pb
        if getattr(self, "io", None) is None:
            import torch
            self.io = E2EBuffers(moment_stack(pb), torch.device("cuda", torch.cuda.current_device()))
        shape = (pb.m + 3, pb.ny, pb.nx)
        self.io.upload()
        self.s.init_moments_device(self.io.d_in.view(shape))
        self.s.step(n)
        self.s.moments_device(self.io.d_out.view(shape))
        self.io.download()
        return 2 * self.io.nbytes


RESIDENT_MAX_STEPS = 4096  # steps per launch of the tile-resident step


class _Single3D:
    """The 3-D solver (D3Q7 scalars, D3Q19 fluid) for the timing loops."""

    def __init__(self, lib, pb, storage):
        if storage != "fp32":
            raise SystemExit("the 3-D solver stores FP32 populations")
        self.lib, self.pb = lib, pb
        self.s = lib.Solver3D(pb)
        info = self.s.info()
        self.nodes, self.bytes_per_lup, self.storage = pb.nodes, info.bytes_per_lup, 0
        self.block = [info.block_x, info.block_y]
        self.m = pb.m
        self.kernel = f"step3d_kernel<{pb.m}>"

    stream = property(lambda self: self.s.stream)

    def step(self, n):
        self.s.step(n)

    def steps_per_launch(self, n):
        return 1

    def updates_per_pass(self, n):
        return 1

    def launches(self, n):
        return n

    def e2e_step(self, n):
        pb = self.pb
        self.s.init_moments(pb.phi0, pb.u0, pb.p0)
        self.s.step(n)
        self.s.moments()
        return 2 * (pb.m + 4) * pb.nodes * 4


class _Batch:
    def __init__(self, lib, pbs, storage, mode=None, tile=None):
        if storage != "fp32":
            raise SystemExit("the batched solver stores FP32 populations")
        self.lib, self.pbs = lib, pbs
        if tile:  # (x, y) or, for mode 2, (x, y, tile height, nodes per thread)
            self.s = lib.BatchSolver(pbs, mode=mode or 0, tile=tile[:2], chain_tile_y=tile[2] if len(tile) > 2 else 0,
                                     chain_lanes=tile[3] if len(tile) > 3 else 0)
        else:
            self.s = lib.BatchSolver(pbs)
        info = self.s.info()
        self.nodes, self.bytes_per_lup, self.storage = info.nodes, info.bytes_per_lup, 0
        self.block = [info.tile_x, info.tile_y]
        self.m = pbs[0].m
        if info.mode == 1:
            self.block = [info.chain_block_x, info.chain_block_y]
            self.kernel = (f"step_kernel<{self.m},float> x {info.count} instance chains "
                           f"(graph of 32 steps over a 32-stream pool)")
        elif info.mode == 2:
            self.block = [info.chain_block_x, info.chain_block_y]
            name = "step2_kernel_x2" if info.chain_lanes == 2 else "step2_kernel"
            lanes = "two nodes per thread on paired FP32 lanes, " if info.chain_lanes == 2 else ""
            self.kernel = (f"{name}<{self.m}> x {info.count} instance chains (two time steps per launch, {lanes}"
                           f"CTAs of {info.chain_block_x}x{info.chain_block_y}, output tiles "
                           f"{info.chain_block_x - 2}x{info.chain_tile_y}; graph of 32 steps over a 32-stream pool)")
        else:
            self.kernel = (f"batch_kernel<{self.m}> (persistent, {info.grid_blocks} CTAs, "
                           f"{info.steps_per_launch} steps/launch)")
        self.mode = info.mode
        self.count = info.count
        self.spl = info.steps_per_launch

    def steps_per_launch(self, n):
        """Lattice steps per launch of the dominant kernel inside step(n) (chains:
        one or two lattice steps of one instance, counted here per whole sweep step)."""
        return {1: 1, 2: 2 if n >= 2 else 1}.get(self.mode, min(n, self.spl))

    def updates_per_pass(self, n):
        """Updates per read + write of the state: the persistent kernel passes over
        global memory every step; chains of two-step launches once per two steps."""
        return 2 if (self.mode == 2 and n >= 2) else 1

    def launches(self, n):
        if self.mode == 1:
            return n * self.count
        if self.mode == 2:
            return (n // 2 + n % 2) * self.count
        return -(-n // self.spl)

    stream = property(lambda self: self.s.stream)

    def step(self, n):
        self.s.step(n)

    def e2e_step(self, n):
        """Every instance's pinned FP32 moments up in one copy, initialisation, n steps,
        all moments down in one copy (the batch's device calls, k = -1)."""
        if getattr(self, "io", None) is None:
            import torch
            self.io = E2EBuffers(np.concatenate([moment_stack(pb).ravel() for pb in self.pbs]),
                                 torch.device("cuda", torch.cuda.current_device()))
        self.io.upload()
        self.s.init_moments_device(self.io.d_in)
        self.s.step(n)
        self.s.moments_device(self.io.d_out)
        self.io.download()
        return 2 * self.io.nbytes


class _Slab:
    """One rank's slab of a single lattice split along y (paper_2101_03055_gb300.slab):
    one step per launch and a halo exchange with the neighbouring ranks (NCCL
    send/recv of the crossing rows) after every step.  `nodes` counts the whole
    lattice: the job advances one lattice together (strong scaling)."""

    def __init__(self, lib, pb, storage, rank, world):
        if storage != "fp32":
            raise SystemExit("a split lattice stores FP32 populations")
        import torch
        from paper_2101_03055_gb300 import slab
        self.lib, self.pb = lib, pb
        self.s = slab.SlabSolver(pb, rank, world)
        info = lib.cdf_lb_get_info(self.s.h)
        self.nodes, self.bytes_per_lup, self.storage = pb.nodes, info.bytes_per_lup, 0
        self.block = [info.block_x, info.block_y]
        self.m = pb.m
        self.local_nodes = pb.nx * self.s.plan.rows
        self.kernel = (f"step_kernel_flat<{pb.m},float>" if info.block_y == 0 else f"step_kernel<{pb.m},float>") + \
            f" (slab of {self.s.plan.rows} of {pb.ny} rows, halo exchange after every step)"
        self._stream = torch.cuda.current_stream().cuda_stream

    stream = property(lambda self: self._stream)

    def step(self, n):
        self.s.step(n)

    def steps_per_launch(self, n):
        return 1

    def updates_per_pass(self, n):
        return 1

    def launches(self, n):
        return n

    def e2e_step(self, n):
        from paper_2101_03055_gb300 import slab
        pb, p = self.pb, self.s.plan
        rows = lambda f: slab.local_rows(f, p, pb.ny)  # noqa: E731
        self.lib.cdf_lb_init_moments(self.s.h, rows(pb.phi0), rows(pb.u0), None if pb.p0 is None else rows(pb.p0))
        self.s.exchange()
        self.s.step(n)
        self.s.moments()
        return 2 * (pb.m + 3) * pb.nx * p.lny * 4


def conv_line(N, H, W, Cin, Cout, reps, device, peak_tflops, peak_gbs):
    """The surrogate's 3x3 convolution (forward, bias + ReLU; tcgen05 path) on one
    layer shape: TFLOP/s from CUDA events over `reps` back-to-back launches, against
    the measured BF16 tensor peak, and the bytes it moves (input, weights, output)
    against the HBM copy bandwidth."""
    import torch
    from paper_2101_03055_gb300 import surrogate as sur
    g = torch.Generator(device="cpu").manual_seed(N * 131 + Cin)
    x = torch.randn((N, H, W, Cin), generator=g).to(device=device, dtype=torch.bfloat16)
    w = (torch.randn((Cout, 3, 3, Cin), generator=g) / (3 * Cin ** 0.5)).to(device=device, dtype=torch.bfloat16)
    b = torch.zeros(Cout, dtype=torch.float32, device=device)
    y = torch.empty((N, H, W, Cout), dtype=torch.bfloat16, device=device)
    def run():
        sur._call("cdf_nn_conv3x3_fwd", sur._p(x), sur._p(w), sur._p(b), sur._p(y), N, H, W, Cin, Cout, 1,
                  sur._stream())

    def timed(path):
        sur.set_tensor_path(path)
        for _ in range(3):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps
    us_sync = timed(2)  # the same MMAs with synchronously staged tiles, for comparison
    us = timed(1)
    flops = 2.0 * N * H * W * 9 * Cin * Cout
    nbytes = 2.0 * N * H * W * (Cin + Cout) + 2.0 * 9 * Cin * Cout
    tf = flops / us / 1e6
    return {"description": f"3x3 convolution forward (bias + ReLU), N={N} {H}x{W}, {Cin}->{Cout} channels, BF16 "
                           f"operands, FP32 accumulation in tensor memory",
            "value": tf, "unit": "TFLOP/s", "launch_us": us, "flops_per_launch": flops,
            "kernel": (f"conv3x3_slab_kernel<{min(Cout, 128 if Cin < 64 else 64)},{Cin // 8}> (no im2col copy, "
                       f"persistent)" if W % 128 == 0 and Cin in (16, 32, 64) else
                       f"conv3x3_tc_pipe_kernel<false,{Cout if Cout <= 128 else 128}>" if Cin >= 128 else
                       f"conv3x3_tc_kernel<false,{Cout if Cout <= 128 else 128}>"), "gpu_launches": 2 * reps,
            "synchronous_staging": {"kernel": f"conv3x3_tc_kernel<false,{Cout if Cout <= 128 else 128}>",
                                    "launch_us": us_sync, "value": flops / us_sync / 1e6},
            "roofline": {"bound": "tensor" if flops / nbytes > peak_tflops * 1e12 / (peak_gbs * 1e9) else "hbm",
                         "achieved": tf, "peak": peak_tflops, "unit": "TFLOP/s", "frac": tf / peak_tflops,
                         "traffic": None, "peak_source": "measured BF16 GEMM burst (MEASURED_PEAKS.json bf16_tflops)",
                         "bytes_per_launch": nbytes, "hbm_gbs": nbytes / us / 1e3,
                         "hbm_frac": nbytes / us / 1e3 / peak_gbs}}


def wgrad_line(N, H, W, Cin, Cout, reps, device, peak_tflops, peak_gbs):
    """The surrogate's 3x3 convolution weight and bias gradient (tcgen05 path: pixel
    splits into a workspace, then fixed-order sums) on one layer shape: TFLOP/s of
    the whole call (its four launches) from CUDA events over `reps` calls, against
    the measured BF16 tensor peak."""
    import torch
    from paper_2101_03055_gb300 import surrogate as sur
    g = torch.Generator(device="cpu").manual_seed(N * 137 + Cout)
    x = torch.randn((N, H, W, Cin), generator=g).to(device=device, dtype=torch.bfloat16)
    dy = torch.randn((N, H, W, Cout), generator=g).to(device=device, dtype=torch.bfloat16)
    dw = torch.zeros((Cout, 3, 3, Cin), dtype=torch.float32, device=device)
    db = torch.zeros(Cout, dtype=torch.float32, device=device)
    sur.set_tensor_path(1)
    for _ in range(3):
        sur.conv3x3_bwd_weight(x, dy, dw, db)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        sur.conv3x3_bwd_weight(x, dy, dw, db)
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / reps
    flops = 2.0 * N * H * W * 9 * Cin * Cout
    nbytes = 2.0 * N * H * W * (Cin + Cout) + 4.0 * 9 * Cin * Cout
    tf = flops / us / 1e6
    bn = 256 if Cout % 256 == 0 else (128 if Cout % 128 == 0 else (64 if Cout % 64 == 0 else 32))
    return {"description": f"3x3 convolution weight + bias gradient, N={N} {H}x{W}, {Cin}->{Cout} channels, BF16 "
                           f"operands, FP32 accumulation in tensor memory, pixel splits summed in a fixed order",
            "value": tf, "unit": "TFLOP/s", "launch_us": us, "flops_per_launch": flops,
            "kernel": f"conv3x3_wgrad_tc_kernel<{bn}>", "gpu_launches": 4 * reps,
            "roofline": {"bound": "tensor" if flops / nbytes > peak_tflops * 1e12 / (peak_gbs * 1e9) else "hbm",
                         "achieved": tf, "peak": peak_tflops, "unit": "TFLOP/s", "frac": tf / peak_tflops,
                         "traffic": None, "peak_source": "measured BF16 GEMM burst (MEASURED_PEAKS.json bf16_tflops)",
                         "bytes_per_launch": nbytes, "hbm_gbs": nbytes / us / 1e3,
                         "hbm_frac": nbytes / us / 1e3 / peak_gbs}}


def measured_tensor_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh)["bf16_tflops"])
    return 1900.0


def time_to_steady_line(n=256, cases=8, tol=1e-5, check_every=10_000, max_steps=3_000_000):
    """The surrogate's warm start against the start from rest on n x n double-diffusive
    cavities (held-out parameter draws, seed 1): lattice steps and GPU seconds until the
    stop test of Sec. 3.1.1 (R over check_every steps) drops below tol, each case and
    start on its own single-lattice solver.  The network is the committed one trained on 64^2
    steady states; its prediction is resampled to n x n.  None when no trained
    weights are present."""
    from paper_2101_03055_gb300 import surrogate as S
    path = S.default_model_path()
    if not os.path.exists(path):
        return None
    net = S.UNet(seed=0)
    net.load_state(dict(np.load(path)))
    prms = S.draw_parameters(cases, 1)
    res = S.time_to_steady(net, prms, n, 64, tol=tol, check_every=check_every, max_steps=max_steps)
    c, w = res["cold"]["first"], res["warm"]["first"]
    both = (c > 0) & (w > 0)
    med = lambda a: float(np.median(a)) if len(a) else None  # noqa: E731
    return {"description": f"{cases} held-out {n}x{n} double-diffusive cavities (Ra logU[1e4, 1e6], Nc U[-2, 2], "
                           f"Le U[1, 10], Sr, Df U[0, 0.5], Pr 0.7): steps until R < {tol:g} over {check_every} "
                           f"steps, from rest and from the U-Net prediction (trained on 64^2 steady states, "
                           f"resampled; fluid at rest, hydrostatic p)",
            "cases_reached_both": int(both.sum()), "cold_steps": c.tolist(), "warm_steps": w.tolist(),
            "median_cold_steps": med(c[both]), "median_warm_steps": med(w[both]),
            "median_ratio_warm_over_cold": med(w[both] / c[both]),
            "cold_s": res["cold"]["seconds"].round(3).tolist(), "warm_s": res["warm"]["seconds"].round(3).tolist(),
            "median_cold_s": med(res["cold"]["seconds"][both]), "median_warm_s": med(res["warm"]["seconds"][both]),
            "median_ratio_s_warm_over_cold": med(res["warm"]["seconds"][both] / res["cold"]["seconds"][both]),
            "timing": "wall clock around each case's cdf_lb_run_to_steady on its own single-lattice solver "
                      "(device synchronised on both sides)",
            "max_steps": max_steps}


CONV_SHAPES = {"unet_conv3x3_256x256x32": (16, 256, 256, 32, 32), "unet_conv3x3_32x32x256": (16, 32, 32, 256, 256)}
WGRAD_SHAPES = {"unet_wgrad3x3_256x256x32": (16, 256, 256, 32, 32),
                "unet_wgrad3x3_32x32x256": (16, 32, 32, 256, 256)}


def copy_pass(nbytes: int, device) -> dict:
    """Time of one device copy of nbytes / 2 bytes (read + write = nbytes)."""
    import torch
    full = max(16, nbytes // 2 // 4)
    n = min(full, 1 << 27)  # at most 512 MiB a buffer; the time is scaled to the full size
    a = torch.zeros(n, dtype=torch.float32, device=device)
    b = torch.zeros_like(a)
    s = torch.cuda.Stream(device=device)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        for _ in range(3):
            b.copy_(a)
            a.copy_(b)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            for _ in range(16):
                b.copy_(a)
                a.copy_(b)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record(s)
        for _ in range(reps):
            g.replay()
        e1.record(s)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / (32 * reps) * full / n
    del a, b, g
    return {"us": us, "bytes": 8 * full, "gbs": 8 * full / us / 1e3,
            "what": "one torch copy of a state-sized buffer (bytes read + written = one lattice step's)"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def all_max(x: float, world: int, device) -> float:
    """Max of x over ranks (the whole job is as slow as its slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank: int, lb_steps: int, bench_steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: every rank advances its own instance (weak scaling),
    so the job processed world x nodes x steps lattice updates in the slowest rank's time."""
    return world * nodes_per_rank * lb_steps * bench_steps / (max_ms * 1e-3) / 1e6


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _oracle_sim(pb):
    """The FP64 oracle (2-D or 3-D) of a problem, as it stands."""
    if isinstance(pb, I.Problem3D):
        from oracle import oracle3d
        oracle3d.build()
        return oracle3d.Sim(pb)
    import oracle
    oracle.build()
    return oracle.OracleSim(pb)


def _dims(pb) -> str:
    return f"{pb.nx}x{pb.ny}x{pb.nz}" if isinstance(pb, I.Problem3D) else f"{pb.nx}x{pb.ny}"


def _oracle_threads(pb, n: int) -> int:
    if isinstance(pb, I.Problem3D):
        return 1  # the 3-D oracle runs one thread
    import oracle
    return oracle.set_threads(n)


def _time_oracle(pbs, budget_s: float):
    """Steps of the oracle on the problems `pbs` (round robin, about budget_s of
    work); returns (lattice updates, seconds, steps per problem)."""
    sims = [_oracle_sim(pb) for pb in pbs]
    t0 = time.perf_counter()
    for o in sims:
        o.step(1)
    per = time.perf_counter() - t0
    n = max(1, int(budget_s / max(per, 1e-9)))
    t0 = time.perf_counter()
    for o in sims:
        o.step(n)
    dt = time.perf_counter() - t0
    return sum(pb.nodes for pb in pbs) * n, dt, n


def _sample(wl):
    """The oracle's sample of a workload: a batched sweep's first eight instances."""
    return wl[:8] if isinstance(wl, list) else [wl]


def cpu_baseline(wl, budget_s: float = 10.0):
    """The FP64 oracle as it stands on a bounded sample of the workload: with all
    host cores (OpenMP over the node and row loops; same results) and with one
    thread, each for about `budget_s`."""
    pbs = _sample(wl)
    dims = ", ".join(_dims(pb) for pb in pbs[:3]) + (", ..." if len(pbs) > 3 else "")
    cores = _oracle_threads(pbs[0], 0)
    lups, dt, n = _time_oracle(pbs, budget_s)
    _oracle_threads(pbs[0], 1)
    lups1, dt1, n1 = _time_oracle(pbs, budget_s)
    return {"value": lups / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": f"{n} time steps of {len(pbs)} lattice(s) ({dims}; FP64, {cores} threads, "
                      f"{lups / 1e6:.1f} M lattice updates, {dt:.1f} s)",
            "single_thread": {"value": lups1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                              "sample": f"{n1} time steps of the same lattices ({lups1 / 1e6:.1f} M lattice "
                                        f"updates, {dt1:.1f} s)"}}


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on all host cores, same metric and workload
    (a batched sweep: a sample of its instances)."""
    if rank != 0:
        return
    wl = workload(args.workload, 0)
    pbs = _sample(wl)
    cores = _oracle_threads(pbs[0], 0)
    sims = [_oracle_sim(pb) for pb in pbs]
    per_step_budget = 4.0
    t0 = time.perf_counter()
    for o in sims:
        o.step(1)
    per = time.perf_counter() - t0
    n = max(1, int(per_step_budget / max(per, 1e-9)))
    for _ in range(args.warmup):
        for o in sims:
            o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for o in sims:
            o.step(n)
    dt = time.perf_counter() - t0
    nodes = sum(pb.nodes for pb in pbs)
    value = nodes * n * args.steps / dt / 1e6
    dims = ", ".join(_dims(pb) for pb in pbs[:3]) + (", ..." if len(pbs) > 3 else "")
    line = {
        "impl": "reference", "metric": "MLUPS (lattice updates per second, millions)", "value": value,
        "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": describe(args.workload),
                   "sample_lattices": len(pbs), "sample_nodes": nodes, "m": pbs[0].m, "lb_steps_per_step": n},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{n} time steps of {len(pbs)} lattice(s) ({dims}) per benchmark step, "
                                   f"FP64, {cores} threads"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def make_runner(lib, name, rank, args, fixed=True):
    """The solver of workload `name` (the options of the command line apply to the
    main workload only: fixed = True)."""
    wl = workload(name, rank)
    if isinstance(wl, list):
        if fixed and args.batch_tile:
            tile = tuple(int(v) for v in args.batch_tile.split(","))
            return _Batch(lib, wl, args.storage, args.batch_mode, tile)
        return _Batch(lib, wl, args.storage if fixed else "fp32")
    if isinstance(wl, I.Problem3D):
        return _Single3D(lib, wl, args.storage if fixed else "fp32")
    if not fixed:
        return _Single(lib, wl, "fp32")
    block = tuple(int(v) for v in args.block.split(",")) if args.block else None
    tshape = tuple(int(v) for v in args.temporal_shape.split(",")) if args.temporal_shape else None
    return _Single(lib, wl, args.storage, args.resident, block, args.temporal, tshape)


def default_lb_steps(nodes: int) -> int:
    """About 0.1 s of lattice updates at ~30 GLUPS, a multiple of 32, at most 20000."""
    return int(min(20000, max(32, 3e9 / nodes)) // 32 * 32)


def time_runner(runner, S, K, W, flush, device, world):
    """K timed benchmark steps of S lattice steps (after W untimed ones), L2 flushed
    between them; returns the max over ranks of the summed event times (ms)."""
    import torch
    lib_stream = torch.cuda.ExternalStream(runner.stream, device=device)
    for _ in range(W):
        runner.step(S)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    barrier(world)
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()  # evict L2 between benchmark steps
        torch.cuda.synchronize()
        ev[k][0].record(lib_stream)
        runner.step(S)
        ev[k][1].record(lib_stream)
    torch.cuda.synchronize()
    barrier(world)
    kernel_ms = sum(a.elapsed_time(b) for a, b in ev)
    return all_max(kernel_ms, world, device)


L2_BYTES = 126e6  # GB300 L2, less a margin


def roofline_of(runner, name, S, K, t_ms, peak, peak_kind):
    """The dominant kernel's roofline: bytes it must move per launch (state read and
    written once) over its launch time, against the measured copy bandwidth."""
    nodes = getattr(runner, "local_nodes", runner.nodes)  # a slab's kernel moves its own rows
    upp = runner.updates_per_pass(S)
    state_bytes = runner.bytes_per_lup * nodes
    pass_s = t_ms * 1e-3 / (S * K) * upp  # time of one pass over the state
    achieved = state_bytes / pass_s / 1e9
    l2 = state_bytes < L2_BYTES  # the buffer read and the buffer written both fit in L2
    rec = recorded_profile(name, runner.kernel)
    r = {"bound": "effective (L2-resident)" if l2 else "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": achieved / peak, "traffic": None if rec is None else rec["dram_bytes_per_launch"],
         "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
         "bytes_per_launch": state_bytes, "bytes_per_lup": runner.bytes_per_lup,
         "lattice_updates_per_pass": upp, "kernel": runner.kernel,
         "launch_us": pass_s * 1e6 / max(1, runner.steps_per_launch(S) // upp),
         "lattice_steps_per_launch": runner.steps_per_launch(S)}
    if l2:
        r["l2_resident"] = True
        r["note"] = ("the state stays in the 129 MB L2 inside a benchmark step: achieved is the algorithmic "
                     "bytes over the launch time, an effective figure, not HBM traffic")
    if rec is not None and "issue_active" in rec:
        r["limiter"] = "instruction issue"
        r["issue_active"] = rec["issue_active"]
    return r


EXTRA_WORKLOADS = ("chemotaxis_plume_512x256", "ddc_cavity_1024", "chemotaxis_plume_regularised_512x256")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_plume_sweep_256")
    ap.add_argument("--lb-steps", type=int, default=None,
                    help="lattice time steps per benchmark step (default: about 0.1 s of work, a multiple "
                         "of 32, at most 20000)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--resident", type=int, default=0, choices=[-1, 0, 1],
                    help="tile-resident step: 0 = the autotuner decides, 1 = always, -1 = never")
    ap.add_argument("--temporal", type=int, default=0, choices=[-1, 0, 1],
                    help="two time steps per launch: 0 = the autotuner decides, 1 = always, -1 = never")
    ap.add_argument("--temporal-shape", default=None,
                    help="'X,Y,TH': CTA shape and output tile height of the two-step kernel (with --temporal 1); "
                         "default: autotuned")
    ap.add_argument("--block", default=None,
                    help="CTA shape 'X,Y' of the single-lattice step (Y = 0: flat launch); default: autotuned")
    ap.add_argument("--split", default="none", choices=["none", "slab"],
                    help="slab: one single lattice split along y over the ranks, halo exchange through NCCL "
                         "after every step (strong scaling); none: every rank its own instance (weak scaling)")
    ap.add_argument("--batch-mode", type=int, default=0, choices=[0, 1, 2],
                    help="with --batch-tile: the batched solver's mode (0 persistent, 1 chains, 2 two-step chains)")
    ap.add_argument("--batch-tile", default=None,
                    help="'X,Y': tile (mode 0) or CTA shape (modes 1, 2) of the batched solver, 'X,Y,TH,LANES' in "
                         "mode 2 (tile height, nodes per thread); default: autotuned")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workloads of the N = 1 line")
    ap.add_argument("--e2e-steps", type=int, default=3)
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    from paper_2101_03055_gb300 import build, lib
    build.build()
    if args.workload in CONV_SHAPES:  # one convolution layer of the surrogate, alone (profiling)
        peak, _ = measured_peaks()
        line = conv_line(*CONV_SHAPES[args.workload], max(1, args.steps), device, measured_tensor_peak(), peak)
        line.update({"metric": "TFLOP/s of the 3x3 convolution", "n_gpus": 1, "steps": args.steps,
                     "config": {"workload": args.workload}, "dtype": "bf16", "data": "synthetic"})
        print(json.dumps(line), flush=True)
        return
    if args.workload in WGRAD_SHAPES:  # the weight gradient of one convolution layer, alone (profiling)
        peak, _ = measured_peaks()
        line = wgrad_line(*WGRAD_SHAPES[args.workload], max(1, args.steps), device, measured_tensor_peak(), peak)
        line.update({"metric": "TFLOP/s of the 3x3 convolution weight gradient", "n_gpus": 1, "steps": args.steps,
                     "config": {"workload": args.workload}, "dtype": "bf16", "data": "synthetic"})
        print(json.dumps(line), flush=True)
        return
    if args.split == "slab":
        wl = workload(args.workload, 0)  # one lattice for the whole job
        if not isinstance(wl, I.Problem):
            raise SystemExit("--split slab needs a single 2-D lattice workload")
        runner = _Slab(lib, wl, args.storage, rank, world)
    else:
        runner = make_runner(lib, args.workload, rank, args)
    nodes = runner.nodes
    S = args.lb_steps if args.lb_steps is not None else default_lb_steps(nodes)
    K, W = args.steps, args.warmup
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        t_ms = time_runner(runner, S, K, W, flush, device, world)
        wall = time.perf_counter() - wall0
    strong = args.split == "slab"
    value = job_mlups(nodes, S, K, 1 if strong else world, t_ms)

    # e2e: pinned FP32 moments copied in, S steps through the C ABI, moments copied out to
    # pinned host memory and waited for, every step (the first call allocates the buffers)
    E = max(1, args.e2e_steps)
    runner.e2e_step(S)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    moved = 0
    for _ in range(E):
        moved = runner.e2e_step(S)
    torch.cuda.synchronize()
    e2e_s = all_max(time.perf_counter() - t0, world, device)
    e2e_value = (1 if strong else world) * nodes * S * E / e2e_s / 1e6
    stage_bytes = moved // 2

    # context for an L2-resident state: the time of a plain device copy of one step's bytes
    cp = copy_pass(int(runner.bytes_per_lup * nodes), device) if runner.bytes_per_lup * nodes < L2_BYTES else None
    peak, peak_kind = measured_peaks()
    roof = roofline_of(runner, args.workload, S, K, t_ms, peak, peak_kind)
    launches = runner.launches(S) * K
    state_bytes = nodes * runner.bytes_per_lup / 2
    block, m, storage = runner.block, runner.m, runner.storage

    extra, tts = {}, None
    if world == 1 and not strong and not args.no_extra and args.workload not in EXTRA_WORKLOADS:
        del runner
        torch.cuda.synchronize()
        for name in EXTRA_WORKLOADS:
            r = make_runner(lib, name, rank, args, fixed=False)
            Sx, Kx = default_lb_steps(r.nodes), min(K, 5)
            with ClockSampler(local) as clk_x:
                tx = time_runner(r, Sx, Kx, max(3, min(W, 3)), flush, device, 1)
            extra[name] = {
                "description": describe(name), "value": job_mlups(r.nodes, Sx, Kx, 1, tx), "unit": "MLUPS",
                "ms_per_step": tx / Kx, "steps": Kx, "lb_steps_per_step": Sx, "nodes": r.nodes,
                "gpu_launches": r.launches(Sx) * Kx, "clocks": clk_x.summary(),
                "roofline": roofline_of(r, name, Sx, Kx, tx, peak, peak_kind)}
            del r
            torch.cuda.synchronize()
        for name, shape in CONV_SHAPES.items():
            extra[name] = conv_line(*shape, 50, device, measured_tensor_peak(), peak)
        for name, shape in WGRAD_SHAPES.items():
            extra[name] = wgrad_line(*shape, 50, device, measured_tensor_peak(), peak)
        tts = time_to_steady_line()

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    line = {
        "metric": "MLUPS (lattice updates per second, millions)",
        "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "strong" if strong else "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": describe(args.workload), "nodes": nodes,
                   "storage": {0: "f32", 1: "f16", 2: "bf16"}[storage] + " populations (arithmetic in f32)",
                   "m": m, "lb_steps_per_step": S, "block": block,
                   "l2": "flushed between benchmark steps (256 MiB write); the state is L2-resident "
                         "within a step" if 2 * state_bytes < L2_BYTES else
                         "flushed between benchmark steps; working set larger than L2",
                   "parallelism": (f"slabs x{world} (one lattice split along y, halo exchange after every step)"
                                   if strong else f"replicas x{world} (independent instances, seed = rank)")},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": stage_bytes,
                "d2h_bytes_per_step": stage_bytes, "steps": E},
        "roofline": roof,
        **({"copy_pass": cp} if cp else {}),
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s": wall,
    }
    if extra:
        line["extra"] = extra
    if world == 1 and not strong and not args.no_extra and tts is not None:
        line["time_to_steady"] = tts
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(workload(args.workload, 0))
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
