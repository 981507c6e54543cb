"""Convolutional surrogate that warm-starts steady solves of the double-diffusive
cavity (Sec. 3.2 setup), trained on steady states the solver generates itself.

A 4-level U-Net (base 32 channels: 32-64-128-256, two 3x3 convolutions with
ReLU per level, 2x2 average pooling, nearest upsampling with skip
concatenation, 1x1 head) maps seven input planes -- log10 Ra, Nc, Le, Sr, Df
and the node coordinates -- to (u_x, u_y, T, C).  Every layer runs in this
package's BF16 kernels (include/cdf_nn.h; tensor cores, FP32 accumulation);
PyTorch only allocates device memory.  The prediction initialises
cdf_lb_init_moments_device, and the lattice Boltzmann residual decides
convergence as for a start from rest.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import inputs as I
from . import lib

NN_SIGNATURES = {
    "cdf_nn_conv3x3_fwd": [ctypes.c_void_p] * 4 + [ctypes.c_int] * 6 + [ctypes.c_void_p],
    "cdf_nn_conv3x3_bwd_data": [ctypes.c_void_p] * 3 + [ctypes.c_int] * 5 + [ctypes.c_void_p],
    "cdf_nn_conv3x3_bwd_weight": [ctypes.c_void_p] * 4 + [ctypes.c_int] * 5 + [ctypes.c_void_p, ctypes.c_longlong,
                                                                              ctypes.c_void_p],
    "cdf_nn_relu_bwd": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p],
    "cdf_nn_avgpool2_fwd": [ctypes.c_void_p] * 2 + [ctypes.c_int] * 4 + [ctypes.c_void_p],
    "cdf_nn_avgpool2_bwd": [ctypes.c_void_p] * 2 + [ctypes.c_int] * 4 + [ctypes.c_void_p],
    "cdf_nn_upsample2_fwd": [ctypes.c_void_p] * 2 + [ctypes.c_int] * 6 + [ctypes.c_void_p],
    "cdf_nn_upsample2_bwd": [ctypes.c_void_p] * 2 + [ctypes.c_int] * 6 + [ctypes.c_void_p],
    "cdf_nn_copy_channels": [ctypes.c_void_p] * 2 + [ctypes.c_longlong] + [ctypes.c_int] * 6 + [ctypes.c_void_p],
    "cdf_nn_head_fwd": [ctypes.c_void_p] * 4 + [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "cdf_nn_head_bwd": [ctypes.c_void_p] * 6 + [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "cdf_nn_mse": [ctypes.c_void_p] * 4 + [ctypes.c_longlong, ctypes.c_void_p],
    "cdf_nn_adam": [ctypes.c_void_p] * 5 + [ctypes.c_longlong] + [ctypes.c_float] * 4 + [ctypes.c_longlong,
                                                                                         ctypes.c_void_p],
    "cdf_nn_set_tensor_path": [ctypes.c_int],
    "cdf_nn_error_flag": [ctypes.POINTER(ctypes.c_int)],
    "cdf_nn_conv3x3_bwd_weight_workspace": [ctypes.c_int] * 5,
}
NN_RESTYPES = {"cdf_nn_conv3x3_bwd_weight_workspace": ctypes.c_longlong}
_nn = None


def nn_lib():
    global _nn
    if _nn is None:
        L = lib.load()
        for name, args in NN_SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = NN_RESTYPES.get(name, ctypes.c_int)
        L.cdf_nn_last_error.restype = ctypes.c_char_p
        _nn = L
    return _nn


def set_tensor_path(tcgen05):
    """Convolutions on the 5th-generation tensor cores (True or 1, the default: the faster
    staging per layer; 2: synchronous staging; 3: persistent warp-specialised forward;
    4: the forward without im2col copy where the shape allows it) or on the warp-level
    MMA kernels (False or 0)."""
    _call("cdf_nn_set_tensor_path", int(tcgen05))


def tensor_error_flag() -> int:
    """1 if a bounded wait of a tcgen05 convolution ever ran out."""
    v = ctypes.c_int(0)
    _call("cdf_nn_error_flag", ctypes.byref(v))
    return v.value


def _call(name, *args):
    st = getattr(nn_lib(), name)(*args)
    if st != 0:
        raise RuntimeError(f"{name}: {nn_lib().cdf_nn_last_error().decode()}")


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream or None)


# ---- thin same-name wrappers of include/cdf_nn.h ----------------------------------------
def conv3x3_fwd(x, w, b, relu):
    import torch
    N, H, W, Cin = x.shape
    Cout = w.shape[0]
    y = torch.empty((N, H, W, Cout), dtype=torch.bfloat16, device=x.device)
    _call("cdf_nn_conv3x3_fwd", _p(x), _p(w), _p(b), _p(y), N, H, W, Cin, Cout, int(relu), _stream())
    return y


def conv3x3_bwd_data(dy, w, Cin):
    import torch
    N, H, W, Cout = dy.shape
    dx = torch.empty((N, H, W, Cin), dtype=torch.bfloat16, device=dy.device)
    _call("cdf_nn_conv3x3_bwd_data", _p(dy), _p(w), _p(dx), N, H, W, Cin, Cout, _stream())
    return dx


_workspace = {}


def conv3x3_bwd_weight(x, dy, dw, db):
    """Accumulates the weight and bias gradients; the split partial sums go to a
    device workspace kept per device (grown to the largest shape seen)."""
    import torch
    N, H, W, Cin = x.shape
    Cout = dy.shape[3]
    need = int(nn_lib().cdf_nn_conv3x3_bwd_weight_workspace(N, H, W, Cin, Cout))
    ws = _workspace.get(x.device)
    if ws is None or ws.numel() * 4 < need:
        ws = torch.empty((max(need, 4) + 3) // 4, dtype=torch.float32, device=x.device)
        _workspace[x.device] = ws
    _call("cdf_nn_conv3x3_bwd_weight", _p(x), _p(dy), _p(dw), _p(db), N, H, W, Cin, Cout, _p(ws),
          ws.numel() * 4, _stream())


def relu_bwd(d, y):
    _call("cdf_nn_relu_bwd", _p(d), _p(y), d.numel(), _stream())


def avgpool2_fwd(x):
    import torch
    N, H, W, C = x.shape
    y = torch.empty((N, H // 2, W // 2, C), dtype=torch.bfloat16, device=x.device)
    _call("cdf_nn_avgpool2_fwd", _p(x), _p(y), N, H, W, C, _stream())
    return y


def avgpool2_bwd(dy, H, W):
    import torch
    N, _, _, C = dy.shape
    dx = torch.empty((N, H, W, C), dtype=torch.bfloat16, device=dy.device)
    _call("cdf_nn_avgpool2_bwd", _p(dy), _p(dx), N, H, W, C, _stream())
    return dx


def upsample2_into(x, y, coff):
    N, H, W, C = x.shape
    _call("cdf_nn_upsample2_fwd", _p(x), _p(y), N, H, W, C, y.shape[3], coff, _stream())


def upsample2_bwd_from(dy, C, coff):
    import torch
    N, H2, W2, Cy = dy.shape
    dx = torch.empty((N, H2 // 2, W2 // 2, C), dtype=torch.bfloat16, device=dy.device)
    _call("cdf_nn_upsample2_bwd", _p(dy), _p(dx), N, H2 // 2, W2 // 2, C, Cy, coff, _stream())
    return dx


def copy_channels(x, y, src_off, dst_off, count, accumulate=False):
    P = x.numel() // x.shape[-1]
    _call("cdf_nn_copy_channels", _p(x), _p(y), P, x.shape[-1], y.shape[-1], src_off, dst_off, count,
          int(accumulate), _stream())


def head_fwd(x, w, b):
    import torch
    N, H, W, C = x.shape
    O = w.shape[0]
    out = torch.empty((N, H, W, O), dtype=torch.float32, device=x.device)
    _call("cdf_nn_head_fwd", _p(x), _p(w), _p(b), _p(out), N * H * W, C, O, _stream())
    return out


def head_bwd(x, w, dout, dw, db):
    import torch
    N, H, W, C = x.shape
    O = w.shape[0]
    dx = torch.empty((N, H, W, C), dtype=torch.bfloat16, device=x.device)
    _call("cdf_nn_head_bwd", _p(x), _p(w), _p(dout), _p(dx), _p(dw), _p(db), N * H * W, C, O, _stream())
    return dx


def mse(pred, target):
    import torch
    grad = torch.empty_like(pred)
    loss = torch.zeros(1, dtype=torch.float32, device=pred.device)
    _call("cdf_nn_mse", _p(pred), _p(target), _p(grad), _p(loss), pred.numel(), _stream())
    return loss, grad


def adam(w, g, m, v, w_bf16, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    _call("cdf_nn_adam", _p(w), _p(g), _p(m), _p(v), _p(w_bf16), w.numel(), lr, b1, b2, eps, step, _stream())


# ---- the network ----------------------------------------------------------------------------
IN_PLANES = 7
IN_PAD = 16
OUT_PLANES = 4


class UNet:
    """4-level U-Net; parameter names follow the FP64 oracle (e{L}a/b, d{L}a/b, head)."""

    def __init__(self, base: int = 32, levels: int = 4, cin: int = IN_PAD, cout: int = OUT_PLANES, seed: int = 0):
        import torch
        self.levels, self.cin, self.cout = levels, cin, cout
        self.ch = [base * 2 ** L for L in range(levels)]
        g = torch.Generator().manual_seed(seed)
        shapes = {}
        prev = cin
        for L, c in enumerate(self.ch):
            shapes[f"e{L}a"] = (c, prev)
            shapes[f"e{L}b"] = (c, c)
            prev = c
        for L in range(levels - 2, -1, -1):
            shapes[f"d{L}a"] = (self.ch[L], self.ch[L + 1] + self.ch[L])
            shapes[f"d{L}b"] = (self.ch[L], self.ch[L])
        self.conv_names = list(shapes)
        self.shapes = shapes
        self.master, self.bf16, self.m, self.v = {}, {}, {}, {}
        for name, (co, ci) in shapes.items():
            fan_in = 9 * ci
            w = torch.randn((co, 3, 3, ci), generator=g) * math.sqrt(2.0 / fan_in)
            self.master[name + ".w"] = w.cuda()
            self.master[name + ".b"] = torch.zeros(co).cuda()
        self.master["head.w"] = (torch.randn((cout, self.ch[0]), generator=g) * math.sqrt(1.0 / self.ch[0])).cuda()
        self.master["head.b"] = torch.zeros(cout).cuda()
        for k, t in self.master.items():
            self.m[k] = torch.zeros_like(t)
            self.v[k] = torch.zeros_like(t)
            if k.endswith(".w") and not k.startswith("head"):
                self.bf16[k] = t.to(torch.bfloat16)
        self.step_count = 0

    # forward: returns FP32 output [N, H, W, cout] and the activations the backward needs
    def forward(self, x):
        acts = {}
        h = x
        skips = []
        for L in range(self.levels):
            if L > 0:
                h = avgpool2_fwd(h)
            acts[f"e{L}.in"] = h
            h1 = conv3x3_fwd(h, self.bf16[f"e{L}a.w"], self.master[f"e{L}a.b"], True)
            h2 = conv3x3_fwd(h1, self.bf16[f"e{L}b.w"], self.master[f"e{L}b.b"], True)
            acts[f"e{L}a"], acts[f"e{L}b"] = h1, h2
            skips.append(h2)
            h = h2
        import torch
        for L in range(self.levels - 2, -1, -1):
            N, Hh, Ww, C = h.shape
            cat = torch.empty((N, 2 * Hh, 2 * Ww, C + self.ch[L]), dtype=torch.bfloat16, device=h.device)
            upsample2_into(h, cat, 0)
            copy_channels(skips[L], cat, 0, C, self.ch[L])
            acts[f"d{L}.cat"] = cat
            h1 = conv3x3_fwd(cat, self.bf16[f"d{L}a.w"], self.master[f"d{L}a.b"], True)
            h2 = conv3x3_fwd(h1, self.bf16[f"d{L}b.w"], self.master[f"d{L}b.b"], True)
            acts[f"d{L}a"], acts[f"d{L}b"] = h1, h2
            h = h2
        acts["head.in"] = h
        return head_fwd(h, self.master["head.w"], self.master["head.b"]), acts

    def backward(self, acts, dout):
        import torch
        grads = {k: torch.zeros_like(t) for k, t in self.master.items()}
        dh = head_bwd(acts["head.in"], self.master["head.w"], dout, grads["head.w"], grads["head.b"])
        dskip = [None] * self.levels
        for L in range(0, self.levels - 1):
            dh, dskip[L] = self._block_bwd(f"d{L}", acts[f"d{L}.cat"], acts, dh, grads, split=self.ch[L])
        for L in range(self.levels - 1, -1, -1):
            if dskip[L] is not None:
                copy_channels(dskip[L], dh, 0, 0, self.ch[L], accumulate=True)
            dx, _ = self._block_bwd(f"e{L}", acts[f"e{L}.in"], acts, dh, grads, split=None)
            if L > 0:
                N, H, W, C = acts[f"e{L - 1}b"].shape
                dh = avgpool2_bwd(dx, H, W)
        return grads

    def _block_bwd(self, name, x_in, acts, dh, grads, split):
        # second conv
        relu_bwd(dh, acts[f"{name}b"])
        conv3x3_bwd_weight(acts[f"{name}a"], dh, grads[f"{name}b.w"], grads[f"{name}b.b"])
        d1 = conv3x3_bwd_data(dh, self.bf16[f"{name}b.w"], acts[f"{name}a"].shape[3])
        relu_bwd(d1, acts[f"{name}a"])
        conv3x3_bwd_weight(x_in, d1, grads[f"{name}a.w"], grads[f"{name}a.b"])
        dx = conv3x3_bwd_data(d1, self.bf16[f"{name}a.w"], x_in.shape[3])
        if split is None:
            return dx, None
        cup = x_in.shape[3] - split
        import torch
        dskip = torch.empty((*dx.shape[:3], split), dtype=torch.bfloat16, device=dx.device)
        copy_channels(dx, dskip, cup, 0, split)
        return upsample2_bwd_from(dx, cup, 0), dskip

    def adam_step(self, grads, lr):
        self.step_count += 1
        for k, w in self.master.items():
            adam(w, grads[k], self.m[k], self.v[k], self.bf16.get(k), lr, self.step_count)

    def state(self):
        return {k: t.detach().cpu().numpy() for k, t in self.master.items()}

    def load_state(self, st):
        import torch
        for k, v in st.items():
            self.master[k].copy_(torch.as_tensor(v))
            if k in self.bf16:
                self.bf16[k].copy_(self.master[k].to(torch.bfloat16))


# ---- data: steady cavity states from the solver ---------------------------------------------
U_SCALE = 0.1 * math.sqrt(1.0 / 3.0)  # the buoyancy velocity of the lattice mapping (Ma = 0.1)


def draw_parameters(count: int, seed: int, log10_Ra=(4.0, 6.0), Nc=(-2.0, 2.0), Le=(1.0, 10.0), SrDf=(0.0, 0.5)):
    """Ra ~ logU[1e4, 1e6], Nc ~ U[-2, 2], Le ~ U[1, 10], Sr, Df ~ U[0, 0.5] by default
    (uniforms from counters 8k..8k+4 of `seed`)."""
    out = []
    for k in range(count):
        u = I.uniform(seed, np.arange(8 * k, 8 * k + 5))
        lin = lambda r, t: r[0] + (r[1] - r[0]) * t  # noqa: E731
        out.append(dict(Ra=10 ** lin(log10_Ra, u[0]), Nc=lin(Nc, u[1]), Le=lin(Le, u[2]), Sr=lin(SrDf, u[3]),
                        Df=lin(SrDf, u[4])))
    return out


def cavity(n: int, prm) -> I.Problem:
    return I.ddc_cavity(n, Ra=prm["Ra"], Pr=0.7, Le=prm["Le"], Nc=prm["Nc"], Df=prm["Df"], Sr=prm["Sr"])


def input_planes(n: int, prms) -> np.ndarray:
    """[N, n, n, IN_PAD] float32 inputs: log10 Ra - 5, Nc / 2, (Le - 5.5) / 4.5, 4 Sr - 1, 4 Df - 1, x, y."""
    N = len(prms)
    x = np.zeros((N, n, n, IN_PAD), np.float32)
    c = (np.arange(n) + 0.5) / n
    for k, prm in enumerate(prms):
        x[k, :, :, 0] = math.log10(prm["Ra"]) - 5
        x[k, :, :, 1] = prm["Nc"] / 2
        x[k, :, :, 2] = (prm["Le"] - 5.5) / 4.5
        x[k, :, :, 3] = 4 * prm["Sr"] - 1
        x[k, :, :, 4] = 4 * prm["Df"] - 1
        x[k, :, :, 5] = c[None, :]
        x[k, :, :, 6] = c[:, None]
    return x


def targets_from_moments(M) -> np.ndarray:
    """(u_x / U, u_y / U, T - 1/2, C - 1/2) from a moment stack [m+3][ny][nx]."""
    return np.stack([M[2] / U_SCALE, M[3] / U_SCALE, M[0] - 0.5, M[1] - 0.5], axis=-1).astype(np.float32)


def binomial_filter(a: np.ndarray) -> np.ndarray:
    """One pass of the separable [1, 2, 1] / 4 filter over the last two axes (edge
    values repeated): removes the grid-scale (Nyquist) content of a field."""
    pad = [(0, 0)] * (a.ndim - 2)
    p = np.pad(a, pad + [(1, 1), (0, 0)], mode="edge")
    a = 0.25 * (p[..., :-2, :] + 2.0 * p[..., 1:-1, :] + p[..., 2:, :])
    p = np.pad(a, pad + [(0, 0), (1, 1)], mode="edge")
    return 0.25 * (p[..., :-2] + 2.0 * p[..., 1:-1] + p[..., 2:])


def moments_from_prediction(y, pb=None, velocity: str = "zero") -> np.ndarray:
    """Inverse of targets_from_moments for one sample [n, n, 4] -> [5][n][n]; with the
    problem given, p is the hydrostatic pressure of the predicted buoyancy (dp/dy = F_y).

    velocity: "zero" (the default) starts the fluid from rest under the predicted
    scalars, "filtered" passes the predicted velocity through one binomial
    filter, "raw" keeps it.  Grid-scale errors of a predicted velocity excite
    lattice modes that the collision damps very slowly (in a 16^2 cavity 5 %
    white noise on u was still 3e-3 away from the steady state after 3e5 steps;
    filtered, it converged in 5e3); on the 64^2 held-out cavities even the
    filtered prediction reached relative L2 1e-3 fastest but mostly stalled above
    1e-4, while the start from the predicted scalars with the fluid at rest
    reached 1e-4 in every case, so that is the default."""
    n = y.shape[0]
    M = np.zeros((5, n, n))
    M[0], M[1] = y[..., 2] + 0.5, y[..., 3] + 0.5
    M[2], M[3] = y[..., 0] * U_SCALE, y[..., 1] * U_SCALE
    if velocity == "filtered":
        M[2:4] = binomial_filter(M[2:4])
    elif velocity == "zero":
        M[2:4] = 0.0
    elif velocity != "raw":
        raise ValueError(velocity)
    if pb is not None:
        Fy = pb.g[1] * (pb.F0 + sum(pb.beta[a] * (M[a] - pb.phi_ref[a]) for a in range(2)))
        p = np.cumsum(Fy, axis=0) - 0.5 * Fy
        M[4] = p - p.mean()
    return M


def generate_steady_states(prms, n: int, steps: int = 2_000_000, check_every: int = 10_000, steady_tol: float = 1e-5):
    """Run every cavity from rest for `steps` steps with the batched solver (the
    persistent kernel: many small lattices in one launch); returns the final
    moment stacks, the residual over the last `check_every` steps and a mask of
    the cases that are steady to within the FP32 round-off floor (R < steady_tol)."""
    pbs = [cavity(n, prm) for prm in prms]
    b = lib.BatchSolver(pbs, tile=(64, 4), mode=0)
    b.step(steps - check_every)
    R = b.residuals_after(check_every)
    Ms = [b.moments(k) for k in range(len(pbs))]
    b.close()
    return Ms, R, R < steady_tol


def rel_l2_distance(M, Mref) -> float:
    """max over q in (T, C, u_x, u_y) of ||q - q_ref||_2 / ||q_ref||_2."""
    return max(float(np.linalg.norm(M[q] - Mref[q]) / max(np.linalg.norm(Mref[q]), 1e-300)) for q in range(4))


def _steps_to_reference(b, inits, refs, eps_list, check_every, max_steps):
    """Re-initialise every instance and step until its relative L2 distance to its
    reference state drops below each eps (checked every `check_every` steps)."""
    for k, (phi, u, p) in enumerate(inits):
        lib.cdf_batch_init_moments(b.h, k, phi, u, p)
    n = len(inits)
    first = {e: np.full(n, -1, dtype=np.int64) for e in eps_list}
    last = np.full(n, np.inf)
    taken = 0
    tight = min(eps_list)
    while taken < max_steps:
        b.step(check_every)
        taken += check_every
        for k in np.flatnonzero(first[tight] < 0):
            last[k] = rel_l2_distance(b.moments(k), refs[k])
            for e in eps_list:
                if last[k] < e and first[e][k] < 0:
                    first[e][k] = taken
        if (first[tight] >= 0).all():
            break
    return first, taken, last


def warm_start_comparison(net: UNet, prms, n: int, eps_list=(1e-3, 1e-4), ref_steps: int = 6_000_000,
                          check_every: int = 10_000, steady_tol: float = 2e-6, max_steps: int = 0,
                          warm_kinds=None):
    """For held-out parameters: the steady state is the state after `ref_steps`
    steps from rest (kept only where the residual then is below steady_tol); the
    time to steady state of a start is the first multiple of `check_every` steps
    at which its relative L2 distance to that state (worst of T, C, u_x, u_y) is
    below eps, for starts from rest and from the network's prediction, each run
    for at most max_steps (default ref_steps / 2, so the start from rest is not
    timed against its own end state).  warm_kinds maps the name of each network
    start to its velocity treatment (moments_from_prediction); default
    {"warm": "zero", "warm_velocity": "filtered"}."""
    max_steps = max_steps or ref_steps // 2
    warm_kinds = warm_kinds or {"warm": "zero", "warm_velocity": "filtered"}
    import time
    import torch
    x = torch.as_tensor(input_planes(n, prms)).cuda().to(torch.bfloat16)
    pred = predict(net, x).float().cpu().numpy()
    pbs = [cavity(n, prm) for prm in prms]
    b = lib.BatchSolver(pbs, tile=(64, 4), mode=0)
    b.step(ref_steps - check_every)
    R = b.residuals_after(check_every)
    refs = [b.moments(k) for k in range(len(pbs))]
    steady = R < steady_tol
    f64 = lambda a: np.ascontiguousarray(a, np.float64)  # noqa: E731
    starts = {"cold": [(f64(pb.phi0), f64(pb.u0), f64(pb.p0)) for pb in pbs]}
    for name, vel in warm_kinds.items():
        starts[name] = []
        for k, pb in enumerate(pbs):
            M = moments_from_prediction(pred[k], pb, vel)
            starts[name].append((f64(M[:2]), f64(M[2:4]), f64(M[4])))
    out = {"steady": steady, "R_ref": R, "prediction": pred,
           "prediction_error": np.array([rel_l2_distance(moments_from_prediction(pred[k], None, "raw"), refs[k])
                                         for k in range(len(pbs))])}
    for name, inits in starts.items():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        first, taken, last = _steps_to_reference(b, inits, refs, eps_list, check_every, max_steps)
        torch.cuda.synchronize()
        out[name] = dict(first=first, seconds=time.perf_counter() - t0, steps=taken, last_distance=last)
    b.close()
    return out


def upsample_prediction(pred: np.ndarray, n: int) -> np.ndarray:
    """Bilinear resampling of predictions [N, m, m, 4] on an m x m cell-centred grid to
    n x n (the fields are dimensionless, so a network trained on one lattice size gives
    the others their steady state up to its discretisation error)."""
    import torch
    import torch.nn.functional as Fn
    t = torch.as_tensor(np.ascontiguousarray(pred.transpose(0, 3, 1, 2)), dtype=torch.float32)
    up = Fn.interpolate(t, size=(n, n), mode="bilinear", align_corners=False)
    return up.numpy().transpose(0, 2, 3, 1)


def time_to_steady(net: UNet, prms, n: int, n_net: int = 64, tol: float = 1e-5, check_every: int = 10_000,
                   max_steps: int = 4_000_000, velocity: str = "zero"):
    """Lattice steps and GPU seconds to the stop test of Sec. 3.1.1 (the residual R of
    cdf_lb_run_to_steady over `check_every` steps below `tol`) for n x n cavities of
    the parameters `prms`, from rest and from the network's prediction (made on the
    n_net x n_net lattice the network was trained on and resampled to n x n; the
    fluid at rest by default, see moments_from_prediction).  Each case and start runs
    on its own single-lattice solver (the configuration the autotuner picks for
    n x n), so the seconds are that case's own.  Returns per start the steps at which
    each case met the test (-1: not within max_steps), the seconds of each run and
    the last residuals."""
    import time
    import torch
    x = torch.as_tensor(input_planes(n_net, prms)).cuda().to(torch.bfloat16)
    pred = predict(net, x).float().cpu().numpy()
    if n != n_net:
        pred = upsample_prediction(pred, n)
    pbs = [cavity(n, prm) for prm in prms]
    f64 = lambda a: np.ascontiguousarray(a, np.float64)  # noqa: E731
    starts = {"cold": [(f64(pb.phi0), f64(pb.u0), f64(pb.p0)) for pb in pbs], "warm": []}
    for k, pb in enumerate(pbs):
        M = moments_from_prediction(pred[k], pb, velocity)
        starts["warm"].append((f64(M[:2]), f64(M[2:4]), f64(M[4])))
    out = {}
    for name, inits in starts.items():
        first = np.full(len(pbs), -1, dtype=np.int64)
        secs = np.zeros(len(pbs))
        R = np.full(len(pbs), np.inf)
        for k, (phi, u, p) in enumerate(inits):
            s = lib.Solver(pbs[k], init=False)
            s.init_moments(phi, u, p)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ok, steps, R[k] = s.run_to_steady(tol, check_every, max_steps)
            torch.cuda.synchronize()
            secs[k] = time.perf_counter() - t0
            first[k] = steps if ok else -1
            s.close()
        out[name] = {"first": first, "seconds": secs, "steps": int(max(first.max(), 0)), "R": R}
    return out


def train(net: UNet, x, y, epochs: int, batch: int, lr: float, seed: int = 0, log=None):
    """x: torch bf16 [S, n, n, 16], y: torch fp32 [S, n, n, 4]; plain Adam with a cosine decay."""
    import torch
    S = x.shape[0]
    r = np.random.default_rng(seed)
    steps_per_epoch = max(1, S // batch)
    total = epochs * steps_per_epoch
    it = 0
    hist = []
    for ep in range(epochs):
        perm = torch.as_tensor(r.permutation(S), device=x.device)
        ep_loss = 0.0
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            xb, yb = x.index_select(0, idx).contiguous(), y.index_select(0, idx).contiguous()
            out, acts = net.forward(xb)
            loss, dout = mse(out, yb)
            grads = net.backward(acts, dout)
            cur = lr * 0.5 * (1 + math.cos(math.pi * it / total))
            net.adam_step(grads, cur)
            ep_loss += float(loss.item())
            it += 1
        hist.append(ep_loss / steps_per_epoch)
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def predict(net: UNet, x, batch: int = 64):
    import torch
    outs = []
    for s in range(0, x.shape[0], batch):
        out, _ = net.forward(x[s:s + batch].contiguous())
        outs.append(out)
    return torch.cat(outs)


def default_model_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "surrogate_cavity64.npz")


def run_experiment(n=64, train_count=2000, eval_count=200, epochs=100, batch=32, lr=2e-3, steps=2_000_000,
                   check_every=10_000, steady_tol=1e-5, seed=0, ref_steps=6_000_000, log=print):
    """Generate steady states, train the U-Net, and compare warm with cold starts on
    held-out parameters.  Returns a JSON-ready summary."""
    import time
    import torch
    t0 = time.perf_counter()
    prms = draw_parameters(train_count, seed)
    Ms, R, steady = generate_steady_states(prms, n, steps, check_every, steady_tol)
    keep = np.flatnonzero(steady)
    t_data = time.perf_counter() - t0
    log(f"data: {len(keep)}/{train_count} steady (R < {steady_tol:g} after {steps} steps) in {t_data:.1f} s")
    x = torch.as_tensor(input_planes(n, [prms[k] for k in keep])).cuda().to(torch.bfloat16)
    y = torch.as_tensor(np.stack([targets_from_moments(Ms[k]) for k in keep])).cuda()
    net = UNet(seed=seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = train(net, x, y, epochs, batch, lr, seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    log(f"train: {epochs} epochs on {len(keep)} states in {t_train:.1f} s, loss {hist[0]:.3e} -> {hist[-1]:.3e}")
    eprm = draw_parameters(eval_count, seed + 1)
    res = warm_start_comparison(net, eprm, n, (1e-3, 1e-4), ref_steps, check_every)
    st = res["steady"]
    kinds = [k for k in res if k not in ("steady", "R_ref", "prediction", "prediction_error")]
    summary = {"n": n, "train_requested": train_count, "train_steady": int(len(keep)), "eval": eval_count,
               "eval_steady": int(st.sum()), "steps_training_data": steps, "steps_reference": ref_steps,
               "max_steps_timed": ref_steps // 2, "check_every": check_every,
               "steady_tol_training": steady_tol, "data_seconds": t_data, "train_seconds": t_train, "epochs": epochs,
               "loss_first": hist[0], "loss_last": hist[-1],
               "seconds": {k: res[k]["seconds"] for k in kinds}}
    for eps in (1e-3, 1e-4):
        c = res["cold"]["first"][eps]
        entry = {"cold_reached": int((st & (c >= 0)).sum()),
                 "median_final_distance": {k: float(np.median(res[k]["last_distance"][st])) for k in kinds}}
        for k in kinds:
            if k == "cold":
                continue
            w = res[k]["first"][eps]
            both = st & (c >= 0) & (w >= 0)
            ratio = w[both] / np.maximum(c[both], 1)
            entry[k] = {
                "reached": int((st & (w >= 0)).sum()), "cases_both": int(both.sum()),
                "median_steps_cold": float(np.median(c[both])) if both.any() else None,
                "median_steps": float(np.median(w[both])) if both.any() else None,
                "median_ratio_over_cold": float(np.median(ratio)) if both.any() else None,
                "mean_ratio_over_cold": float(np.mean(ratio)) if both.any() else None,
                "fraction_faster": float((ratio < 1).mean()) if both.any() else None,
                "total_steps_cold": int(c[both].sum()), "total_steps": int(w[both].sum())}
        summary[f"eps{eps:g}"] = entry
    pe = res["prediction_error"][st]
    summary["prediction_rel_l2"] = {"median": float(np.median(pe)), "p10": float(np.percentile(pe, 10)),
                                    "p90": float(np.percentile(pe, 90))} if st.any() else None
    summary["eval_cases"] = [dict(eprm[k], steady=bool(st[k]), R_ref=float(res["R_ref"][k]),
                                  prediction_rel_l2=float(res["prediction_error"][k]),
                                  **{f"{kind}_{e:g}": int(res[kind]["first"][e][k]) for kind in kinds
                                     for e in (1e-3, 1e-4)})
                             for k in range(eval_count)]
    summary["train_cases"] = [dict(prms[k], steady=bool(steady[k]), R=float(R[k])) for k in range(train_count)]
    log(str({k: v for k, v in summary.items() if not k.endswith("_cases")}))
    return summary, net


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="surrogate warm-start experiment on the double-diffusive cavity")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--steps", type=int, default=2_000_000, help="steps from rest for the training states")
    ap.add_argument("--ref-steps", type=int, default=6_000_000, help="steps from rest for the held-out references")
    ap.add_argument("--check-every", type=int, default=10_000)
    ap.add_argument("--out", default="")
    ap.add_argument("--time-to-steady", type=int, default=0, metavar="N",
                    help="instead of the experiment: steps to the stop test on N x N cavities from rest and from "
                         "the committed network's prediction (time_to_steady)")
    ap.add_argument("--cases", type=int, default=8)
    ap.add_argument("--tol", type=float, nargs="+", default=[1e-5, 2e-6])
    ap.add_argument("--max-steps", type=int, default=5_000_000)
    a = ap.parse_args()
    from . import build
    build.build()
    if a.time_to_steady:
        net = UNet(seed=0)
        net.load_state(dict(np.load(default_model_path())))
        prms = draw_parameters(a.cases, 1)
        out = {"params": prms, "n": a.time_to_steady, "max_steps": a.max_steps, "runs": {}}
        for tol in a.tol:
            res = time_to_steady(net, prms, a.time_to_steady, 64, tol=tol, check_every=a.check_every,
                                 max_steps=a.max_steps)
            out["runs"][f"{tol:g}"] = {k: {"first": v["first"].tolist(), "seconds": v["seconds"].tolist(),
                                          "steps": v["steps"],
                                          "R": v["R"].tolist()} for k, v in res.items()}
            print(tol, {k: v["first"].tolist() for k, v in res.items()}, flush=True)
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(out, fh, indent=1)
    else:
        summ, net = run_experiment(a.n, a.train, a.eval, a.epochs, steps=a.steps, check_every=a.check_every,
                                   ref_steps=a.ref_steps)
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(summ, fh, indent=1)
            np.savez(a.out.replace(".json", "_model.npz"), **net.state())
