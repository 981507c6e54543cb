"""FP64 CPU oracle of the surrogate network's layers (TEST INFRASTRUCTURE).

Plain numpy, NHWC activations, weights [Cout][3][3][Cin], written from the
definitions: 3x3 cross-correlation with zero padding, its gradients with
respect to input, weights and bias, 2x2 average pooling, nearest 2x
upsampling, the 1x1 head, mean squared error and one Adam step (Kingma & Ba,
"Adam: a method for stochastic optimization", 2015, Algorithm 1).  Pinned in
tests/test_nn_oracle_pins.py against scipy's correlate, central finite
differences and adjointness identities.
"""
from __future__ import annotations

import numpy as np


def conv3x3_fwd(x, w, b=None, relu=False):
    """y[n,y,x,co] = sum_{ky,kx,ci} x[n, y+ky-1, x+kx-1, ci] w[co,ky,kx,ci] (+ b), zero padded."""
    N, H, W, Ci = x.shape
    Co = w.shape[0]
    xp = np.zeros((N, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((N, H, W, Co))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("nhwc,oc->nhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    if b is not None:
        y += b
    return np.maximum(y, 0.0) if relu else y


def conv3x3_bwd_data(dy, w):
    """Gradient of sum(dy * conv3x3_fwd(x, w)) with respect to x."""
    N, H, W, Co = dy.shape
    Ci = w.shape[3]
    dxp = np.zeros((N, H + 2, W + 2, Ci))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("nhwo,oc->nhwc", dy, w[:, ky, kx, :])
    return dxp[:, 1:-1, 1:-1, :]


def conv3x3_bwd_weight(x, dy):
    """Gradients of sum(dy * conv3x3_fwd(x, w) + dy * b) with respect to w and b."""
    N, H, W, Ci = x.shape
    Co = dy.shape[3]
    xp = np.zeros((N, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    dw = np.zeros((Co, 3, 3, Ci))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("nhwo,nhwc->oc", dy, xp[:, ky:ky + H, kx:kx + W, :])
    return dw, dy.sum(axis=(0, 1, 2))


def avgpool2_fwd(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def upsample2_fwd(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_bwd(dy):
    N, H2, W2, C = dy.shape
    return dy.reshape(N, H2 // 2, 2, W2 // 2, 2, C).sum(axis=(2, 4))


def head_fwd(x, w, b):
    return np.einsum("nhwc,oc->nhwo", x, w) + b


def head_bwd(x, w, dout):
    return np.einsum("nhwo,oc->nhwc", dout, w), np.einsum("nhwo,nhwc->oc", dout, x), dout.sum(axis=(0, 1, 2))


def mse(pred, target):
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# The U-Net of the surrogate, forward and backward, layer by layer.
# ---------------------------------------------------------------------------
def unet_forward(params, x, levels):
    """params: dict of FP64 arrays named like the GPU network's; returns (out, cache)."""
    acts = {}
    h = x
    skips = []
    for L in range(levels):
        if L > 0:
            h = avgpool2_fwd(h)
        h1 = conv3x3_fwd(h, params[f"e{L}a.w"], params[f"e{L}a.b"], relu=True)
        h2 = conv3x3_fwd(h1, params[f"e{L}b.w"], params[f"e{L}b.b"], relu=True)
        acts[f"e{L}.in"], acts[f"e{L}a"], acts[f"e{L}b"] = h, h1, h2
        skips.append(h2)
        h = h2
    for L in range(levels - 2, -1, -1):
        up = upsample2_fwd(h)
        cat = np.concatenate([up, skips[L]], axis=3)
        h1 = conv3x3_fwd(cat, params[f"d{L}a.w"], params[f"d{L}a.b"], relu=True)
        h2 = conv3x3_fwd(h1, params[f"d{L}b.w"], params[f"d{L}b.b"], relu=True)
        acts[f"d{L}.cat"], acts[f"d{L}a"], acts[f"d{L}b"] = cat, h1, h2
        h = h2
    out = head_fwd(h, params["head.w"], params["head.b"])
    acts["head.in"] = h
    return out, acts


def unet_backward(params, acts, dout, levels):
    g = {}
    dh, g["head.w"], g["head.b"] = head_bwd(acts["head.in"], params["head.w"], dout)
    dskip = [None] * levels
    for L in range(0, levels - 1):
        d = dh * (acts[f"d{L}b"] > 0)
        g[f"d{L}b.w"], g[f"d{L}b.b"] = conv3x3_bwd_weight(acts[f"d{L}a"], d)
        d1 = conv3x3_bwd_data(d, params[f"d{L}b.w"]) * (acts[f"d{L}a"] > 0)
        g[f"d{L}a.w"], g[f"d{L}a.b"] = conv3x3_bwd_weight(acts[f"d{L}.cat"], d1)
        dcat = conv3x3_bwd_data(d1, params[f"d{L}a.w"])
        cup = dcat.shape[3] - acts[f"e{L}b"].shape[3]
        dskip[L] = dcat[..., cup:]
        dh = upsample2_bwd(dcat[..., :cup])
    # dh is now the gradient at the output of the deepest encoder level
    for L in range(levels - 1, -1, -1):
        if dskip[L] is not None:
            dh = dh + dskip[L]
        d = dh * (acts[f"e{L}b"] > 0)
        g[f"e{L}b.w"], g[f"e{L}b.b"] = conv3x3_bwd_weight(acts[f"e{L}a"], d)
        d1 = conv3x3_bwd_data(d, params[f"e{L}b.w"]) * (acts[f"e{L}a"] > 0)
        g[f"e{L}a.w"], g[f"e{L}a.b"] = conv3x3_bwd_weight(acts[f"e{L}.in"], d1)
        dx = conv3x3_bwd_data(d1, params[f"e{L}a.w"])
        if L > 0:
            dh = avgpool2_bwd(dx)
    return g
