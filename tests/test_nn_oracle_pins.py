"""Pins of the FP64 oracle of the surrogate network's layers (CPU)."""
import numpy as np
import pytest

from oracle import nn_oracle as R


def rng(s):
    return np.random.default_rng(s)


def test_conv_matches_scipy_correlate():
    from scipy.signal import correlate2d
    r = rng(0)
    x = r.normal(size=(2, 7, 9, 3))
    w = r.normal(size=(4, 3, 3, 3))
    b = r.normal(size=4)
    y = R.conv3x3_fwd(x, w, b)
    for n in range(2):
        for co in range(4):
            ref = sum(correlate2d(x[n, :, :, ci], w[co, :, :, ci], mode="same") for ci in range(3)) + b[co]
            np.testing.assert_allclose(y[n, :, :, co], ref, rtol=1e-12, atol=1e-12)
    assert np.all(R.conv3x3_fwd(x, w, b, relu=True) >= 0)


def test_conv_backward_passes_are_adjoints():
    """<dy, conv(x, w)> = <bwd_data(dy, w), x> = <bwd_weight(x, dy).dw, w> (bilinear form)."""
    r = rng(1)
    x, w, dy = r.normal(size=(2, 6, 5, 3)), r.normal(size=(4, 3, 3, 3)), r.normal(size=(2, 6, 5, 4))
    lhs = np.sum(dy * R.conv3x3_fwd(x, w))
    assert np.sum(R.conv3x3_bwd_data(dy, w) * x) == pytest.approx(lhs, rel=1e-12)
    dw, db = R.conv3x3_bwd_weight(x, dy)
    assert np.sum(dw * w) == pytest.approx(lhs, rel=1e-12)
    np.testing.assert_allclose(db, dy.sum(axis=(0, 1, 2)))


def test_pool_upsample_head_adjoints():
    r = rng(2)
    x, y = r.normal(size=(2, 6, 4, 3)), r.normal(size=(2, 3, 2, 3))
    assert np.sum(R.avgpool2_fwd(x) * y) == pytest.approx(np.sum(x * R.avgpool2_bwd(y)), rel=1e-12)
    u, v = r.normal(size=(2, 3, 2, 3)), r.normal(size=(2, 6, 4, 3))
    assert np.sum(R.upsample2_fwd(u) * v) == pytest.approx(np.sum(u * R.upsample2_bwd(v)), rel=1e-12)
    w, b, d = r.normal(size=(4, 3)), r.normal(size=4), r.normal(size=(2, 6, 4, 4))
    dx, dw, db = R.head_bwd(x, w, d)
    assert np.sum(d * (R.head_fwd(x, w, b) - b)) == pytest.approx(np.sum(dx * x), rel=1e-12)
    assert np.sum(dw * w) == pytest.approx(np.sum(dx * x), rel=1e-12)


def tiny_params(r, cin=4, c=(4, 8), cout=3):
    p = {}
    chans = [cin] + list(c)
    for L in range(len(c)):
        p[f"e{L}a.w"] = r.normal(size=(c[L], 3, 3, chans[L])) * 0.4
        p[f"e{L}a.b"] = r.normal(size=c[L]) * 0.1
        p[f"e{L}b.w"] = r.normal(size=(c[L], 3, 3, c[L])) * 0.4
        p[f"e{L}b.b"] = r.normal(size=c[L]) * 0.1
    for L in range(len(c) - 1):
        cat = c[L + 1] + c[L]
        p[f"d{L}a.w"] = r.normal(size=(c[L], 3, 3, cat)) * 0.3
        p[f"d{L}a.b"] = r.normal(size=c[L]) * 0.1
        p[f"d{L}b.w"] = r.normal(size=(c[L], 3, 3, c[L])) * 0.4
        p[f"d{L}b.b"] = r.normal(size=c[L]) * 0.1
    p["head.w"] = r.normal(size=(cout, c[0])) * 0.4
    p["head.b"] = r.normal(size=cout) * 0.1
    return p


def test_unet_gradient_by_finite_differences():
    r = rng(3)
    levels = 2
    p = tiny_params(r)
    x = r.normal(size=(2, 8, 8, 4))
    t = r.normal(size=(2, 8, 8, 3))
    out, acts = R.unet_forward(p, x, levels)
    loss, dout = R.mse(out, t)
    g = R.unet_backward(p, acts, dout, levels)
    assert set(g) == set(p)
    eps = 1e-6
    for name in p:
        for _ in range(3):
            idx = tuple(r.integers(0, s) for s in p[name].shape)
            q = {k: v.copy() for k, v in p.items()}
            q[name][idx] += eps
            lp = R.mse(R.unet_forward(q, x, levels)[0], t)[0]
            q[name][idx] -= 2 * eps
            lm = R.mse(R.unet_forward(q, x, levels)[0], t)[0]
            fd = (lp - lm) / (2 * eps)
            assert g[name][idx] == pytest.approx(fd, rel=1e-4, abs=1e-9), name


def test_adam_first_step_moves_by_lr_times_sign():
    """With bias correction the first Adam step is lr * g / (|g| + eps') ~ lr * sign(g)."""
    g = np.array([3.0, -0.2, 1e-3])
    w, m, v = R.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(w, -0.01 * np.sign(g), rtol=1e-6)
