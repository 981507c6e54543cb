"""The surrogate's BF16 kernels against the FP64 oracle (oracle/nn_oracle.py).

Inputs are drawn in FP64, rounded to BF16, and the oracle runs on the rounded
values, so only the kernels' own arithmetic differs: BF16 outputs carry one
rounding (unit roundoff 2^-9, relative L2 ~1e-3, bound 8e-3); FP32 outputs
(weight gradients, head, loss) differ only by summation order (bound 1e-5).
The whole U-Net keeps BF16 activations between layers, so its outputs and
gradients are held to 3e-2 / 6e-2 relative L2 against the all-FP64 oracle.
"""
import math

import numpy as np
import pytest

from oracle import nn_oracle as R

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def S(cdf):
    import torch
    from paper_2101_03055_gb300 import surrogate
    surrogate.nn_lib()
    return surrogate, torch


@pytest.fixture(params=["tcgen05", "tcgen05_sync", "tcgen05_ws", "tcgen05_slab", "mma"])
def path(S, request):
    """Run a convolution test on each tensor-core path, and check afterwards that no
    bounded wait of the tcgen05 kernels ran out."""
    sur, torch = S
    sur.set_tensor_path({"tcgen05": 1, "tcgen05_sync": 2, "tcgen05_ws": 3, "tcgen05_slab": 4, "mma": 0}[request.param])
    yield request.param
    torch.cuda.synchronize()
    sur.set_tensor_path(True)
    assert sur.tensor_error_flag() == 0


def bf(torch, a):
    t = torch.as_tensor(np.asarray(a, np.float32)).cuda().to(torch.bfloat16)
    return t, t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,H,W,Cin,Cout", [(2, 9, 13, 16, 32), (1, 8, 8, 32, 64), (2, 5, 7, 96, 32),
                                            (1, 4, 4, 384, 128), (2, 24, 20, 64, 128),
                                            # rows of whole 128-pixel tiles: the forward without im2col
                                            # copy (paths 1 and 4), Cin 16 / 32 / 64, every output tile
                                            # width, tiles at the image's top and bottom rows
                                            (2, 3, 256, 16, 32), (1, 4, 128, 32, 32), (1, 2, 128, 32, 96),
                                            (1, 3, 256, 32, 128), (2, 3, 128, 64, 64), (1, 2, 128, 64, 128),
                                            (1, 1, 128, 16, 64)])
def test_conv_forward(S, path, N, H, W, Cin, Cout):
    sur, torch = S
    r = np.random.default_rng(N * 1000 + Cin)
    x, xr = bf(torch, r.normal(size=(N, H, W, Cin)))
    w, wr = bf(torch, r.normal(size=(Cout, 3, 3, Cin)) / math.sqrt(9 * Cin))
    b = torch.as_tensor(r.normal(size=Cout).astype(np.float32)).cuda()
    for relu in (False, True):
        y = sur.conv3x3_fwd(x, w, b, relu).float().cpu().numpy()
        assert rel(y, R.conv3x3_fwd(xr, wr, b.cpu().numpy().astype(np.float64), relu)) < 8e-3


@pytest.mark.parametrize("N,H,W,Cin,Cout", [(2, 9, 13, 16, 32), (1, 8, 8, 64, 64), (2, 5, 7, 96, 32),
                                            (1, 4, 4, 384, 128), (2, 24, 20, 128, 64), (1, 16, 12, 128, 256),
                                            (2, 64, 64, 32, 32), (1, 40, 40, 64, 512), (2, 96, 96, 32, 32)])
def test_conv_backward(S, path, N, H, W, Cin, Cout):
    sur, torch = S
    r = np.random.default_rng(N * 7 + Cin)
    x, xr = bf(torch, r.normal(size=(N, H, W, Cin)))
    w, wr = bf(torch, r.normal(size=(Cout, 3, 3, Cin)) / math.sqrt(9 * Cin))
    dy, dyr = bf(torch, r.normal(size=(N, H, W, Cout)))
    dx = sur.conv3x3_bwd_data(dy, w, Cin).float().cpu().numpy()
    assert rel(dx, R.conv3x3_bwd_data(dyr, wr)) < 8e-3
    dw = torch.zeros((Cout, 3, 3, Cin), dtype=torch.float32, device="cuda")
    db = torch.zeros(Cout, dtype=torch.float32, device="cuda")
    sur.conv3x3_bwd_weight(x, dy, dw, db)
    dwr, dbr = R.conv3x3_bwd_weight(xr, dyr)
    assert rel(dw.cpu().numpy(), dwr) < 1e-5
    assert rel(db.cpu().numpy(), dbr) < 1e-5


def test_weight_gradient_is_deterministic(S):
    """The tensor-core weight gradient adds its pixel splits in a fixed order: two
    calls on the same inputs give the same bits (the warp-level path adds atomically)."""
    sur, torch = S
    sur.set_tensor_path(True)
    r = np.random.default_rng(3)
    x, _ = bf(torch, r.normal(size=(4, 48, 40, 64)))
    dy, _ = bf(torch, r.normal(size=(4, 48, 40, 128)))
    outs = []
    for _ in range(2):
        dw = torch.zeros((128, 3, 3, 64), dtype=torch.float32, device="cuda")
        db = torch.zeros(128, dtype=torch.float32, device="cuda")
        sur.conv3x3_bwd_weight(x, dy, dw, db)
        outs.append((dw.cpu().numpy(), db.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert sur.tensor_error_flag() == 0


def test_small_layers(S):
    sur, torch = S
    r = np.random.default_rng(5)
    x, xr = bf(torch, r.normal(size=(2, 6, 10, 32)))
    y = sur.avgpool2_fwd(x).float().cpu().numpy()
    assert rel(y, R.avgpool2_fwd(xr)) < 8e-3
    d, dr = bf(torch, r.normal(size=(2, 3, 5, 32)))
    assert rel(sur.avgpool2_bwd(d, 6, 10).float().cpu().numpy(), R.avgpool2_bwd(dr)) < 8e-3
    cat = torch.zeros((2, 6, 10, 48), dtype=torch.bfloat16, device="cuda")
    sur.upsample2_into(d, cat, 0)
    s, sr = bf(torch, r.normal(size=(2, 6, 10, 16)))
    sur.copy_channels(s, cat, 0, 32, 16)
    c = cat.float().cpu().numpy()
    np.testing.assert_array_equal(c[..., :32], R.upsample2_fwd(dr))
    np.testing.assert_array_equal(c[..., 32:], sr)
    back = sur.upsample2_bwd_from(cat, 32, 0).float().cpu().numpy()
    assert rel(back, R.upsample2_bwd(c[..., :32])) < 8e-3
    h, hr = bf(torch, r.normal(size=(2, 6, 10, 32)))
    w = torch.as_tensor(r.normal(size=(4, 32)).astype(np.float32)).cuda()
    b = torch.as_tensor(r.normal(size=4).astype(np.float32)).cuda()
    out = sur.head_fwd(h, w, b)
    assert rel(out.cpu().numpy(), R.head_fwd(hr, w.cpu().numpy().astype(np.float64), b.cpu().numpy())) < 1e-5
    t = torch.as_tensor(r.normal(size=(2, 6, 10, 4)).astype(np.float32)).cuda()
    loss, grad = sur.mse(out, t)
    lr_, gr = R.mse(out.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64))
    assert loss.item() == pytest.approx(lr_, rel=1e-5)
    assert rel(grad.cpu().numpy(), gr) < 1e-6
    dw = torch.zeros_like(w)
    db = torch.zeros_like(b)
    dx = sur.head_bwd(h, w, grad, dw, db)
    dxr, dwr, dbr = R.head_bwd(hr, w.cpu().numpy().astype(np.float64), gr)
    assert rel(dx.float().cpu().numpy(), dxr) < 8e-3
    assert rel(dw.cpu().numpy(), dwr) < 1e-5 and rel(db.cpu().numpy(), dbr) < 1e-5
    wt = torch.as_tensor(r.normal(size=50).astype(np.float32)).cuda()
    g = torch.as_tensor(r.normal(size=50).astype(np.float32)).cuda()
    m, v = torch.zeros_like(wt), torch.zeros_like(wt)
    w0 = wt.cpu().numpy().astype(np.float64)
    sur.adam(wt, g, m, v, None, 1e-2, 1)
    wr, _, _ = R.adam_step(w0, g.cpu().numpy().astype(np.float64), np.zeros(50), np.zeros(50), 1, 1e-2)
    np.testing.assert_allclose(wt.cpu().numpy(), wr, rtol=1e-5, atol=1e-7)


def test_unet_forward_backward_against_oracle(S):
    sur, torch = S
    net = sur.UNet(base=32, levels=4, seed=3)
    # biases non-zero so every term is exercised
    r = np.random.default_rng(9)
    for k, t in net.master.items():
        if k.endswith(".b"):
            t.copy_(torch.as_tensor(r.normal(size=t.shape).astype(np.float32) * 0.05))
    params = {}
    for k, t in net.master.items():
        params[k] = (net.bf16[k].float() if k in net.bf16 else t).cpu().numpy().astype(np.float64)
    x, xr = bf(torch, np.concatenate([r.normal(size=(2, 16, 16, 7)), np.zeros((2, 16, 16, 9))], axis=3))
    out, acts = net.forward(x)
    oref, aref = R.unet_forward(params, xr, 4)
    assert rel(out.cpu().numpy(), oref) < 3e-2
    t = torch.as_tensor(r.normal(size=out.shape).astype(np.float32)).cuda()
    loss, dout = sur.mse(out, t)
    grads = net.backward(acts, dout)
    _, dref = R.mse(oref, t.cpu().numpy().astype(np.float64))
    gref = R.unet_backward(params, aref, dref, 4)
    worst = max(rel(grads[k].cpu().numpy(), gref[k]) for k in gref)
    assert worst < 6e-2, worst


def test_training_reduces_loss(S):
    """A few hundred Adam steps on a small smooth regression task lower the loss."""
    sur, torch = S
    r = np.random.default_rng(1)
    n = 16
    prm = [dict(Ra=10 ** (4 + 2 * a), Nc=b, Le=2.0, Sr=0.1, Df=0.1) for a, b in r.uniform(0, 1, size=(64, 2))]
    x = torch.as_tensor(sur.input_planes(n, prm)).cuda().to(torch.bfloat16)
    xx = x.float()
    y = torch.stack([xx[..., 0] * xx[..., 5], xx[..., 1] * xx[..., 6], torch.sin(3 * xx[..., 5]), xx[..., 6] ** 2],
                    dim=-1).contiguous()
    net = sur.UNet(base=32, levels=4, seed=0)
    hist = sur.train(net, x, y, epochs=40, batch=16, lr=2e-3)
    assert hist[-1] < 0.2 * hist[0]


@pytest.mark.parametrize("N,H,W,Cin,Cout", [(2, 3, 256, 16, 32), (1, 4, 128, 32, 64), (1, 3, 128, 64, 128)])
def test_conv_forward_without_im2col_same_bits(S, N, H, W, Cin, Cout):
    """The forward kernel without im2col copy (path 4) issues the same MMAs in the same
    K order as the staged kernels (tap by tap, 16 channels at a time), so its output
    equals the synchronous-staging kernel's (path 2) bit for bit."""
    sur, torch = S
    r = np.random.default_rng(7 * Cin + W)
    x, _ = bf(torch, r.normal(size=(N, H, W, Cin)))
    w, _ = bf(torch, r.normal(size=(Cout, 3, 3, Cin)) / math.sqrt(9 * Cin))
    b = torch.as_tensor(r.normal(size=Cout).astype(np.float32)).cuda()
    try:
        out = {}
        for p in (2, 4):
            sur.set_tensor_path(p)
            out[p] = sur.conv3x3_fwd(x, w, b, True).cpu()
        torch.cuda.synchronize()
        assert torch.equal(out[2], out[4])
    finally:
        sur.set_tensor_path(True)
    assert sur.tensor_error_flag() == 0
