"""GPU checks of the proposal network against the FP64 oracle (oracle/cnn.py),
element by element.

Each layer is checked on its own inputs: the BF16 tensors the GPU kept (input
activations, output gradients) go through the oracle's FP64 convolution, and
every GPU output element must be a correct rounding of a value within the FP32
accumulation bound of the FP64 result:
  * BF16 outputs (activations, pre-activation gradients): round_bf16(z - e) <=
    g <= round_bf16(z + e) (after the ReLU or the ReLU mask), with
    e = n 2^-23 sum|terms| for n accumulated terms (FP32 accumulation, one
    rounding per add, truncating or rounding; the BF16 x BF16 products of the
    tensor cores are exact);
  * FP32 outputs (logits, weight and bias gradients): |g - z| <= e.
A layer whose inputs are exact can then differ from the oracle only by the one
rounding of its output, so a wrong tap, channel, sign or mask fails here even
on a few elements. The share of BF16 elements that took the other neighbour of a
boundary value is reported. The Adam update is compared per parameter with
oracle.cnn.adam over two steps.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U23 = 2.0 ** -23


def _oc():
    from oracle import cnn as oc
    return oc


def _check_bf16(g, z, e, label, relu=True, mask=None):
    """g: GPU BF16 values (float64), z: FP64 values before rounding (before the ReLU
    or mask), e: per-element accumulation bound. Returns the share of elements that
    differ from round_bf16(z)."""
    oc = _oc()
    lo, hi = z - e, z + e
    if relu:
        lo, hi, zz = np.maximum(lo, 0.0), np.maximum(hi, 0.0), np.maximum(z, 0.0)
    else:
        zz = z
    if mask is not None:
        lo, hi, zz = lo * mask, hi * mask, zz * mask
    rlo, rhi = oc.round_bf16(lo), oc.round_bf16(hi)
    bad = ~((g >= rlo) & (g <= rhi))
    assert not bad.any(), (f"{label}: {int(bad.sum())} of {g.size} elements outside their rounding "
                           f"interval, first at {np.argwhere(bad)[0].tolist()}: gpu {g[bad][0]} vs "
                           f"oracle {zz[bad][0]}")
    return float(np.mean(g != oc.round_bf16(zz)))


def _check_f32(g, z, e, label):
    d = np.abs(g - z)
    bad = d > e
    assert not bad.any(), (f"{label}: {int(bad.sum())} of {g.size} elements beyond the bound, worst "
                           f"{float((d - e).max())} at {np.unravel_index(int(np.argmax(d - e)), d.shape)}")


def _bound(x, W, b, n):
    """n 2^-23 sum |terms| of conv(x, W, b), elementwise."""
    oc = _oc()
    return n * U23 * oc.conv(np.abs(x), np.abs(W), np.abs(b))


# ---------------------------------------------------------------- conv64 building block

def _run_conv(lib, x, w, bias, mask, relu, transpose):
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    wpack = torch.empty(73728, dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.qlp_cnn_pack_w64(ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(wpack.data_ptr()),
                              int(transpose), stream)
    assert rc == 0
    y = torch.empty_like(x)
    rc = lib.qlp_cnn_conv64(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(wpack.data_ptr()),
                            ctypes.c_void_p(bias.data_ptr() if bias is not None else 0),
                            ctypes.c_void_p(mask.data_ptr() if mask is not None else 0),
                            ctypes.c_void_p(y.data_ptr()), x.shape[0], x.shape[1], int(relu),
                            ctypes.c_void_p(err.data_ptr()), stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return y


@pytest.mark.parametrize("B,L", [(1, 128), (3, 512), (5, 1024)])
def test_conv64_forward_matches_oracle(gpu_lib, B, L):
    import torch
    oc = _oc()
    g = torch.Generator(device="cpu").manual_seed(B * 1000 + L)
    x = torch.randn(B, L, 64, generator=g).to(torch.bfloat16)
    w = torch.randn(9, 64, 64, generator=g) * 0.05
    bias = torch.randn(64, generator=g) * 0.1
    lib = gpu_lib.lib()
    xd = x.float().numpy().astype(np.float64)
    wd = oc.round_bf16(w.numpy())                          # the tensor cores' BF16 weights
    bd = bias.numpy().astype(np.float64)
    y = _run_conv(lib, x.cuda(), w.cuda(), bias.cuda(), None, True, False).float().cpu().numpy()
    _check_bf16(y.astype(np.float64), oc.conv(xd, wd, bd), _bound(xd, wd, bd, 577), "conv64 relu+bias")
    y2 = _run_conv(lib, x.cuda(), w.cuda(), None, None, False, False).float().cpu().numpy()
    z0 = np.zeros(64)
    _check_bf16(y2.astype(np.float64), oc.conv(xd, wd, z0), _bound(xd, wd, z0, 576), "conv64 plain",
                relu=False)


def test_conv64_input_gradient_matches_oracle(gpu_lib):
    # the transposed packing computes dx[m] = sum_k W[k]^T dy[m - k + 4], masked where mask > 0
    import torch
    oc = _oc()
    g = torch.Generator(device="cpu").manual_seed(7)
    B, L = 2, 256
    w = torch.randn(9, 64, 64, generator=g) * 0.05
    dy = torch.randn(B, L, 64, generator=g).to(torch.bfloat16)
    mask = torch.randn(B, L, 64, generator=g).to(torch.bfloat16)
    dx = _run_conv(gpu_lib.lib(), dy.cuda(), w.cuda(), None, mask.cuda(), False, True).float().cpu().numpy()
    wd = oc.round_bf16(w.numpy())
    dyd = dy.float().numpy().astype(np.float64)
    # dx = conv(dy, W') with W'[k][ci][co] = W[8 - k][co][ci]
    wt = np.ascontiguousarray(np.transpose(wd[::-1], (0, 2, 1)))
    z = oc.conv(dyd, wt, np.zeros(64))
    e = _bound(dyd, wt, np.zeros(64), 576)
    m = (mask.float().numpy() > 0).astype(np.float64)
    _check_bf16(dx.astype(np.float64), z, e, "conv64 input gradient", relu=False, mask=m)


@pytest.mark.parametrize("B,L", [(1, 128), (3, 512), (2, 4096)])
def test_conv64_weight_gradient_matches_oracle(gpu_lib, B, L):
    # dW[kk][co][ci] = sum_p dY[p][co] X[p + kk - 4][ci], db = sum_p dY[p]: the
    # oracle's conv_backward on the same BF16 operands, per element within the FP32
    # accumulation bound
    import torch
    from paper_2302_01293_gb300 import qlpbls
    oc = _oc()
    g = torch.Generator(device="cpu").manual_seed(11)
    x = torch.randn(B, L, 64, generator=g).to(torch.bfloat16)
    dy = torch.randn(B, L, 64, generator=g).to(torch.bfloat16)
    dw, db = qlpbls.conv64_wgrad(dy.cuda(), x.cuda())
    xd = x.float().numpy().astype(np.float64)
    dyd = dy.float().numpy().astype(np.float64)
    W0 = np.zeros((9, 64, 64))
    dW, dB, _ = oc.conv_backward(xd, W0, dyd)
    aW, aB, _ = oc.conv_backward(np.abs(xd), W0, np.abs(dyd))
    n = B * L + 64
    _check_f32(dw.cpu().numpy().astype(np.float64), dW, n * U23 * aW, "conv64 weight gradient")
    _check_f32(db.cpu().numpy().astype(np.float64), dB, n * U23 * aB, "conv64 bias gradient")


# ---------------------------------------------------------------- the whole network

def _net_case(gpu_lib, B=2, L=256, seed=4, pos_weight=30.0):
    import torch
    oc = _oc()
    rng = np.random.default_rng(seed)
    snr = rng.normal(size=(B, L)).astype(np.float32) * 2.0
    mask = (rng.uniform(size=(B, L)) > 0.1).astype(np.float32)
    harm = [np.roll(snr * mask, d, axis=1) * mask for d in (37, -37, 59, -59)]  # stand-ins for 2P .. P/3
    x0 = torch.tensor(np.stack([snr * mask, mask] + harm, axis=-1)).to(torch.bfloat16)
    labels = np.zeros((B, L), np.float32)
    labels[0, 40:43] = 1.0
    labels[1 % B, 200:203] = 1.0
    params = oc.init_params(3).astype(np.float32)
    net = gpu_lib.CNN(max_batch=B, length=L, seed=1)
    net.set_params(params)
    net.backward(x0.cuda(), torch.tensor(labels).cuda(), pos_weight)
    return net, x0, labels, params


def test_network_layers_match_oracle(gpu_lib):
    """Forward and backward of the 6-layer network, layer by layer on the GPU's own
    stored tensors, against the oracle's FP64 convolutions (module docstring)."""
    from paper_2302_01293_gb300 import qlpbls
    oc = _oc()
    B, L, pw = 2, 256, 30.0
    net, x0, labels, params = _net_case(gpu_lib, B, L, pos_weight=pw)
    p = oc.unflatten(params.astype(np.float64))
    act = {0: x0.float().numpy().astype(np.float64)}
    gact = {}
    for k in range(1, 6):
        act[k] = net.tensor(qlpbls.CNN_ACT, k, B).astype(np.float64)
        gact[k] = net.tensor(qlpbls.CNN_GACT, k, B).astype(np.float64)
    logit = net.tensor(qlpbls.CNN_LOGIT, 0, B).astype(np.float64)
    dlogit = net.tensor(qlpbls.CNN_DLOGIT, 0, B).astype(np.float64)
    _, grad = net.params(with_grads=True)
    gg = oc.unflatten(grad.astype(np.float64))
    flips = {}

    # forward: layer k from the GPU's layer k-1 output
    for k in range(1, 6):
        W = oc.round_bf16(p[f"W{k}"]) if k >= 2 else p[f"W{k}"]
        n = 9 * act[k - 1].shape[2] + 1
        flips[f"act{k}"] = _check_bf16(act[k], oc.conv(act[k - 1], W, p[f"b{k}"]),
                                       _bound(act[k - 1], W, p[f"b{k}"], n), f"layer {k} output")
    z6 = oc.conv(act[5], p["W6"], p["b6"])[..., 0]
    _check_f32(logit, z6, _bound(act[5], p["W6"], p["b6"], 577)[..., 0], "logits")

    # loss and its gradient from the GPU's logits
    loss_o, dz = oc.bce(logit, labels, pw)
    assert net.loss() == pytest.approx(loss_o, rel=1e-5)
    _check_f32(dlogit, dz, 8 * 2.0 ** -24 * ((pw * labels + 1.0) / logit.size + np.abs(dz)), "dlogits")

    # backward: gradients of layer k's weights and of layer k-1's pre-activation
    dW, db, dx = oc.conv_backward(act[5], p["W6"], dlogit[..., None])
    aW, aB, ax = oc.conv_backward(np.abs(act[5]), np.abs(p["W6"]), np.abs(dlogit[..., None]))
    npos = B * L + 64
    _check_f32(gg["W6"], dW, npos * U23 * aW, "W6 gradient")
    _check_f32(gg["b6"], db, npos * U23 * aB, "b6 gradient")
    flips["gact5"] = _check_bf16(gact[5], dx, 10 * U23 * ax, "layer 5 pre-activation gradient",
                                 relu=False, mask=(act[5] > 0).astype(np.float64))
    for k in range(5, 0, -1):
        W = oc.round_bf16(p[f"W{k}"]) if k >= 2 else p[f"W{k}"]
        dW, db, dx = oc.conv_backward(act[k - 1], W, gact[k])
        aW, aB, ax = oc.conv_backward(np.abs(act[k - 1]), np.abs(W), np.abs(gact[k]))
        _check_f32(gg[f"W{k}"], dW, npos * U23 * aW, f"W{k} gradient")
        _check_f32(gg[f"b{k}"], db, npos * U23 * aB, f"b{k} gradient")
        if k >= 2:
            flips[f"gact{k - 1}"] = _check_bf16(gact[k - 1], dx, 577 * U23 * ax,
                                                f"layer {k - 1} pre-activation gradient", relu=False,
                                                mask=(act[k - 1] > 0).astype(np.float64))
    # a correct rounding takes the other neighbour only near a BF16 boundary
    assert max(flips.values()) < 0.01, flips
    net.close()


def test_network_end_to_end_against_oracle(gpu_lib):
    """The same network against the oracle run end to end in the GPU's precision
    (BF16 at exactly the tensors the GPU stores in BF16): here the BF16 boundary
    cases of one layer feed the next, so agreement is per element to a stated
    propagation bound: logits within 2^-7 of their RMS, every gradient element
    within 2^-5 of its tensor's RMS (a BF16 ulp is 2^-8 relative; a handful of
    boundary flips per layer moves a sum of 576 terms by far less), loss 1e-4."""
    oc = _oc()
    B, L, pw = 2, 256, 30.0
    net, x0, labels, params = _net_case(gpu_lib, B, L, pos_weight=pw)
    from paper_2302_01293_gb300 import qlpbls
    logit = net.tensor(qlpbls.CNN_LOGIT, 0, B).astype(np.float64)
    xx = x0.float().numpy().astype(np.float64)
    lo, _, _ = oc.forward(params.astype(np.float64), xx, bf16=True)
    rms = float(np.sqrt(np.mean(lo * lo)))
    assert np.abs(logit - lo).max() <= 2.0 ** -7 * rms
    loss, ograd = oc.backward(params.astype(np.float64), xx, labels, pw, bf16=True)
    assert net.loss() == pytest.approx(loss, rel=1e-4)
    _, ggrad = net.params(with_grads=True)
    o = 0
    for name, shp in oc.SHAPES:
        n = int(np.prod(shp))
        a, b = ggrad[o:o + n].astype(np.float64), ograd[o:o + n]
        o += n
        r = float(np.sqrt(np.mean(b * b)))
        assert np.abs(a - b).max() <= 2.0 ** -5 * r + 1e-30, (name, float(np.abs(a - b).max()), r)
    net.close()


def test_adam_steps_match_oracle(gpu_lib):
    """Two Adam steps (bias-corrected, beta 0.9 / 0.999, eps 1e-8) on the GPU's own
    gradients against oracle.cnn.adam per parameter: relative 1e-6 of the parameter
    plus 1e-6 of the learning rate (FP32 moments and update)."""
    import torch
    oc = _oc()
    B, L, pw, lr = 2, 256, 30.0, 1e-3
    net, x0, labels, params = _net_case(gpu_lib, B, L, pos_weight=pw)
    p0 = params.astype(np.float64)
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    for step in (1, 2):
        if step == 2:
            net.backward(x0.cuda(), torch.tensor(labels).cuda(), pw)
        pg, grad = net.params(with_grads=True)
        net.adam_step(lr)
        torch.cuda.synchronize()
        p_new = net.params().astype(np.float64)
        po, m, v = oc.adam(pg.astype(np.float64), grad.astype(np.float64), m, v, step, lr)
        d = np.abs(p_new - po)
        tol = 1e-6 * np.abs(po) + 1e-6 * lr
        assert np.all(d <= tol), (step, float((d - tol).max()), int(np.argmax(d - tol)))
    net.close()


def test_training_reduces_loss(gpu_lib):
    """A few Adam steps on a fixed batch lower the loss (the update is wired)."""
    import torch
    B, L = 4, 512
    rng = np.random.default_rng(8)
    snr = rng.normal(size=(B, L)).astype(np.float32)
    labels = np.zeros((B, L), np.float32)
    for b in range(B):
        k = int(rng.integers(20, L - 20))
        snr[b, k - 1:k + 2] += 8.0
        labels[b, k - 1:k + 2] = 1.0
    zero = np.zeros_like(snr)
    x0 = torch.tensor(np.stack([snr, np.ones_like(snr), zero, zero, zero, zero], -1)).to(torch.bfloat16).cuda()
    lab = torch.tensor(labels).cuda()
    net = gpu_lib.CNN(max_batch=B, length=L, seed=2)
    net.backward(x0, lab, 20.0)
    l0 = net.loss()
    for _ in range(30):
        net.train_step(x0, lab, 20.0, 2e-3)
    net.backward(x0, lab, 20.0)
    l1 = net.loss()
    assert l1 < 0.5 * l0
    net.close()
