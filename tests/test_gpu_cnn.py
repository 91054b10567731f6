"""GPU checks of the CNN building blocks against plain PyTorch FP32 on the same
BF16-rounded operands (the tensor-core conv accumulates in FP32 and stores BF16)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _conv_ref(x, w, bias, relu):
    import torch
    import torch.nn.functional as F
    xf = x.float().permute(0, 2, 1)                    # [B, 64, L]
    wr = w.to(torch.bfloat16).float().permute(1, 2, 0)  # [co, ci, k]
    y = F.conv1d(xf, wr, bias, padding=4)
    if relu:
        y = torch.relu(y)
    return y.permute(0, 2, 1)


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
def test_conv64_forward_matches_torch(gpu_lib, B, L):
    import torch
    g = torch.Generator(device="cpu").manual_seed(B * 1000 + L)
    x = torch.randn(B, L, 64, generator=g).to(torch.bfloat16).cuda()
    w = (torch.randn(9, 64, 64, generator=g) * 0.05).cuda()
    bias = (torch.randn(64, generator=g) * 0.1).cuda()
    lib = gpu_lib.lib()
    y = _run_conv(lib, x, w, bias, None, True, False).float()
    ref = _conv_ref(x, w, bias, True)
    scale = ref.abs().max().item()
    assert (y - ref).abs().max().item() <= 1e-2 * scale
    # no ReLU, no bias
    y2 = _run_conv(lib, x, w, None, None, False, False).float()
    ref2 = _conv_ref(x, w, None, False)
    assert (y2 - ref2).abs().max().item() <= 1e-2 * ref2.abs().max().item()


def test_conv64_input_gradient_matches_autograd(gpu_lib):
    import torch
    import torch.nn.functional as F
    g = torch.Generator(device="cpu").manual_seed(7)
    B, L = 2, 256
    x = torch.randn(B, L, 64, generator=g).to(torch.bfloat16).cuda()
    w = (torch.randn(9, 64, 64, generator=g) * 0.05).cuda()
    dy = torch.randn(B, L, 64, generator=g).to(torch.bfloat16).cuda()
    mask = torch.randn(B, L, 64, generator=g).to(torch.bfloat16).cuda()
    xf = x.float().permute(0, 2, 1).clone().requires_grad_(True)
    wr = w.to(torch.bfloat16).float().permute(1, 2, 0)
    y = F.conv1d(xf, wr, None, padding=4)
    y.backward(dy.float().permute(0, 2, 1))
    ref = xf.grad.permute(0, 2, 1) * (mask.float() > 0)
    dx = _run_conv(gpu_lib.lib(), dy, w, None, mask, False, True).float()
    assert (dx - ref).abs().max().item() <= 1e-2 * ref.abs().max().item()


@pytest.mark.parametrize("B,L", [(1, 128), (3, 512), (2, 4096)])
def test_conv64_weight_gradient_matches_autograd(gpu_lib, B, L):
    # dW[kk][co][ci] = sum_p dY[p][co] X[p + kk - 4][ci] against torch's conv1d weight gradient
    # on the same BF16 operands (FP32 sums; tolerance for the summation order)
    import torch
    import torch.nn.functional as F
    from paper_2302_01293_gb300 import qlpbls
    g = torch.Generator(device="cpu").manual_seed(11)
    x = torch.randn(B, L, 64, generator=g).to(torch.bfloat16)
    dy = torch.randn(B, L, 64, generator=g).to(torch.bfloat16)
    dw, db = qlpbls.conv64_wgrad(dy.cuda(), x.cuda())
    xf = x.float().permute(0, 2, 1).requires_grad_(False)
    w = torch.zeros(64, 64, 9, requires_grad=True)
    y = F.conv1d(xf, w, padding=4)
    y.backward(dy.float().permute(0, 2, 1))
    ref = w.grad.permute(2, 0, 1)                                # [kk][co][ci]
    scale = float(np.sqrt(B * L))
    np.testing.assert_allclose(dw.cpu().numpy(), ref.numpy(), atol=2e-5 * scale, rtol=1e-4)
    np.testing.assert_allclose(db.cpu().numpy(), dy.float().sum((0, 1)).numpy(), atol=1e-5 * scale, rtol=1e-4)


def test_network_gradients_match_oracle(gpu_lib):
    """Full forward + backward of the 6-layer network on the GPU vs the oracle taken
    in the GPU's precision (BF16 activations, activation gradients and middle-layer
    weights; FP64 elsewhere): loss to 1e-3, every parameter tensor's gradient to
    2e-2 relative L2 and cosine >= 0.999. Against the all-FP64 oracle the loss
    agrees to 1e-2 and every gradient keeps cosine >= 0.99."""
    import torch
    from oracle import cnn as oc
    B, L = 2, 256
    rng = np.random.default_rng(4)
    snr = rng.normal(size=(B, L)).astype(np.float32)
    mask = (rng.uniform(size=(B, L)) > 0.1).astype(np.float32)
    x0 = np.stack([snr, mask], axis=-1)
    x0 = torch.tensor(x0).to(torch.bfloat16)
    labels = np.zeros((B, L), np.float32)
    labels[0, 40:43] = 1.0
    labels[1, 200:203] = 1.0
    params = oc.init_params(3).astype(np.float32)
    net = gpu_lib.CNN(max_batch=B, length=L, seed=1)
    net.set_params(params)
    net.backward(x0.cuda(), torch.tensor(labels).cuda(), 30.0)
    gloss = net.loss()
    _, ggrad = net.params(with_grads=True)
    # oracle on the same BF16-rounded input and FP32 parameters
    xx = x0.float().numpy().astype(np.float64)
    loss, ograd = oc.backward(params.astype(np.float64), xx, labels, 30.0, bf16=True)
    loss64, ograd64 = oc.backward(params.astype(np.float64), xx, labels, 30.0)
    assert gloss == pytest.approx(loss, rel=1e-3)
    assert gloss == pytest.approx(loss64, rel=1e-2)
    o = 0
    for name, shp in oc.SHAPES:
        n = int(np.prod(shp))
        a, b, c = ggrad[o:o + n].astype(np.float64), ograd[o:o + n], ograd64[o:o + n]
        o += n
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        cos64 = float(a @ c / max(np.linalg.norm(a) * np.linalg.norm(c), 1e-30))
        assert rel <= 2e-2 and cos >= 0.999 and cos64 >= 0.99, (name, rel, cos, cos64)
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
    x0 = torch.tensor(np.stack([snr, np.ones_like(snr)], -1)).to(torch.bfloat16).cuda()
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
