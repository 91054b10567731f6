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
