"""Learned-initialiser layers (BF16 tensor-core kernels) against the FP64 reference.

Layer tests feed both sides the same BF16-rounded operands, so they differ
only by FP32 accumulation (tolerance 1e-5).  The whole-decoder test also
rounds every activation to BF16 on the GPU side; its error is reported
separately with a loose bound.
"""

import ctypes

import numpy as np
import pytest
import torch

from oracle import decoder_oracle as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _bf(t):
    """float -> (bf16 bit tensor on GPU, its exact value in float64 on CPU)."""
    b = t.to(torch.bfloat16)
    return b.view(torch.int16).cuda().contiguous(), b.double().cpu()


def _rel(a, b):
    a = a.double().cpu()
    b = b.double().cpu()
    return float((a - b).norm() / b.norm())


SHAPES = [(2, 37, 70, 45), (1, 128, 128, 64), (3, 5, 1, 200)]


@pytest.mark.parametrize("B,Ci,Co,T", SHAPES)
def test_convt_forward(B, Ci, Co, T):
    from paper_2602_11896_gb300 import _native
    lib = _native.load()
    g = torch.Generator().manual_seed(B * 1000 + Ci)
    xb, x64 = _bf(torch.randn(B, Ci, T, generator=g))
    wb, w64 = _bf(torch.randn(Ci, Co, 9, generator=g) * 0.1)
    bias = torch.randn(Co, generator=g)
    y = torch.empty(B, Co, 2 * T, device="cuda")
    assert lib.jtfs_convt_forward(_p(xb), _p(wb), _p(bias.cuda()), _p(y), B, Ci, Co, T, _s()) == 0
    ref = D.conv_transpose(x64, w64, bias.double())
    assert _rel(y, ref) <= 1e-5


@pytest.mark.parametrize("B,Ci,Co,T", SHAPES)
def test_convt_gradients(B, Ci, Co, T):
    from paper_2602_11896_gb300 import _native
    lib = _native.load()
    g = torch.Generator().manual_seed(7 + T)
    xb, x64 = _bf(torch.randn(B, Ci, T, generator=g))
    wb, w64 = _bf(torch.randn(Ci, Co, 9, generator=g) * 0.1)
    dyf = torch.randn(B, Co, 2 * T, generator=g)
    dyb, dy64 = _bf(dyf)
    x64.requires_grad_(True)
    w64.requires_grad_(True)
    b64 = torch.zeros(Co, dtype=torch.float64, requires_grad=True)
    (D.conv_transpose(x64, w64, b64) * dy64).sum().backward()
    dx = torch.empty(B, Ci, T, device="cuda")
    assert lib.jtfs_convt_backward_data(_p(dyb), _p(wb), _p(dx), B, Ci, Co, T, _s()) == 0
    assert _rel(dx, x64.grad) <= 1e-5
    ws = torch.empty(max(lib.jtfs_convt_weight_workspace_bytes(B, Ci, Co, T), 4), dtype=torch.uint8, device="cuda")
    dw = torch.empty(Ci, Co, 9, device="cuda")
    db = torch.empty(Co, device="cuda")
    dy32 = dy64.float().cuda()
    assert lib.jtfs_convt_backward_weight(_p(xb), _p(dyb), _p(dy32), _p(dw), _p(db), B, Ci, Co, T, _p(ws), _s()) == 0
    assert _rel(dw, w64.grad) <= 1e-5
    assert _rel(db, dy64.sum((0, 2))) <= 1e-5


def test_gelu_and_adam():
    from paper_2602_11896_gb300 import _native
    lib = _native.load()
    z = torch.linspace(-6, 6, 1001, device="cuda")
    h = torch.empty(1001, dtype=torch.int16, device="cuda")
    assert lib.jtfs_gelu_forward(_p(z), _p(h), z.numel(), _s()) == 0
    ref = D.gelu(z.cpu())
    assert (h.view(torch.bfloat16).double().cpu() - ref).abs().max().item() <= 2 ** -8 * (ref.abs().max().item() + 1)
    dh = torch.randn(1001, device="cuda")
    dz = torch.empty_like(dh)
    assert lib.jtfs_gelu_backward(_p(dh), _p(z), _p(dz), z.numel(), _s()) == 0
    zz = z.double().cpu().requires_grad_(True)
    (D.gelu(zz) * dh.double().cpu()).sum().backward()
    assert _rel(dz, zz.grad) <= 1e-5
    p = torch.randn(100, device="cuda")
    p0 = p.clone()
    gr = torch.randn(100, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    assert lib.jtfs_adam_update(_p(p), _p(gr), _p(m), _p(v), ctypes.c_void_p(0), 100, 0.01, 1, _s()) == 0
    assert torch.allclose(p, p0 - 0.01 * gr / (gr.abs() + 1e-8), atol=1e-6)


def test_decoder_forward_backward_bf16_error_report():
    """Whole 3-layer decoder vs an FP64 decoder with the same (BF16-rounded) weights."""
    from paper_2602_11896_gb300.initialiser import Decoder
    dec = Decoder(in_channels=12, frames=16, channels=32, layers=3, seed=3)
    phi = torch.rand(2, 12, 16, device="cuda")
    y = dec.forward(phi)
    ws = [w.cpu().to(torch.bfloat16).double().requires_grad_(True) for w in dec.w]
    bs = [b.cpu().double().requires_grad_(True) for b in dec.b]
    h = phi.cpu().to(torch.bfloat16).double()
    for li in range(3):
        z = D.conv_transpose(h, ws[li], bs[li])
        h = D.gelu(z) if li < 2 else z
    ref = h.reshape(2, -1)
    err_fwd = _rel(y, ref)
    dy = torch.randn_like(y)
    dec.backward(dy)
    (ref * dy.double().cpu()).sum().backward()
    err_w = max(_rel(dec.gw[i], ws[i].grad) for i in range(3))
    print(f"BF16 decoder error vs FP64: forward {err_fwd:.2e}, weight gradients {err_w:.2e}")
    assert err_fwd <= 3e-2 and err_w <= 5e-2
