"""Learned-initialiser layers (BF16 tensor-core kernels) against the FP64 reference.

Layer tests feed both sides the same BF16-rounded operands, so they differ
only by FP32 accumulation order (tolerance 1e-5).  Activations are
channels-last on the GPU ([B][T][C]); the reference works in [B][C][T].
The whole-decoder test also rounds every activation and gradient to BF16 on
the GPU side; its error is reported separately with a loose bound.
"""

import ctypes

import pytest
import torch

from oracle import decoder_oracle as D

pytestmark = pytest.mark.gpu

C = 128


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def lib():
    from paper_2602_11896_gb300 import _native
    return _native.load()


@pytest.fixture(autouse=True)
def _no_barrier_timeouts(lib):
    yield
    torch.cuda.synchronize()
    assert lib.jtfs_decoder_error() == 0


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _bf(t):
    """float tensor -> (bf16 bits on the GPU, the same values in float64 on the CPU)."""
    b = t.to(torch.bfloat16)
    return b.view(torch.int16).cuda().contiguous(), b.double().cpu()


def _from_bf(bits):
    return bits.cpu().view(torch.bfloat16).double()


def _rel(a, b):
    a = a.detach().double().cpu()
    b = b.detach().double().cpu()
    return float((a - b).norm() / b.norm())


def _channels_last_input(B, Ci, T, cip, g):
    """x [B][T][cip] bf16 (channels >= Ci zero) and its float64 [B][Ci][T] value."""
    x = torch.zeros(B, T, cip)
    x[:, :, :Ci] = torch.randn(B, T, Ci, generator=g)
    xb, x64 = _bf(x)
    return xb, x64[:, :, :Ci].permute(0, 2, 1).contiguous()


def _packed(lib, w, with_wd):
    Ci = w.shape[0]
    cip = lib.jtfs_convt_padded_channels(Ci)
    wf = torch.empty(2 * C, 5 * cip, dtype=torch.int16, device="cuda")
    wd = torch.empty(C, 9 * C, dtype=torch.int16, device="cuda") if with_wd else None
    assert lib.jtfs_convt_pack_weights(_p(w), _p(wf), _p(wd), Ci, C, _s()) == 0
    return cip, wf, wd


FWD_SHAPES = [(2, 37, 45), (1, 128, 300), (3, 801, 130), (2, 128, 1024)]


@pytest.mark.parametrize("B,Ci,T", FWD_SHAPES)
def test_convt_forward(lib, B, Ci, T):
    g = torch.Generator().manual_seed(B * 1000 + Ci + T)
    cip = lib.jtfs_convt_padded_channels(Ci)
    xb, x64 = _channels_last_input(B, Ci, T, cip, g)
    w = (torch.randn(Ci, C, 9, generator=g) * 0.1).to(torch.bfloat16).float().cuda()
    bias = torch.randn(C, generator=g).cuda()
    _, wf, _ = _packed(lib, w, False)
    z = torch.empty(B, 2 * T, C, device="cuda")
    h = torch.empty(B, 2 * T, C, dtype=torch.int16, device="cuda")
    assert lib.jtfs_convt_forward(_p(xb), _p(wf), _p(bias), _p(z), _p(h), B, cip, C, T, _s()) == 0
    ref = D.conv_transpose(x64, w.cpu().double(), bias.cpu().double())  # [B][C][2T]
    assert _rel(z.permute(0, 2, 1), ref) <= 1e-5
    hg = D.gelu(ref)
    assert _rel(_from_bf(h).permute(0, 2, 1), hg) <= 2 ** -8


@pytest.mark.parametrize("B,T", [(2, 45), (1, 300), (2, 1024)])
@pytest.mark.parametrize("gelu", [True, False])
def test_convt_backward_data(lib, B, T, gelu):
    g = torch.Generator().manual_seed(7 + T + gelu)
    gb, g64 = _bf(torch.randn(B, 2 * T, C, generator=g))
    w = (torch.randn(C, C, 9, generator=g) * 0.1).to(torch.bfloat16).float().cuda()
    _, _, wd = _packed(lib, w, True)
    zprev = torch.randn(B, T, C, generator=g).cuda() if gelu else None
    out32 = torch.empty(B, T, C, device="cuda")
    out16 = torch.empty(B, T, C, dtype=torch.int16, device="cuda")
    assert lib.jtfs_convt_backward_data(_p(gb), _p(wd), _p(zprev), _p(out32), _p(out16), B, C, C, T, _s()) == 0
    x = torch.zeros(B, C, T, dtype=torch.float64, requires_grad=True)
    (D.conv_transpose(x, w.cpu().double(), torch.zeros(C, dtype=torch.float64)) * g64.permute(0, 2, 1)).sum().backward()
    ref = x.grad
    if gelu:
        zz = zprev.cpu().double().permute(0, 2, 1).requires_grad_(True)
        D.gelu(zz).sum().backward()
        ref = ref * zz.grad
    assert _rel(out32.permute(0, 2, 1), ref) <= 1e-5
    assert _rel(_from_bf(out16).permute(0, 2, 1), ref) <= 2 ** -8


@pytest.mark.parametrize("B,Ci,T", [(2, 37, 45), (1, 128, 300), (2, 801, 100), (2, 128, 3000), (32, 128, 64)])
def test_convt_backward_weight(lib, B, Ci, T):
    g = torch.Generator().manual_seed(11 + Ci + T)
    cip = lib.jtfs_convt_padded_channels(Ci)
    xb, x64 = _channels_last_input(B, Ci, T, cip, g)
    gb, g64 = _bf(torch.randn(B, 2 * T, C, generator=g))
    ws = torch.empty(max(lib.jtfs_convt_weight_workspace_bytes(B, cip, C, T), 16), dtype=torch.uint8, device="cuda")
    dw = torch.empty(Ci, C, 9, device="cuda")
    assert lib.jtfs_convt_backward_weight(_p(xb), _p(gb), _p(dw), B, Ci, cip, C, T, _p(ws), _s()) == 0
    w = torch.zeros(Ci, C, 9, dtype=torch.float64, requires_grad=True)
    (D.conv_transpose(x64, w, torch.zeros(C, dtype=torch.float64)) * g64.permute(0, 2, 1)).sum().backward()
    assert _rel(dw, w.grad) <= 1e-5


def test_bias_grad(lib):
    g = torch.Generator().manual_seed(3)
    rows = 2 * 1500 + 7
    x = torch.randn(rows, C, generator=g)
    ws = torch.empty(lib.jtfs_convt_bias_workspace_bytes(rows), dtype=torch.uint8, device="cuda")
    db = torch.empty(C, device="cuda")
    assert lib.jtfs_convt_bias_grad(_p(x.cuda()), _p(db), rows, C, _p(ws), _s()) == 0
    assert _rel(db, x.double().sum(0)) <= 1e-6


@pytest.mark.parametrize("B,T", [(2, 45), (3, 1000)])
def test_output_layer(lib, B, T):
    g = torch.Generator().manual_seed(5 + T)
    xb, x64 = _channels_last_input(B, C, T, C, g)
    w = (torch.randn(C, 1, 9, generator=g) * 0.1).cuda()
    bias = torch.randn(1, generator=g).cuda()
    y = torch.empty(B, 2 * T, device="cuda")
    assert lib.jtfs_convt_out_forward(_p(xb), _p(w), _p(bias), _p(y), B, C, T, _s()) == 0
    w64 = w.cpu().double().requires_grad_(True)
    b64 = bias.cpu().double().requires_grad_(True)
    xr = x64.clone().requires_grad_(True)
    ref = D.conv_transpose(xr, w64, b64)[:, 0]
    assert _rel(y, ref) <= 1e-5
    dy = torch.randn(B, 2 * T, generator=g)
    (ref * dy.double()).sum().backward()
    zprev = torch.randn(B, T, C, generator=g)
    g32 = torch.empty(B, T, C, device="cuda")
    assert lib.jtfs_convt_out_backward_data(_p(dy.cuda()), _p(w), _p(zprev.cuda()), _p(g32), None, B, C, T,
                                            _s()) == 0
    zz = zprev.double().permute(0, 2, 1).requires_grad_(True)
    D.gelu(zz).sum().backward()
    assert _rel(g32.permute(0, 2, 1), xr.grad * zz.grad) <= 1e-5
    ws = torch.empty(lib.jtfs_convt_out_workspace_bytes(B, T), dtype=torch.uint8, device="cuda")
    dw = torch.empty(C, 1, 9, device="cuda")
    db = torch.empty(1, device="cuda")
    assert lib.jtfs_convt_out_backward_weight(_p(xb), _p(dy.cuda()), _p(dw), _p(db), B, C, T, _p(ws), _s()) == 0
    assert _rel(dw, w64.grad) <= 1e-5
    assert _rel(db, b64.grad) <= 1e-5


def test_pack_input(lib):
    g = torch.Generator().manual_seed(9)
    B, Cin, T = 2, 801, 70
    phi = torch.rand(B, Cin, T, generator=g)
    scale = torch.rand(Cin, generator=g) + 0.5
    cip = lib.jtfs_convt_padded_channels(Cin)
    assert cip == 896
    x = torch.empty(B, T, cip, dtype=torch.int16, device="cuda")
    assert lib.jtfs_convt_pack_input(_p(phi.cuda()), _p(scale.cuda()), _p(x), B, Cin, T, _s()) == 0
    ref = torch.zeros(B, T, cip)
    ref[:, :, :Cin] = (phi * scale[None, :, None]).permute(0, 2, 1)
    assert torch.equal(x.cpu(), ref.to(torch.bfloat16).view(torch.int16))


def test_adam(lib):
    p = torch.randn(100, device="cuda")
    p0 = p.clone()
    gr = torch.randn(100, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    assert lib.jtfs_adam_update(_p(p), _p(gr), _p(m), _p(v), None, 100, 0.01, 1, _s()) == 0
    assert torch.allclose(p, p0 - 0.01 * gr / (gr.abs() + 1e-8), atol=1e-6)


def test_argument_errors(lib):
    t = torch.empty(1024, dtype=torch.int16, device="cuda")
    f = torch.empty(1024, device="cuda")
    assert lib.jtfs_convt_forward(_p(t), _p(t), _p(f), _p(f), None, 1, 128, 64, 4, _s()) == -1   # Co != 128
    assert lib.jtfs_convt_forward(_p(t), _p(t), _p(f), _p(f), None, 1, 100, 128, 4, _s()) == -1  # Cip % 128
    assert lib.jtfs_convt_backward_data(_p(t), _p(t), None, None, None, 1, 128, 128, 4, _s()) == -1


def test_decoder_forward_backward_bf16_error_report():
    """Whole 3-layer decoder vs an FP64 decoder with the same (BF16-rounded) weights."""
    from paper_2602_11896_gb300.initialiser import Decoder
    dec = Decoder(in_channels=12, frames=16, channels=128, layers=3, seed=3)
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
    err_b = max(_rel(dec.gb[i], bs[i].grad) for i in range(3))
    dec.check_errors()
    print(f"BF16 decoder error vs FP64: forward {err_fwd:.2e}, weight gradients {err_w:.2e}, bias {err_b:.2e}")
    assert err_fwd <= 3e-2 and err_w <= 5e-2 and err_b <= 5e-2
