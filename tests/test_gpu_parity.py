"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: relative L2 error <= 1e-4 per Phi block (S0, first order, each
active n2) and for gradients, the FP32-versus-FP64 bound the method's
workloads state.
"""

import math

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from workloads import get_workload, signals

pytestmark = pytest.mark.gpu

TOL = 1e-4

CASES = {
    "tiny_n256": dict(N=256, J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2),
    "tiny_n512_q3": dict(N=512, J=5, Q=3, Q2=2, J_fr=2, Q_fr=2, T=32, F=3),
    "tiny_T_eq_N": dict(N=256, J=3, Q=2, Q2=1, J_fr=1, Q_fr=1, T=256, F=1),
    "tiny_short_rows": dict(N=256, J=5, Q=2, Q2=1, J_fr=2, Q_fr=1, T=32, F=4),
    "tones8k_n8192": dict(N=2 ** 13, J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4),
    "four_step_n32768": dict(N=2 ** 15, J=5, Q=2, Q2=1, J_fr=2, Q_fr=1, T=32, F=2),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _plan(params, batch):
    from paper_2602_11896_gb300 import JTFSPlan
    return JTFSPlan(**params, batch=batch)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _block_errors(phi_gpu, phi_ref, ref_plan):
    g = O.phi_blocks(torch.as_tensor(phi_gpu, dtype=torch.float64), ref_plan)
    r = O.phi_blocks(torch.as_tensor(phi_ref, dtype=torch.float64), ref_plan)
    return {k: _rel(g[k], r[k]) for k in r}


def _inputs(N, B, seed):
    return np.stack([signals.white_noise(N, seed + i) for i in range(B)])


@pytest.mark.parametrize("name", list(CASES))
def test_forward_parity(name):
    params = CASES[name]
    B = 3
    plan = _plan(params, B)
    ref = O.Plan(**params)
    x = _inputs(params["N"], B, 10)
    phi = plan.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    phi_ref = O.jtfs(torch.tensor(x, dtype=torch.float64), ref)["phi"].numpy()
    assert phi.shape == phi_ref.shape
    for b in range(B):
        errs = _block_errors(phi[b:b + 1], phi_ref[b:b + 1], ref)
        assert max(errs.values()) <= TOL, (b, errs)


@pytest.mark.parametrize("name", list(CASES))
def test_backward_parity(name):
    """Adjoint: dx = J^T dphi against autograd through the oracle."""
    params = CASES[name]
    B = 2
    plan = _plan(params, B)
    ref = O.Plan(**params)
    x = _inputs(params["N"], B, 20)
    dphi = np.random.default_rng(5).standard_normal((B, ref.phi_size)).astype(np.float32)
    dx = plan.backward(torch.tensor(x, device="cuda"), torch.tensor(dphi, device="cuda")).cpu().numpy()
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    (O.jtfs(xt, ref)["phi"] * torch.tensor(dphi, dtype=torch.float64)).sum().backward()
    for b in range(B):
        assert _rel(dx[b], xt.grad[b].numpy()) <= TOL


@pytest.mark.parametrize("name", ["tiny_n256", "tones8k_n8192", "four_step_n32768"])
def test_loss_grad_parity(name):
    params = CASES[name]
    B = 2
    plan = _plan(params, B)
    ref = O.Plan(**params)
    N = params["N"]
    y = _inputs(N, B, 30)
    tgt_sig = np.stack([signals.harmonic_tones(N, 8000.0, 40 + b) for b in range(B)])
    tgt = O.jtfs(torch.tensor(tgt_sig, dtype=torch.float64), ref)["phi"]
    loss, dy = plan.loss_grad(torch.tensor(y, device="cuda"), tgt.float().cuda())
    E, g = O.loss_and_grad(torch.tensor(y, dtype=torch.float64), tgt, ref)
    assert _rel(loss.cpu().numpy(), E.numpy()) <= TOL
    for b in range(B):
        assert _rel(dy[b].cpu().numpy(), g[b].numpy()) <= TOL


def test_autograd_function_uses_adjoint():
    from paper_2602_11896_gb300 import jtfs
    params = CASES["tiny_n512_q3"]
    plan = _plan(params, 2)
    x = torch.tensor(_inputs(params["N"], 2, 50), device="cuda", requires_grad=True)
    w = torch.randn(2, plan.phi_size, device="cuda")
    (jtfs(x, plan) * w).sum().backward()
    dx = plan.backward(x.detach(), w)
    assert torch.equal(x.grad, dx)


def test_metamer_step_is_adam_on_the_gradient():
    params = CASES["tiny_n256"]
    B = 2
    plan = _plan(params, B)
    ref = O.Plan(**params)
    y0 = torch.tensor(_inputs(params["N"], B, 60), device="cuda")
    tgt = plan.forward(torch.tensor(_inputs(params["N"], B, 70), device="cuda"))
    y = y0.clone()
    m = torch.zeros_like(y)
    v = torch.zeros_like(y)
    ym, mm, vm = y0.double().clone(), torch.zeros_like(y0).double(), torch.zeros_like(y0).double()
    for step in (1, 2, 3):
        _, g = plan.loss_grad(y, tgt)
        loss = plan.metamer_step(y, tgt, m, v, step, 0.1)
        g = g.double()
        mm = 0.9 * mm + 0.1 * g
        vm = 0.999 * vm + 0.001 * g * g
        ym = ym - 0.1 * (mm / (1 - 0.9 ** step)) / (torch.sqrt(vm / (1 - 0.999 ** step)) + 1e-8)
        assert torch.allclose(y.double(), ym, rtol=0, atol=1e-5)
        assert loss.shape == (B,)
        ym = y.double().clone()   # follow the device iterate (removes drift from rounding)


def test_zero_input_and_zero_gradient():
    """Phi(0) = 0; at 0 every modulus has derivative 0, so only S0 (linear) backpropagates."""
    params = CASES["tiny_n256"]
    plan = _plan(params, 1)
    ref = O.Plan(**params)
    x = torch.zeros(1, params["N"], device="cuda")
    assert plan.forward(x).abs().max().item() == 0.0
    dphi = np.random.default_rng(1).standard_normal((1, ref.phi_size)).astype(np.float32)
    dx = plan.backward(x, torch.tensor(dphi, device="cuda")).cpu().numpy()
    xt = torch.zeros(1, params["N"], dtype=torch.float64, requires_grad=True)
    (O.jtfs(xt, ref)["phi"] * torch.tensor(dphi, dtype=torch.float64)).sum().backward()
    assert _rel(dx, xt.grad.numpy()) <= TOL


def test_batch_clips_are_independent():
    params = CASES["tones8k_n8192"]
    plan4 = _plan(params, 4)
    plan1 = _plan(params, 1)
    x = torch.tensor(_inputs(params["N"], 4, 80), device="cuda")
    phi4 = plan4.forward(x)
    for b in range(4):
        assert torch.equal(plan1.forward(x[b:b + 1].contiguous())[0], phi4[b])


def test_deterministic():
    params = CASES["tones8k_n8192"]
    plan = _plan(params, 2)
    x = torch.tensor(_inputs(params["N"], 2, 90), device="cuda")
    tgt = plan.forward(torch.tensor(_inputs(params["N"], 2, 91), device="cuda"))
    l1, g1 = plan.loss_grad(x, tgt)
    l2, g2 = plan.loss_grad(x, tgt)
    assert torch.equal(l1, l2) and torch.equal(g1, g2)


def test_shift_by_T_at_chirps_workload_size():
    """Property at full size: shifting every clip by T shifts every Phi frame by one."""
    wl = get_workload("chirps22k_b8_n65536")
    plan = _plan(wl.params, wl.batch)
    ref = O.Plan(**wl.params)
    x = torch.tensor(wl.targets(), device="cuda")
    a = plan.forward(x).reshape(wl.batch, -1, ref.n_frames)
    b = plan.forward(torch.roll(x, wl.T, -1).contiguous()).reshape(wl.batch, -1, ref.n_frames)
    assert _rel(b.cpu().numpy(), torch.roll(a, 1, -1).cpu().numpy()) <= TOL


def test_chirps_workload_full_size_sampled_clip():
    """Batch-8, 2^16-sample workload in the bench's launch configuration: clip 5's
    Phi and gradient against the oracle (one clip is what the oracle computes in
    seconds); the other clips are covered by the batch-independence test."""
    wl = get_workload("chirps22k_b8_n65536")
    plan = _plan(wl.params, wl.batch)
    ref = O.Plan(**wl.params)
    y = torch.tensor(wl.inits(), device="cuda")
    xt = torch.tensor(wl.targets(), device="cuda")
    tgt = plan.forward(xt)
    b = 5
    tgt_ref = O.jtfs(torch.tensor(wl.targets()[b:b + 1], dtype=torch.float64), ref)["phi"]
    errs = _block_errors(tgt[b:b + 1].cpu().numpy(), tgt_ref.numpy(), ref)
    assert max(errs.values()) <= TOL, errs
    tgt[b] = tgt_ref[0].float().cuda()          # both sides use the oracle's target for clip b
    loss, dy = plan.loss_grad(y, tgt)
    E, g = O.loss_and_grad(torch.tensor(wl.inits()[b:b + 1], dtype=torch.float64), tgt_ref, ref,
                           checkpoint_blocks=True)
    assert _rel(loss[b:b + 1].cpu().numpy(), E.numpy()) <= TOL
    assert _rel(dy[b].cpu().numpy(), g[0].numpy()) <= TOL


def _path_errors(phi_gpu, phi_ref, meta, size):
    """Relative L2 error of every path of one clip's Phi (offsets from jtfs_path_meta)."""
    off = list(meta["offset"]) + [size]
    out = {}
    for p in range(len(meta["offset"])):
        key = (int(meta["order"][p]), int(meta["n2"][p]), int(meta["beta_idx"][p]))
        out[key] = _rel(phi_gpu[off[p]:off[p + 1]], phi_ref[off[p]:off[p + 1]])
    return out


@pytest.mark.parametrize("name,clip", [("tones8k_n8192", 0), ("chirps22k_b8_n65536", 5)])
def test_every_path_within_tolerance(name, clip):
    """Per path, not per block: S0, every first-order beta and every (n2, beta) path of one clip of the
    workload in the bench's launch configuration, through the tensor-core groups (default) and through
    the FFT kernels for every group, each against the oracle at <= 1e-4 relative L2."""
    wl = get_workload(name)
    plan = _plan(wl.params, wl.batch)
    ref = O.Plan(**wl.params)
    meta = plan.path_meta()
    assert len(meta["offset"]) == 1 + (1 + ref.K) + len(ref.active) * (1 + 2 * ref.K)
    sig = wl.targets()
    phi_ref = O.jtfs(torch.tensor(sig[clip:clip + 1], dtype=torch.float64), ref)["phi"][0].numpy()
    base = list(plan.tuning())
    for tc in (1, 0):
        plan.set_tuning(base[:3] + [tc])
        phi = plan.forward(torch.tensor(sig, device="cuda"))[clip].cpu().numpy()
        errs = _path_errors(phi, phi_ref, meta, plan.phi_size)
        worst = max(errs, key=errs.get)
        assert errs[worst] <= TOL, (tc, worst, errs[worst])


def test_forward_parity_64_frames_tensor_core_pooling():
    """A plan with 64 frames (tensor-core time pooling of its dense groups) against the oracle."""
    params = dict(N=2 ** 14, J=8, Q=8, Q2=1, J_fr=3, Q_fr=1, T=256, F=4)
    plan = _plan(params, 1)
    assert plan.tuning()[4] == 1
    x = _inputs(params["N"], 1, 71)
    phi = plan.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    ref_plan = O.Plan(**params)
    ref = O.jtfs(torch.tensor(x), ref_plan)["phi"].numpy()
    for k, e in _block_errors(phi, ref, ref_plan).items():
        assert e <= TOL, (k, e)


def test_gradient_parity_64_frames_tensor_core_pooling():
    """The same 64-frame plan: loss and gradient (tensor-core adjoint pooling) against the oracle."""
    params = dict(N=2 ** 14, J=8, Q=8, Q2=1, J_fr=3, Q_fr=1, T=256, F=4)
    plan = _plan(params, 1)
    assert plan.tuning()[4] == 1
    ref_plan = O.Plan(**params)
    y = _inputs(params["N"], 1, 81)
    tgt = O.jtfs(torch.tensor(_inputs(params["N"], 1, 91)), ref_plan)["phi"]
    loss, dy = plan.loss_grad(torch.tensor(y, device="cuda"), tgt.float().cuda())
    E, g = O.loss_and_grad(torch.tensor(y), tgt, ref_plan)
    assert _rel(loss.cpu().numpy(), E.numpy()) <= TOL
    assert _rel(dy.cpu().numpy(), g.numpy()) <= TOL
