"""Long signals: 4 clips of 2^20 samples (J=14, Q=16, Q2=2, J_fr=6, Q_fr=2, T=2^13, F=16).

The oracle cannot evaluate the whole transform at 2^20 in test time, so:
* the same filterbanks at reduced N (2^15 forward, 2^14 gradient) against the oracle, every Phi block;
* at full size, in the launch configuration of the long-signal benchmark: S0, every first-order row and
  two sampled second-order paths of one clip against the oracle, every path of the finest second-order
  level at two frames (the oracle evaluated at those frames only), the adjoint on S0, the first order and
  three second-order groups (coarsest, middle, level 11), and the shift-by-T property.
"""

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from workloads import get_workload, signals

pytestmark = pytest.mark.gpu

TOL = 1e-4
WL = get_workload("notes22k_b4_n1048576")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _params(N):
    p = dict(WL.params)
    p["N"] = N
    return p


def _blocks(phi_row, ref_plan, ref):
    """Split one clip's Phi like the oracle's S0 / Phi1 / Phi2 (per active path)."""
    nf = ref_plan.N // ref_plan.T
    n1 = ref["Phi1"][0].numel()
    out = {"S0": phi_row[:nf], "Phi1": phi_row[nf:nf + n1]}
    n2 = (phi_row.size - nf - n1) // max(len(ref_plan.active), 1)
    for a in range(len(ref_plan.active)):
        out[a] = phi_row[nf + n1 + a * n2:nf + n1 + (a + 1) * n2]
    return out


def test_reduced_n_forward_parity():
    from paper_2602_11896_gb300 import JTFSPlan
    params = _params(2 ** 15)
    x = signals.polyphonic_notes(2 ** 15, WL.sr, 400)
    plan = JTFSPlan(**params, batch=1)
    phi = plan.forward(torch.tensor(x[None], device="cuda")).cpu().numpy()[0]
    ref_plan = O.Plan(**params)
    ref = O.jtfs(torch.tensor(x[None], dtype=torch.float64), ref_plan, keep=True)
    got = _blocks(phi, ref_plan, ref)
    assert _rel(got["S0"], ref["S0"][0]) <= TOL
    assert _rel(got["Phi1"], ref["Phi1"][0]) <= TOL
    for a in range(len(ref_plan.active)):
        assert _rel(got[a], ref["Phi2"][0, a]) <= TOL, a


def test_reduced_n_gradient_parity():
    from paper_2602_11896_gb300 import JTFSPlan
    params = _params(2 ** 14)
    x = signals.polyphonic_notes(2 ** 14, WL.sr, 401)
    y = signals.white_noise(2 ** 14, 501)
    ref_plan = O.Plan(**params)
    tgt = O.jtfs(torch.tensor(x[None], dtype=torch.float64), ref_plan)["phi"]
    E, g = O.loss_and_grad(torch.tensor(y[None], dtype=torch.float64), tgt, ref_plan)
    plan = JTFSPlan(**params, batch=1)
    loss, grad = plan.loss_grad(torch.tensor(y[None], device="cuda"), tgt.float().cuda())
    assert _rel([loss.item()], [float(E)]) <= TOL
    assert _rel(grad.cpu().numpy(), g.numpy()) <= TOL


@pytest.fixture(scope="module")
def full():
    from paper_2602_11896_gb300 import JTFSPlan
    torch.cuda.reset_peak_memory_stats()
    plan = JTFSPlan(**WL.params, batch=WL.batch)
    x = WL.targets()
    phi = plan.forward(torch.tensor(x, device="cuda"))
    loss, grad = plan.loss_grad(torch.tensor(WL.inits(), device="cuda"), phi)
    torch.cuda.synchronize()
    peak = torch.cuda.max_memory_allocated()
    return plan, x, phi, loss, grad, peak


def test_full_size_sampled_paths_against_oracle(full):
    plan, x, phi, loss, grad, peak = full
    print(f"peak device memory, forward + loss/gradient of 4 x 2^20: {peak / 2**30:.2f} GiB")
    assert peak < 64 * 2 ** 30
    assert torch.isfinite(loss).all() and torch.isfinite(grad).all()
    ref_plan = O.Plan(**WL.params)
    s2 = [min(ref_plan.psi2[n2].j, ref_plan.lT) for n2 in ref_plan.active]
    order = np.argsort(s2, kind="stable")
    sample = [int(order[-1]), int(order[len(order) // 2])]   # coarsest level and a middle one
    ref = O.jtfs(torch.tensor(x[:1], dtype=torch.float64), ref_plan, active=sample)
    got = _blocks(phi[0].cpu().numpy(), ref_plan, ref)
    assert _rel(got["S0"], ref["S0"][0]) <= TOL
    assert _rel(got["Phi1"], ref["Phi1"][0]) <= TOL
    for a in sample:
        assert _rel(got[a], ref["Phi2_sel"][a][0]) <= TOL, a


def test_full_size_finest_level_against_oracle(full):
    """The finest second-order level of the 4 x 2^20 plan (the most time columns, the largest FFTs of
    Y2) at full size: every path of clip 0 at frames 0 (its phi_T window wraps around the circle) and 77,
    against the oracle evaluated at those frames only."""
    plan, x, phi, _, _, _ = full
    ref_plan = O.Plan(**WL.params)
    s2 = [min(ref_plan.psi2[n2].j, ref_plan.lT) for n2 in ref_plan.active]
    a = int(np.argmin(s2))
    frames = [0, 77]
    ref = O.second_order_frames(torch.tensor(x[:1], dtype=torch.float64), ref_plan, a, frames)[0].numpy()
    off = ref_plan.n_frames * (1 + (1 + ref_plan.K) * ref_plan.R_out)
    paths = 1 + 2 * ref_plan.K
    off += a * paths * ref_plan.R_out * ref_plan.n_frames
    blk = phi[0, off:off + paths * ref_plan.R_out * ref_plan.n_frames].cpu().numpy()
    got = blk.reshape(paths, ref_plan.R_out, ref_plan.n_frames)[..., frames]
    for b in range(paths):
        assert _rel(got[b], ref[b]) <= TOL, (a, b)


def test_full_size_gradient_on_sampled_paths(full):
    """The adjoint at full size (4 x 2^20, the long benchmark's plan): J^T w for weights w on S0, every
    first-order path and three second-order groups of clip 0 (zero elsewhere), against the oracle's
    autograd of the same linear functional of those outputs (FP64; the rest of the transform is not
    evaluated).  Exercises the full-size first-layer adjoint (2^20-point transforms, k_dU1, k_dX) and the
    second-order adjoint chain of a coarsest group (banded phi_T adjoint on the FMA kernel), a middle one
    and one of the level-11 groups (banded phi_T adjoint on the tensor cores: 1024 and 128 samples per
    CTA, D = 64 and 4)."""
    plan, x, phi, _, _, _ = full
    ref_plan = O.Plan(**WL.params)
    s2 = [min(ref_plan.psi2[n2].j, ref_plan.lT) for n2 in ref_plan.active]
    order = np.argsort(s2, kind="stable")
    sample = [int(order[-1]), int(order[len(order) // 2]), int(order[-5])]
    y = WL.inits()
    yt = torch.tensor(y[:1], dtype=torch.float64, requires_grad=True)
    out = O.jtfs(yt, ref_plan, active=sample)
    nf = out["S0"][0].numel()
    n_first = out["Phi1"][0].numel()
    n2 = (plan.phi_size - nf - n_first) // len(ref_plan.active)
    rng = np.random.default_rng(77)
    w_s0 = rng.standard_normal(nf)
    w_1 = rng.standard_normal(n_first)
    dphi = np.zeros((WL.batch, plan.phi_size), dtype=np.float32)
    dphi[0, :nf] = w_s0
    dphi[0, nf:nf + n_first] = w_1
    f = ((out["S0"][0].reshape(-1) * torch.tensor(w_s0)).sum()
         + (out["Phi1"][0].reshape(-1) * torch.tensor(w_1)).sum())
    for a in sample:
        blk = out["Phi2_sel"][a][0].numel()
        assert n2 == blk
        w_2 = rng.standard_normal(blk)
        off2 = nf + n_first + a * n2
        dphi[0, off2:off2 + blk] = w_2
        f = f + (out["Phi2_sel"][a][0].reshape(-1) * torch.tensor(w_2)).sum()
    dx = plan.backward(torch.tensor(y, device="cuda"), torch.tensor(dphi, device="cuda"))[0].cpu().numpy()
    f.backward()
    assert _rel(dx, yt.grad[0].numpy()) <= TOL


def test_full_size_shift_by_T_shifts_frames(full):
    plan, x, phi, _, _, _ = full
    T = WL.T
    xs = np.roll(x, T, axis=1)
    phis = plan.forward(torch.tensor(xs, device="cuda"))
    nf = WL.N // T
    a = phi.cpu().numpy().reshape(WL.batch, -1, nf)
    b = phis.cpu().numpy().reshape(WL.batch, -1, nf)
    assert _rel(b, np.roll(a, 1, axis=2)) <= 1e-5
