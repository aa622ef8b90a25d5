"""Tensor-core frequential scattering against the FFT kernels and the oracle.

The tensor-core path (BF16 hi/lo operands, FP32 accumulation) computes the
same second-order frequential maps (§3.4, Eq. (5), and the adjoint of §2.3)
as the FFT kernels; both must stay within the 1e-4 relative L2 bar per Phi
block of the FP64 oracle.  Here the two GPU paths are compared per block on
the same plan (tuning choice 3 switches between them), the kernels' bounded
waits must not have expired, and the default choice must be the tensor cores
for the shapes they handle.
"""

import numpy as np
import pytest
import torch

from workloads import get_workload, signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


@pytest.mark.parametrize("name", ["tones8k_n8192", "chirps22k_b8_n65536"])
def test_tensor_core_path_matches_fft_path(name):
    from paper_2602_11896_gb300 import JTFSPlan, _native
    lib = _native.load()
    wl = get_workload(name)
    B = 2
    plan = JTFSPlan(**wl.params, batch=B)
    base = list(plan.tuning())
    assert base[3] == 1, "tensor-core path should be the default for this shape"
    x = torch.tensor(np.stack([signals.white_noise(wl.N, 31 + b) for b in range(B)]), device="cuda")
    y = torch.tensor(np.stack([signals.white_noise(wl.N, 41 + b) for b in range(B)]), device="cuda")
    res = {}
    for tc in (0, 1):
        plan.set_tuning(base[:3] + [tc])
        assert plan.tuning()[3] == tc
        phi = plan.forward(x)
        loss, g = plan.loss_grad(y, phi.flip(0).contiguous())
        res[tc] = (phi, loss, g)
    torch.cuda.synchronize()
    assert lib.jtfs_tc_error() == 0
    plan.set_tuning(base)
    info = plan.info
    nf, R, K = info["n_frames"], info["R_out"], info["K"]
    pp = R * nf
    off2 = nf + (K + 1) * pp
    p0, p1 = res[0][0], res[1][0]
    assert torch.equal(p1[:, :off2], p0[:, :off2])          # S0 and first order do not use the tensor cores
    for a in range(info["n_active"]):
        for b in range(2 * K + 1):
            o = off2 + (a * (2 * K + 1) + b) * pp
            assert _rel(p1[:, o:o + pp], p0[:, o:o + pp]) <= 1e-4, (a, b)
    assert _rel(res[1][1], res[0][1]) <= 1e-4
    assert _rel(res[1][2], res[0][2]) <= 1e-4


def test_tensor_core_path_repeats_bit_for_bit():
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload("chirps22k_b8_n65536")
    plan = JTFSPlan(**wl.params, batch=1)
    y = torch.tensor(signals.white_noise(wl.N, 5)[None], device="cuda")
    tgt = plan.forward(torch.tensor(signals.white_noise(wl.N, 6)[None], device="cuda"))
    l0, g0 = plan.loss_grad(y, tgt)
    l1, g1 = plan.loss_grad(y, tgt)
    assert torch.equal(l0, l1) and torch.equal(g0, g1)


POOL_CASES = {
    "chirps22k_b8_n65536": None,                                             # 32 frames
    "frames64_n16384": dict(N=2 ** 14, J=8, Q=8, Q2=1, J_fr=3, Q_fr=1, T=256, F=4),    # 64 frames
}


@pytest.mark.parametrize("name", list(POOL_CASES))
def test_tensor_core_pooling_matches_fma_pooling(name):
    """Time pooling of the dense groups on the tensor cores (BF16 hi/lo split) against the FMA kernels:
    every second-order block within 2e-5, the rest bit-identical, loss and gradient within 2e-5, no
    expired wait, and the tensor-core result repeatable bit for bit."""
    from paper_2602_11896_gb300 import JTFSPlan, _native
    lib = _native.load()
    params = POOL_CASES[name] or get_workload(name).params
    B = 2
    plan = JTFSPlan(**params, batch=B)
    base = list(plan.tuning())
    assert base[4] == 1, "tensor-core pooling should be the default for this frame count"
    N = params["N"]
    x = torch.tensor(np.stack([signals.white_noise(N, 51 + b) for b in range(B)]), device="cuda")
    y = torch.tensor(np.stack([signals.white_noise(N, 61 + b) for b in range(B)]), device="cuda")
    res = {}
    for v in (0, 1):
        plan.set_tuning(base[:4] + [v])
        assert plan.tuning()[4] == v
        phi = plan.forward(x).clone()
        loss, g = plan.loss_grad(y, phi.flip(0).contiguous())
        res[v] = (phi, loss.clone(), g.clone())
    again = plan.forward(x)
    torch.cuda.synchronize()
    assert lib.jtfs_tc_error() == 0
    assert torch.equal(again, res[1][0])
    plan.set_tuning(base)
    info = plan.info
    nf, R, K = info["n_frames"], info["R_out"], info["K"]
    pp = R * nf
    off2 = nf + (K + 1) * pp
    p0, p1 = res[0][0], res[1][0]
    assert torch.equal(p1[:, :off2], p0[:, :off2])
    worst = 0.0
    for a in range(info["n_active"]):
        for b in range(2 * K + 1):
            o = off2 + (a * (2 * K + 1) + b) * pp
            d = (p1[:, o:o + pp].double() - p0[:, o:o + pp].double()).norm() / p0[:, o:o + pp].double().norm()
            worst = max(worst, float(d))
    assert worst <= 2e-5, worst
    assert _rel(res[1][1], res[0][1]) <= 2e-5
    assert _rel(res[1][2], res[0][2]) <= 2e-5
