"""jtfs_forward_noalloc: the forward transform for callers that cannot allocate.

Some callers cannot call cudaMalloc (for example a real-time audio callback
that must not block on the allocator, or a plug-in whose host owns all device
memory), so the library offers a forward entry point that uses a fixed
scratch array compiled into the library instead of a caller workspace.  This
checks it through the C ABI against jtfs_forward on two calls in a row (the
scratch keeps the first call's data, which must not leak into the second),
and that plans larger than the fixed scratch are refused.  This file is
collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

from workloads import signals

pytestmark = pytest.mark.gpu

TOL = 1e-4
PARAMS = dict(N=2 ** 13, J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_noalloc_matches_forward_on_two_calls():
    from paper_2602_11896_gb300 import JTFSPlan, _native
    lib = _native.load()
    plan = JTFSPlan(**PARAMS, batch=2)
    assert plan.workspace_bytes <= 32 << 20
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (3, 11):
        x = torch.tensor(np.stack([signals.white_noise(PARAMS["N"], seed + b) for b in range(2)]),
                         device="cuda")
        ref = plan.forward(x)
        out = torch.full_like(ref, float("nan"))
        rc = lib.jtfs_forward_noalloc(plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      stream)
        assert rc == 0, _native.error_string(rc)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= TOL


def _noalloc(lib, plan, x):
    from paper_2602_11896_gb300 import _native
    out = torch.full((plan.batch, plan.phi_size), float("nan"), device="cuda")
    rc = lib.jtfs_forward_noalloc(plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _native.error_string(rc)
    return out


def test_forward_noalloc_ignores_what_another_plan_left_in_the_scratch():
    """A call of another plan (other N, batch and filterbank, on NaN input) fills the shared scratch with
    garbage laid out differently; the next call must write every scratch byte it reads, so its Phi equals
    jtfs_forward's bit for bit -- and so must the other plan's afterwards."""
    from paper_2602_11896_gb300 import JTFSPlan, _native
    lib = _native.load()
    other = JTFSPlan(N=2 ** 12, J=5, Q=4, Q2=2, J_fr=2, Q_fr=1, T=32, F=2, batch=3)
    plan = JTFSPlan(**PARAMS, batch=2)
    assert other.workspace_bytes <= 32 << 20
    poison = torch.full((3, 2 ** 12), float("nan"), device="cuda")
    assert torch.isnan(_noalloc(lib, other, poison)).any()
    x = torch.tensor(np.stack([signals.white_noise(PARAMS["N"], 23 + b) for b in range(2)]), device="cuda")
    assert torch.equal(_noalloc(lib, plan, x), plan.forward(x))
    xo = torch.tensor(np.stack([signals.white_noise(2 ** 12, 29 + b) for b in range(3)]), device="cuda")
    assert torch.equal(_noalloc(lib, other, xo), other.forward(xo))


def test_forward_noalloc_refuses_plans_beyond_its_scratch():
    from paper_2602_11896_gb300 import JTFSPlan, _native
    lib = _native.load()
    big = JTFSPlan(**PARAMS, batch=16)
    assert big.workspace_bytes > 32 << 20
    x = torch.zeros(16, PARAMS["N"], device="cuda")
    out = torch.empty(16, big.phi_size, device="cuda")
    rc = lib.jtfs_forward_noalloc(big._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -7
    assert "32 MiB" in _native.error_string(rc)
