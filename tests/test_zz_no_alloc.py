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
