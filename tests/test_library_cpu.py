"""C-ABI library on the host: it loads, exports every declared symbol, and its
host-only plans agree with the oracle's filterbanks and schedule.

No compute call touches a GPU here; compute entry points are only checked
for their argument and host-only error paths.
"""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import jtfs_oracle as O
from paper_2602_11896_gb300 import JTFSPlan, _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "jtfs.h")

PARAMS = [
    dict(N=256, J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2),
    dict(N=512, J=5, Q=3, Q2=2, J_fr=2, Q_fr=2, T=32, F=3),
    dict(N=2 ** 13, J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4),
    dict(N=2 ** 16, J=12, Q=12, Q2=1, J_fr=5, Q_fr=2, T=2 ** 11, F=12),
    dict(N=2 ** 20, J=14, Q=16, Q2=2, J_fr=6, Q_fr=2, T=2 ** 13, F=16),
]


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                                 src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = _native.load()
    names = declared_functions()
    assert "jtfs_forward" in names and "metamer_step" in names and len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_native.SIGNATURES)


@pytest.mark.parametrize("params", PARAMS)
def test_host_plan_matches_oracle(params):
    plan = JTFSPlan(**params, batch=2, host_only=True)
    ref = O.Plan(**params)
    info = plan.info
    assert info["N1"] == ref.N1 and info["N2"] == len(ref.psi2) and info["K"] == ref.K
    assert info["N_fr"] == ref.N_fr and info["R_out"] == ref.R_out
    assert info["n_frames"] == ref.n_frames and info["log2_T"] == ref.lT and info["log2_F"] == ref.lF
    assert info["n_active"] == len(ref.active)
    assert plan.phi_size == ref.phi_size == info["phi_size"]
    for which, fb in ((0, ref.psi1), (1, ref.psi2), (2, ref.psi_fr)):
        xi, sg, j = plan.filters(which)
        assert len(xi) == len(fb)
        assert np.abs(xi - [f.xi for f in fb]).max() <= 1e-15
        assert np.abs(sg - [f.sigma for f in fb]).max() <= 1e-15
        assert (j == [f.j for f in fb]).all()
    xi, sg, j = plan.filters(3)
    assert xi.tolist() == [0.0, 0.0]
    assert abs(sg[0] - ref.sigma_phiT) < 1e-18 and abs(sg[1] - ref.sigma_phiF) < 1e-18
    assert j[1] == ref.j_phiF
    assert plan.workspace_bytes > 0


def test_plan_rejects_bad_shapes():
    lib = _native.load()
    h = ctypes.c_void_p()
    bad = [
        (300, 4, 4, 1, 2, 1, 16, 2),       # N not a power of two
        (256, 4, 4, 1, 2, 1, 24, 2),       # T not a power of two
        (256, 4, 4, 1, 2, 1, 512, 2),      # T > N
        (256, 4, 4, 1, 2, 1, 16, 0),       # F < 1
        (2 ** 21, 4, 4, 1, 2, 1, 16, 2),   # N too large
    ]
    for args in bad:
        rc = lib.jtfs_plan(ctypes.byref(h), *args, 1, _native.PLAN_HOST_ONLY)
        assert rc == -2, args
    assert lib.jtfs_plan(None, 256, 4, 4, 1, 2, 1, 16, 2, 1, 1) == -1
    assert lib.jtfs_phi_size(None) == -1
    assert lib.jtfs_workspace_bytes(None) == 0
    assert _native.error_string(-6).startswith("plan has no device")


def test_host_only_plan_refuses_compute():
    plan = JTFSPlan(**PARAMS[0], host_only=True)
    lib = _native.load()
    fake = ctypes.c_void_p(4096)  # never dereferenced: the call fails before any launch
    assert lib.jtfs_forward(plan._h, fake, fake, fake, None) == -6
    assert lib.jtfs_backward(plan._h, fake, fake, fake, fake, None) == -6
    assert lib.jtfs_loss_grad(plan._h, fake, fake, fake, fake, fake, None) == -6
    assert lib.metamer_step(plan._h, fake, fake, fake, fake, 1, 0.1, fake, fake, None) == -6
    assert lib.metamer_step(plan._h, fake, fake, fake, fake, 0, 0.1, fake, fake, None) == -1
    assert lib.jtfs_forward(plan._h, None, fake, fake, None) == -1
    assert lib.jtfs_forward(plan._h, ctypes.c_void_p(4100), fake, fake, None) == -1  # misaligned


def test_python_api_refuses_cpu_tensors():
    import torch
    plan = JTFSPlan(**PARAMS[0], host_only=True)
    with pytest.raises(TypeError):
        plan.forward(torch.zeros(1, 256))


def test_reflect_batch_layout_matches_oracle():
    """Host-only reflect batch: per-clip Phi sizes equal the oracle's cropped reflect layout (R20)."""
    import torch
    from oracle import jtfs_oracle as O
    from paper_2602_11896_gb300 import JTFSBatch
    params = dict(J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2)
    lengths = [1, 37, 200, 256, 4000]
    b = JTFSBatch(lengths, **params, host_only=True, boundary="reflect")
    for i, L in enumerate(lengths):
        want = O.jtfs_reflect(torch.zeros(L, dtype=torch.float64), params).numel()
        assert b.phi_offsets[i + 1] - b.phi_offsets[i] == want
    with pytest.raises(RuntimeError):
        JTFSBatch([2 ** 20], **params, host_only=True, boundary="reflect")


def test_batch_refuses_unpooled_flags():
    """Ragged batches crop Phi as rows x frames, so the unpooled layouts are refused."""
    lib = _native.load()
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 2)(300, 500)
    for flag in (_native.PLAN_UNPOOLED_T, _native.PLAN_UNPOOLED_F):
        rc = lib.jtfs_batch_create(ctypes.byref(h), arr, 2, 4, 4, 1, 2, 1, 16, 2, _native.PLAN_HOST_ONLY | flag)
        assert rc == -1 and not h.value


@pytest.mark.parametrize("variant", [(True, True), (False, True), (True, False), (False, False)])
@pytest.mark.parametrize("name", ["tones8k_n8192", "chirps22k_b8_n65536"])
def test_path_meta_matches_oracle_layout(name, variant):
    """Per-path metadata (host-only plans) against the oracle's Phi layout and frequential filter sets."""
    from paper_2602_11896_gb300 import JTFSPlan
    from workloads import get_workload
    wl = get_workload(name)
    kw = dict(average_local=variant[0], average_local_fr=variant[1])
    plan = JTFSPlan(**wl.params, host_only=True, **kw)
    op = O.Plan(**wl.params, **kw)
    m = plan.path_meta()
    K1, K2 = len(op.beta_first), len(op.beta_second)
    n = 1 + K1 + len(op.active) * K2
    assert all(len(v) == n for v in m.values())
    assert m["order"].tolist() == [0] + [1] * K1 + [2] * (len(op.active) * K2)
    assert m["n2"].tolist() == [-1] * (1 + K1) + [n2 for n2 in op.active for _ in range(K2)]
    assert m["beta_idx"].tolist() == [-1] + list(range(K1)) + list(range(K2)) * len(op.active)
    signs = [int(np.sign(b[0])) for b in op.beta_second]
    assert m["spin"].tolist() == [0] + signs[:K1] + signs * len(op.active)
    # offsets: increasing, path sizes = rows x frames of the oracle's layout, blocks where phi_blocks puts them
    sizes = [op.N if not op.average_local else op.n_frames]
    sizes += [op.rows(b) * op.n_frames for b in op.beta_first]
    sizes += [op.rows(b) * op.frames2(n2) for n2 in op.active for b in op.beta_second]
    ends = np.cumsum(sizes)
    assert m["offset"].tolist() == [0] + ends[:-1].tolist()
    assert ends[-1] == op.phi_size == plan.phi_size


def test_plan_ragged_is_the_ragged_batch():
    lib = _native.load()
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 3)(300, 512, 100)
    assert lib.jtfs_plan_ragged(ctypes.byref(h), arr, 3, 4, 4, 1, 2, 1, 16, 2, _native.PLAN_HOST_ONLY) == 0
    so = (ctypes.c_int64 * 4)()
    po = (ctypes.c_int64 * 4)()
    assert lib.jtfs_batch_layout(h, so, po) == 3
    assert list(so) == [0, 300, 812, 912]
    lib.jtfs_batch_destroy(h)
