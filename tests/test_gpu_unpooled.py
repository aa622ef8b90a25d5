"""Unpooled outputs (average_local / average_local_fr off, oracle reading R21) through the C ABI.

Relative L2 <= 1e-4 per Phi block and for gradients, as the pooled transform.
"""

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from workloads import signals

pytestmark = pytest.mark.gpu

TOL = 1e-4

CASES = {
    "tiny_n256": dict(N=256, J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2),
    "tiny_n512_q3": dict(N=512, J=5, Q=3, Q2=2, J_fr=2, Q_fr=2, T=32, F=3),    # phi_F stride 2 > log2 F
    "tones8k_n8192": dict(N=2 ** 13, J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4),
}
MODES = {"time": (False, True), "freq": (True, False), "both": (False, False)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _inputs(N, B, seed):
    return np.stack([signals.white_noise(N, seed + i) for i in range(B)])


def _plans(params, mode, batch):
    from paper_2602_11896_gb300 import JTFSPlan
    kw = dict(average_local=mode[0], average_local_fr=mode[1])
    return JTFSPlan(**params, batch=batch, **kw), O.Plan(**params, **kw)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("name", list(CASES))
def test_unpooled_forward_parity(name, mode):
    plan, op = _plans(CASES[name], MODES[mode], 2)
    x = _inputs(op.N, 2, 11)
    phi = plan.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    ref = O.jtfs(torch.tensor(x), op)["phi"].numpy()
    assert phi.shape == ref.shape
    g = O.phi_blocks(torch.tensor(phi, dtype=torch.float64), op)
    r = O.phi_blocks(torch.tensor(ref), op)
    for k in r:
        assert _rel(g[k], r[k]) <= TOL, k
    if not op.average_local:
        assert np.array_equal(phi[:, :op.N], x)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("name", list(CASES))
def test_unpooled_gradient_parity(name, mode):
    plan, op = _plans(CASES[name], MODES[mode], 1)
    y = _inputs(op.N, 1, 21)
    tgt = O.jtfs(torch.tensor(_inputs(op.N, 1, 31)), op)["phi"]
    loss, dy = plan.loss_grad(torch.tensor(y, device="cuda"), tgt.float().cuda())
    E, g = O.loss_and_grad(torch.tensor(y), tgt, op)
    assert _rel(loss.cpu().numpy(), E.numpy()) <= TOL
    assert _rel(dy.cpu().numpy(), g.numpy()) <= TOL


def test_time_unpooled_refuses_rows_beyond_the_time_stride():
    from paper_2602_11896_gb300 import JTFSPlan
    with pytest.raises(RuntimeError):
        JTFSPlan(N=256, J=5, Q=2, Q2=1, J_fr=2, Q_fr=1, T=8, F=4, average_local=False)


def test_freq_unpooled_chirp_batch_sampled():
    """The chirp plan (8 x 2^16) unpooled along n1: one sampled clip's first-order block and two
    second-order blocks against the oracle (the generic frequential kernels at full size)."""
    from workloads import get_workload
    wl = get_workload("chirps22k_b8_n65536")
    plan, op = _plans(wl.params, (True, False), 2)
    x = _inputs(op.N, 2, 51)
    phi = plan.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    sel = [0, len(op.active) - 1]
    ref = O.jtfs(torch.tensor(x[1:2]), op, active=sel)
    g = O.phi_blocks(torch.tensor(phi[1:2], dtype=torch.float64), op)
    assert _rel(g["S0"], ref["S0"]) <= TOL
    assert _rel(g["first"], ref["Phi1"].reshape(1, -1)) <= TOL
    for a in sel:
        assert _rel(g[f"n2={op.active[a]}"], ref["Phi2_sel"][a].reshape(1, -1)) <= TOL, a
