"""Device-side error path of the C ABI (jtfs_status) and the graph-capturable
plain metamer step (metamer_step_counted).

* A NaN in y makes §2.3's loss non-finite: the loss reduction raises
  JTFS_ERR_NONFINITE in the status word, jtfs_status returns and clears it.
* A bounded barrier wait of the tensor-core kernels that runs out makes the
  kernel give up (copies and MMAs drained, TMEM freed) and raise
  JTFS_ERR_TIMEOUT.  The test shortens the waits to zero polls
  (jtfs_set_wait_limit), so every such wait gives up at once -- nothing is
  broken, no barrier is left unsatisfied on purpose -- then restores the bound
  and checks that the next call is clean and exact.
* metamer_step_counted reads Adam's step index from device memory, so one
  captured call replays as successive steps: replay equals eager bit for bit,
  and both follow metamer_step with host step indices.
"""

import ctypes

import numpy as np
import pytest
import torch

from workloads import get_workload, signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _plan(batch=2):
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload("tones8k_n8192")
    return JTFSPlan(**wl.params, batch=batch), wl


def _status():
    from paper_2602_11896_gb300 import _native
    return _native.status(torch.cuda.current_stream().cuda_stream)


def _inputs(plan, wl, seed=3):
    B = plan.batch
    x = torch.tensor(np.stack([signals.harmonic_tones(wl.N, 8000.0, seed + b) for b in range(B)]), device="cuda")
    y = torch.tensor(np.stack([signals.white_noise(wl.N, seed + 10 + b) for b in range(B)]), device="cuda")
    return plan.forward(x), y


def test_status_is_clean_after_a_normal_call():
    plan, wl = _plan()
    _status()                      # clear what earlier tests left
    tgt, y = _inputs(plan, wl)
    plan.loss_grad(y, tgt)
    assert _status() == 0
    plan.check_status("clean call")


def test_nan_in_y_reports_nonfinite_then_clears():
    from paper_2602_11896_gb300 import _native
    plan, wl = _plan()
    _status()
    tgt, y = _inputs(plan, wl)
    y_host = y.cpu()
    y_host[1, 777] = float("nan")  # one sample of the second clip, placed on the host
    loss, _ = plan.loss_grad(y_host.cuda(), tgt)
    assert _status() == _native.ERR_NONFINITE
    assert torch.isfinite(loss[0]) and not torch.isfinite(loss[1])
    assert _status() == 0          # read-and-clear
    plan.loss_grad(y, tgt)
    with pytest.raises(_native.DeviceStatusError):
        plan.loss_grad(y_host.cuda(), tgt)
        plan.check_status("nan input")
    plan.check_status("after the error was reported")


def test_nan_target_in_ragged_batch_reports_nonfinite():
    from paper_2602_11896_gb300 import JTFSBatch, _native
    _status()
    lengths = [300, 1000]
    b = JTFSBatch(lengths, J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2)
    x = torch.tensor(np.concatenate([signals.white_noise(L, 50 + i) for i, L in enumerate(lengths)]),
                     device="cuda")
    tgt = b.forward(x)
    tgt[5] = float("inf")
    y = torch.tensor(np.concatenate([signals.white_noise(L, 60 + i) for i, L in enumerate(lengths)]),
                     device="cuda")
    m, v = torch.zeros_like(y), torch.zeros_like(y)
    step = torch.ones(1, dtype=torch.int32, device="cuda")
    b.metamer_step(y, tgt, m, v, step, 0.1)
    assert _status() == _native.ERR_NONFINITE
    assert _status() == 0


def test_expired_tensor_core_wait_reports_timeout_and_next_call_is_exact():
    from paper_2602_11896_gb300 import _native
    lib = _native.load()
    plan, wl = _plan()
    assert plan.tuning()[3] == 1, "the tone plan runs its frequential step on the tensor cores"
    tgt, y = _inputs(plan, wl)
    loss_ref, g_ref = plan.loss_grad(y, tgt)
    loss_ref, g_ref = loss_ref.clone(), g_ref.clone()
    assert _status() == 0
    try:
        _native.check(lib.jtfs_set_wait_limit(0), "jtfs_set_wait_limit")
        plan.loss_grad(y, tgt)
        code = _status()
    finally:
        _native.check(lib.jtfs_set_wait_limit(-1), "jtfs_set_wait_limit")
    assert code == _native.ERR_TIMEOUT
    assert lib.jtfs_tc_error() == 0          # jtfs_status cleared the flag it reported
    info = (ctypes.c_int64 * 4)()
    lib.jtfs_tc_error_info(info, 4)          # clear the diagnostic record
    loss, g = plan.loss_grad(y, tgt)
    assert _status() == 0
    assert torch.equal(loss, loss_ref) and torch.equal(g, g_ref)


def test_counted_step_replays_from_a_graph_like_eager_steps():
    plan, wl = _plan()
    tgt, y0 = _inputs(plan, wl, seed=21)
    K = 5

    def fresh():
        return y0.clone(), torch.zeros_like(y0), torch.zeros_like(y0)

    # Eager, step index on the device.
    y_e, m_e, v_e = fresh()
    step = torch.ones(1, dtype=torch.int32, device="cuda")
    loss_e = torch.empty(K, plan.batch, device="cuda")
    for k in range(K):
        plan.metamer_step_counted(y_e, tgt, m_e, v_e, step, 0.1, loss_out=loss_e[k])
    assert int(step.item()) == K + 1

    # One captured call replayed K times.
    y_g, m_g, v_g = fresh()
    step_g = torch.ones(1, dtype=torch.int32, device="cuda")
    loss_g = torch.empty(plan.batch, device="cuda")
    ws = plan.workspace(y_g.device)
    plan.metamer_step_counted(y_g.clone(), tgt, m_g.clone(), v_g.clone(), step_g.clone(), 0.1, workspace=ws)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.metamer_step_counted(y_g, tgt, m_g, v_g, step_g, 0.1, loss_out=loss_g, workspace=ws)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    losses_g = []
    for _ in range(K):
        g.replay()
        losses_g.append(loss_g.clone())
    torch.cuda.synchronize()
    assert int(step_g.item()) == K + 1
    assert torch.equal(y_g, y_e) and torch.equal(m_g, m_e) and torch.equal(v_g, v_e)
    assert torch.equal(torch.stack(losses_g), loss_e)

    # Host step indices (metamer_step): the same Adam with the same double-precision bias corrections.
    y_h, m_h, v_h = fresh()
    for k in range(K):
        plan.metamer_step(y_h, tgt, m_h, v_h, k + 1, 0.1)
    rel = float((y_h - y_e).norm() / y_h.norm())
    assert rel <= 1e-7, rel
    plan.check_status("counted steps")
