"""Parity of the reconstruction variant of §2.3 with the FP64 oracle, through the C ABI.

Coloured initialisation (relative L2 <= 1e-4 per clip, the transform's FP32
bound), the bold-driver momentum update on given inputs (element-wise, same
accept decisions: both sides compare the same float32 losses), and whole
descents whose accept / reject decisions have wide margins.
"""

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from oracle import reconstruct as R
from workloads import get_workload, signals

pytestmark = pytest.mark.gpu

TOL = 1e-4

TINY = dict(N=512, J=5, Q=3, Q2=2, J_fr=2, Q_fr=2, T=32, F=3)


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


def _noise(N, B, seed):
    return np.stack([signals.white_noise(N, seed + i) for i in range(B)])


@pytest.mark.parametrize("name,batch", [("tones8k_n8192", 1), ("chirps22k_b8_n65536", 8)])
def test_coloured_init_parity(name, batch):
    wl = get_workload(name)
    x = wl.targets()[:batch]
    w = _noise(wl.N, batch, 777)
    plan = _plan(wl.params, batch)
    y0 = plan.coloured_init(torch.tensor(x, device="cuda"), torch.tensor(w, device="cuda")).cpu().numpy()
    ref = R.coloured_init(torch.tensor(x, dtype=torch.float64), torch.tensor(w, dtype=torch.float64),
                          O.Plan(**wl.params)).numpy()
    for b in range(batch):
        assert _rel(y0[b], ref[b]) <= TOL, b
        assert abs(np.linalg.norm(y0[b]) / np.linalg.norm(x[b]) - 1.0) <= 1e-5


def test_coloured_init_tiny_batch_with_zero_clip():
    """Three clips of 512 samples, the middle one silent: its init is exactly zero, the others match."""
    x = _noise(512, 3, 40)
    x[1] = 0.0
    w = _noise(512, 3, 50)
    plan = _plan(TINY, 3)
    y0 = plan.coloured_init(torch.tensor(x, device="cuda"), torch.tensor(w, device="cuda")).cpu().numpy()
    ref = R.coloured_init(torch.tensor(x, dtype=torch.float64), torch.tensor(w, dtype=torch.float64),
                          O.Plan(**TINY)).numpy()
    assert not y0[1].any()
    for b in (0, 2):
        assert _rel(y0[b], ref[b]) <= TOL


def test_momentum_update_parity():
    """Given loss and gradient: first evaluation, decrease, increase, NaN and a tie, one clip each."""
    from paper_2602_11896_gb300 import momentum_update
    rng = np.random.default_rng(3)
    B, n = 5, 1024
    y, u, ga, g = (rng.standard_normal((B, n)).astype(np.float32) for _ in range(4))
    mu = np.array([0.1, 0.3, 0.2, 0.5, 0.7], dtype=np.float32)
    E_acc = np.array([np.inf, 1.0, 1.0, 1.0, 2.0], dtype=np.float32)
    E = np.array([3.0, 0.5, 1.5, np.nan, 2.0], dtype=np.float32)
    st = np.stack([mu, E_acc, np.zeros(B, np.float32), np.full(B, 7.0, np.float32)], 1)
    t = {k: torch.tensor(v, device="cuda") for k, v in dict(y=y, u=u, g_acc=ga, state=st, g=g, E=E).items()}
    opt = {"u": t["u"], "g_acc": t["g_acc"], "state": t["state"]}
    momentum_update(t["y"], opt, t["g"], t["E"], m=0.9)
    ref = R.bold_driver_step(y, u, ga, mu, E_acc, E, g, m=0.9)
    assert ref["accepted"].tolist() == [True, True, False, False, True]
    out_st = opt["state"].cpu().numpy()
    assert out_st[:, 2].tolist() == [1.0, 1.0, 0.0, 0.0, 1.0]
    assert out_st[:, 3].tolist() == [8.0] * B
    np.testing.assert_allclose(out_st[:, 0], ref["mu"], rtol=1e-6)
    np.testing.assert_array_equal(out_st[:, 1], ref["E_acc"].astype(np.float32))
    for key in ("y", "u", "g_acc"):
        got = (t["y"] if key == "y" else opt[key]).cpu().numpy()
        np.testing.assert_allclose(got, ref[key], rtol=1e-5, atol=1e-5)


def test_metamer_step_momentum_matches_oracle():
    """Six evaluations from white noise with mu0 = 300: accepts and rejects, each decision by a wide margin."""
    wl = get_workload("tones8k_n8192")
    op = O.Plan(**wl.params)
    tgt = O.jtfs(torch.tensor(wl.targets(), dtype=torch.float64), op)["phi"]
    y_ref = wl.inits().astype(np.float64)
    plan = _plan(wl.params, 1)
    y = torch.tensor(wl.inits(), device="cuda")
    tgt_gpu = tgt.to(torch.float32).cuda()
    opt = plan.momentum_state(mu0=300.0)
    u = np.zeros_like(y_ref)
    ga = np.zeros_like(y_ref)
    mu = np.array([300.0])
    E_acc = np.array([np.inf])
    decisions = []
    for i in range(6):
        E_ref, g_ref = O.loss_and_grad(torch.tensor(y_ref), tgt, op)
        out = R.bold_driver_step(y_ref, u, ga, mu, E_acc, E_ref.numpy(), g_ref.numpy())
        if np.isfinite(E_acc[0]):
            assert abs(float(E_ref[0]) / E_acc[0] - 1.0) > 0.05     # the decision is not a near tie
        loss = plan.metamer_step_momentum(y, tgt_gpu, opt, m=0.9)
        torch.cuda.synchronize()
        assert abs(float(loss[0]) / float(E_ref[0]) - 1.0) <= TOL, i
        assert bool(opt["state"][0, 2].item()) == bool(out["accepted"][0]), i
        decisions.append(bool(out["accepted"][0]))
        y_ref, u, ga, mu, E_acc = out["y"], out["u"], out["g_acc"], out["mu"], out["E_acc"]
        assert _rel(y.cpu().numpy(), y_ref) <= TOL, i
    assert True in decisions[1:] and False in decisions


def test_momentum_graph_replay_equals_eager():
    """Four evaluations recorded once in a CUDA graph and replayed give the eager iterates bit for bit."""
    wl = get_workload("tones8k_n8192")
    plan = _plan(wl.params, 1)
    x = torch.tensor(wl.targets(), device="cuda")
    tgt = plan.forward(x).clone()
    y0 = plan.coloured_init(x, torch.tensor(wl.inits(), device="cuda")).clone()

    def run(use_graph, steps=4):
        y = y0.clone()
        opt = plan.momentum_state(mu0=300.0)
        loss = torch.empty(1, device="cuda")
        if not use_graph:
            for _ in range(steps):
                plan.metamer_step_momentum(y, tgt, opt, loss_out=loss)
        else:
            plan.metamer_step_momentum(y, tgt, opt, loss_out=loss)
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    plan.metamer_step_momentum(y, tgt, opt, loss_out=loss)
            torch.cuda.current_stream().wait_stream(s)
            for _ in range(steps - 1):
                g.replay()
        torch.cuda.synchronize()
        return y.clone(), loss.clone(), opt["state"].clone()

    ye, le, se = run(False)
    yg, lg, sg = run(True)
    assert se[0, 3].item() == sg[0, 3].item() == 4.0
    assert torch.equal(ye, yg) and torch.equal(le, lg) and torch.equal(se, sg)


def test_compare_reconstruction_runs_every_arm():
    """The comparison helper on the tone clip: four arms, finite non-increasing curves, the target reached by Adam."""
    from paper_2602_11896_gb300.reconstruct import compare_reconstruction
    wl = get_workload("tones8k_n8192")
    plan = _plan(wl.params, 1)
    x = torch.tensor(wl.targets(), device="cuda")
    ev = compare_reconstruction(plan, x, plan.forward(x), torch.tensor(wl.inits(), device="cuda"), steps=12)
    assert set(ev["arms"]) == {"white_adam", "coloured_momentum", "coloured_adam", "white_momentum"}
    for arm in ev["arms"].values():
        c = np.array(arm["curve"])
        assert c.shape == (12,) and np.isfinite(c).all() and (np.diff(c) <= 0).all()
    assert 1 <= ev["arms"]["white_adam"]["steps_to_target"] <= 12
    assert ev["arms"]["coloured_adam"]["initial_loss"] < ev["arms"]["white_adam"]["initial_loss"]
