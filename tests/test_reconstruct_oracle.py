"""Pins of the reconstruction oracle (§2.3): coloured initialisation and bold-driver momentum.

Each check rests on something other than the oracle's own formulas: the
already pinned JTFS oracle (S1), adjoint identities, closed-form behaviour on
tones, bursts and white noise, and a trajectory worked out by hand.
"""

import math

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from oracle import reconstruct as R
from workloads import get_workload

F64 = torch.float64


@pytest.fixture(scope="module")
def plan():
    return O.Plan(**get_workload("tones8k_n8192").params)


def _noise(shape, seed):
    return torch.tensor(np.random.default_rng(seed).standard_normal(shape), dtype=F64)


def test_first_order_is_the_transform_s1(plan):
    x = torch.tensor(get_workload("tones8k_n8192").targets(), dtype=F64)
    S1 = R.first_order(x, plan)
    ref = O.jtfs(x, plan, keep=True)["S1"]
    assert float((S1 - ref).abs().max()) <= 1e-12 * float(ref.abs().max())


@pytest.mark.parametrize("n1", [0, 9, 20, 37])
def test_adjoint_identities(plan, n1):
    """<Psi w, g> = <w, Psi^T g> and <P u, s> = <u, P^T s> for random vectors."""
    k1 = plan.k1[n1]
    w = _noise((2, plan.N), 1)
    g = torch.complex(_noise((2, plan.N >> k1), 2), _noise((2, plan.N >> k1), 3))
    lhs = float((R.analysis(w, plan, n1) * g.conj()).real.sum())
    rhs = float((w * R.synthesis(g, plan, n1)).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    u = _noise((2, plan.N >> k1), 4)
    s = _noise((2, plan.n_frames), 5)
    lhs = float((R.pool_T(u, plan, n1) * s).sum())
    rhs = float((u * R.pool_T_adjoint(s, plan, n1)).sum())
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0)


def test_constant_envelope_interpolates_exactly(plan):
    S1 = torch.full((1, plan.N1, plan.n_frames), 2.5, dtype=F64)
    for n1 in range(plan.N1):
        A = R.envelope(S1, plan, n1)
        assert A.shape[-1] == plan.N >> plan.k1[n1]
        assert float((A - 2.5).abs().max()) <= 1e-9


def test_raw_init_is_the_gradient_of_the_weighted_band_energy(plan):
    """y~ = grad_w 1/2 sum_l c_l sum_t A_l |Psi_l w|^2: the band products are A . Psi w, not conj or |.|."""
    x = torch.tensor(get_workload("tones8k_n8192").targets(), dtype=F64)
    w = _noise((1, plan.N), 7).requires_grad_(True)
    S1 = R.first_order(x, plan)
    Q = sum(0.5 * R.band_gain(plan, n1) * (R.envelope(S1, plan, n1) * R.analysis(w, plan, n1).abs() ** 2).sum()
            for n1 in range(plan.N1))
    (grad,) = torch.autograd.grad(Q, w)
    y = R.coloured_init(x, w.detach(), plan, raw=True)
    assert float((y - grad).norm()) <= 1e-10 * float(grad.norm())


def test_linear_in_noise_and_energy_of_target(plan):
    x = torch.tensor(get_workload("tones8k_n8192").targets(), dtype=F64)
    w1, w2 = _noise((1, plan.N), 11), _noise((1, plan.N), 12)
    y1 = R.coloured_init(x, w1, plan, raw=True)
    y2 = R.coloured_init(x, w2, plan, raw=True)
    y12 = R.coloured_init(x, 2.0 * w1 - w2, plan, raw=True)
    assert float((y12 - (2.0 * y1 - y2)).norm()) <= 1e-10 * float(y12.norm())
    y0 = R.coloured_init(x, w1, plan)
    assert abs(float(y0.norm()) - float(x.norm())) <= 1e-10 * float(x.norm())
    assert float((R.coloured_init(x, 3.0 * w1, plan) - y0).norm()) <= 1e-10 * float(y0.norm())
    assert float((R.coloured_init(0.5 * x, w1, plan) - 0.5 * y0).norm()) <= 1e-10 * float(y0.norm())


def test_zero_target_gives_zero(plan):
    y0 = R.coloured_init(torch.zeros(1, plan.N, dtype=F64), _noise((1, plan.N), 13), plan)
    assert not y0.any()


@pytest.mark.parametrize("f0", [0.05, 0.11, 0.23])
def test_tone_target_puts_the_noise_at_the_tone(plan, f0):
    """A pure tone has S1 only in the bands around f0: the init's spectrum sits within 20% of f0."""
    t = torch.arange(plan.N, dtype=F64)
    x = torch.cos(2 * math.pi * f0 * t)[None]
    y0 = R.coloured_init(x, _noise((1, plan.N), 5), plan)
    P = torch.fft.rfft(y0[0]).abs() ** 2
    f = torch.fft.rfftfreq(plan.N, dtype=F64)
    assert float(P[(f - f0).abs() < 0.2 * f0].sum() / P.sum()) > 0.995


def test_burst_target_keeps_silence_silent(plan):
    """A tone in the first half only: the init's energy follows S1 in time."""
    N = plan.N
    t = torch.arange(N, dtype=F64)
    x = (torch.cos(2 * math.pi * 0.11 * t) * (t < N // 2))[None]
    y0 = R.coloured_init(x, _noise((1, N), 5), plan)[0]
    on = float((y0[4 * plan.T:N // 2 - 4 * plan.T] ** 2).sum())
    off = float((y0[N // 2 + 8 * plan.T:N - 8 * plan.T] ** 2).sum())
    assert off < 1e-6 * on


def test_white_target_band_levels_match(plan):
    """White-noise target: per band, the init's mean S1 matches the target's (flat gain c_l)."""
    x = _noise((1, plan.N), 9)
    y0 = R.coloured_init(x, _noise((1, plan.N), 5), plan)
    r = (R.first_order(y0, plan)[0].mean(-1) / R.first_order(x, plan)[0].mean(-1)).numpy()
    assert r.min() > 0.5 and r.max() < 2.0
    assert 0.8 < math.exp(np.log(r).mean()) < 1.25


def test_coloured_init_is_closer_in_s1_than_white_noise(plan):
    x = torch.tensor(get_workload("tones8k_n8192").targets(), dtype=F64)
    w = _noise((1, plan.N), 5)
    S1x = R.first_order(x, plan)
    d_col = float((R.first_order(R.coloured_init(x, w, plan), plan) - S1x).norm() / S1x.norm())
    d_white = float((R.first_order(w * x.norm() / w.norm(), plan) - S1x).norm() / S1x.norm())
    assert d_col < 0.5 * d_white


def test_bold_driver_trajectory_by_hand():
    """E(y) = y^2 (grad 2y) from y = 1, mu0 = 0.1, m = 0.9; every number worked by hand.

    eval 0: E = 1 <= inf  accept, mu 0.1 (first), u = -0.1*2 = -0.2,             y = 0.8
    eval 1: E = 0.64      accept, mu 0.11, u = -0.18 - 0.11*1.6 = -0.356,         y = 0.444
    eval 2: E = 0.197136  accept, mu 0.121, u = -0.3204 - 0.121*0.888 = -0.427848, y = 0.016152
    eval 3: E = 2.60887104e-4 accept, mu 0.1331,
            u = -0.3850632 - 0.1331*0.032304 = -0.3893628624,                     y = -0.3732108624
    eval 4: E = 0.139286... > E_acc  reject, mu 0.06655, back to 0.016152,
            u = -0.06655*0.032304 = -0.0021498312,                                y = 0.0140021688
    """
    y = np.array([[1.0]])
    u = np.zeros((1, 1))
    g_acc = np.zeros((1, 1))
    mu = np.array([0.1])
    E_acc = np.array([np.inf])
    want_y = [0.8, 0.444, 0.016152, -0.3732108624, 0.0140021688]
    want_mu = [0.1, 0.11, 0.121, 0.1331, 0.06655]
    want_acc = [True, True, True, True, False]
    for i in range(5):
        E = (y ** 2).sum(-1)
        out = R.bold_driver_step(y, u, g_acc, mu, E_acc, E, 2.0 * y)
        y, u, g_acc, mu, E_acc = out["y"], out["u"], out["g_acc"], out["mu"], out["E_acc"]
        assert out["accepted"][0] == want_acc[i]
        assert abs(y[0, 0] - want_y[i]) < 1e-12
        assert abs(mu[0] - want_mu[i]) < 1e-15
    assert abs(E_acc[0] - 2.60887104e-4) < 1e-15


def test_bold_driver_clips_are_independent_and_nan_rejects():
    y = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    u = np.array([[0.5, 0.5], [0.1, -0.1], [1.0, 1.0]])
    g_acc = np.array([[1.0, 1.0], [2.0, 2.0], [4.0, 4.0]])
    mu = np.array([0.2, 0.2, 0.2])
    E_acc = np.array([1.0, 1.0, 1.0])
    E = np.array([0.5, 2.0, np.nan])
    g = np.array([[1.0, -1.0], [7.0, 7.0], [9.0, 9.0]])
    out = R.bold_driver_step(y, u, g_acc, mu, E_acc, E, g)
    assert out["accepted"].tolist() == [True, False, False]
    np.testing.assert_allclose(out["mu"], [0.22, 0.1, 0.1])
    np.testing.assert_allclose(out["E_acc"], [0.5, 1.0, 1.0])
    # clip 0: u = 0.9*0.5 - 0.22*g
    np.testing.assert_allclose(out["u"][0], [0.45 - 0.22, 0.45 + 0.22])
    np.testing.assert_allclose(out["y"][0], [1.0 + 0.23, 2.0 + 0.67])
    # clip 1: back to y - u, then -mu*g_acc (the rejected point's gradient is not used)
    np.testing.assert_allclose(out["u"][1], [-0.2, -0.2])
    np.testing.assert_allclose(out["y"][1], [3.0 - 0.1 - 0.2, 4.0 + 0.1 - 0.2])
    np.testing.assert_allclose(out["g_acc"][1], [2.0, 2.0])
    np.testing.assert_allclose(out["y"][2], [5.0 - 1.0 - 0.4, 6.0 - 1.0 - 0.4])


def test_bold_driver_accepted_loss_never_increases_on_the_jtfs_loss():
    """Behaviour on the real loss (tone clip, mu0 = 300, steps that overshoot): the loss at the accepted
    point never increases, every increase is rejected with the step size halved, and y returns to the
    accepted point before stepping again (the next evaluation's loss is below the rejected one)."""
    wl = get_workload("tones8k_n8192")
    op = O.Plan(**wl.params)
    tgt = O.jtfs(torch.tensor(wl.targets(), dtype=F64), op)["phi"]
    y = wl.inits().astype(np.float64)
    u = np.zeros_like(y)
    g_acc = np.zeros_like(y)
    mu = np.array([300.0])
    E_acc = np.array([np.inf])
    history = []
    for _ in range(8):
        E, g = O.loss_and_grad(torch.tensor(y), tgt, op)
        out = R.bold_driver_step(y, u, g_acc, mu, E_acc, E.numpy(), g.numpy())
        history.append((float(E[0]), bool(out["accepted"][0]), float(mu[0]), float(out["mu"][0]),
                        float(E_acc[0]), float(out["E_acc"][0])))
        y, u, g_acc, mu, E_acc = out["y"], out["u"], out["g_acc"], out["mu"], out["E_acc"]
    accepted = [h[1] for h in history]
    assert True in accepted[1:] and False in accepted
    for E, acc, mu_in, mu_out, ea_in, ea_out in history:
        assert ea_out <= ea_in
        if acc:
            assert E <= ea_in and ea_out == E
        else:
            assert E > ea_in and ea_out == ea_in and mu_out == 0.5 * mu_in
