"""Pins of the reflect boundary in the oracle (reading R20: §3.2's padding on both sides)."""

import math

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O

TINY = dict(J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2)


@pytest.mark.parametrize("L", [1, 2, 5, 37])
def test_reflect_index_is_numpy_reflect_padding(L):
    """The mirror extension equals numpy's 'reflect' padding, including pads longer than the clip."""
    x = np.random.default_rng(L).standard_normal(L)
    left, right = 3 * L + 7, 2 * L + 11
    want = np.pad(x, (left, right), mode="reflect")
    idx = O.reflect_index(torch.arange(-left, L + right), L).numpy()
    np.testing.assert_array_equal(x[idx], want)


def test_pad_width_is_where_the_slowest_envelope_drops_to_1e3():
    plan = O.Plan(N=2 ** 6, **{k: v for k, v in TINY.items()})
    sig = min([f.sigma for f in plan.psi1] + [f.sigma for f in plan.psi2] + [plan.sigma_phiT])
    P = O.reflect_pad_width(TINY)
    env = lambda t: math.exp(-2 * math.pi ** 2 * sig ** 2 * t * t)
    assert env(P) <= 1e-3 < env(P - 1)


@pytest.mark.parametrize("L", [1, 37, 200, 256])
def test_layout_keeps_the_clip_on_the_frame_grid(L):
    T = TINY["T"]
    n, p0, f0, nf = O.reflect_layout(L, TINY)
    P = O.reflect_pad_width(TINY)
    assert n & (n - 1) == 0 and n >= L + 2 * P
    assert p0 % T == 0 and f0 == p0 // T and nf == -(-L // T)
    assert p0 > P - T and n - L - p0 >= P
    assert f0 + nf <= n // T


def test_constant_clip_has_exact_lowpass_and_no_bandpass_energy():
    """A constant's mirror extension is constant: S0 = c on every kept frame, every wavelet path 0."""
    L = 200
    c = 1.75
    phi = O.jtfs_reflect(torch.full((L,), c, dtype=torch.float64), TINY).reshape(-1, -(-L // 16))
    assert float((phi[0] - c).abs().max()) <= 1e-12
    assert float(phi[1:].abs().max()) <= 1e-12
    # Zero padding on the right (R15) does not have this property at the clip's end.
    phi0 = O.jtfs_uneven(torch.full((L,), c, dtype=torch.float64), TINY).reshape(-1, -(-L // 16))
    assert float((phi0[0] - c).abs().max()) > 1e-2


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    L = 97
    y = torch.tensor(rng.standard_normal(L))
    tgt = O.jtfs_reflect(torch.tensor(rng.standard_normal(L)), TINY)
    E, g = O.loss_and_grad_reflect(y, tgt, TINY)
    h = 1e-6
    for i in rng.choice(L, 8, replace=False).tolist() + [0, L - 1]:
        e = torch.zeros(L, dtype=torch.float64)
        e[i] = h
        fd = (((O.jtfs_reflect(y + e, TINY) - tgt) ** 2).sum() - ((O.jtfs_reflect(y - e, TINY) - tgt) ** 2).sum()) / (2 * h)
        assert abs(float(fd) - float(g[i])) <= 1e-6 * max(1.0, abs(float(g[i]))), i
