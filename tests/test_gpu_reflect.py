"""Reflect boundary (mirror padding on both sides, oracle reading R20) through the ragged-batch C ABI."""

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from workloads import signals

pytestmark = pytest.mark.gpu

TOL = 1e-4
TINY = dict(J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2)
TONES = dict(J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _batch(lengths, params):
    from paper_2602_11896_gb300 import JTFSBatch
    return JTFSBatch(lengths, **params, boundary="reflect")


def _clips(lengths, seed):
    return [signals.white_noise(int(L), seed + i) for i, L in enumerate(lengths)]


@pytest.mark.parametrize("lengths,params", [([1, 37, 200, 256, 512, 16], TINY), ([3000, 8192], TONES)])
def test_reflect_forward_matches_oracle_per_clip(lengths, params):
    b = _batch(lengths, params)
    clips = _clips(lengths, 5)
    phi = b.forward(torch.tensor(np.concatenate(clips), device="cuda")).cpu().numpy()
    for i, c in enumerate(clips):
        ref = O.jtfs_reflect(torch.tensor(c, dtype=torch.float64), dict(params)).numpy()
        got = phi[b.phi_offsets[i]:b.phi_offsets[i + 1]]
        assert got.shape == ref.shape, (i, got.shape, ref.shape)
        assert _rel(got, ref) <= TOL, i


def test_reflect_constant_clip():
    """A constant clip: S0 equals the constant on every kept frame, every wavelet path vanishes."""
    L, c = 300, 1.5
    b = _batch([L], TINY)
    phi = b.forward(torch.full((L,), c, device="cuda")).cpu().numpy().reshape(-1, -(-L // 16))
    assert np.abs(phi[0] - c).max() <= 1e-5 * c
    assert np.abs(phi[1:]).max() <= 1e-5 * c


def test_reflect_metamer_step_matches_oracle_gradient():
    lengths = [37, 200, 512]
    b = _batch(lengths, TINY)
    y0 = _clips(lengths, 30)
    targets = [O.jtfs_reflect(torch.tensor(c, dtype=torch.float64), dict(TINY)) for c in _clips(lengths, 40)]
    y = torch.tensor(np.concatenate(y0), device="cuda")
    tgt = torch.cat(targets).float().cuda()
    m = torch.zeros_like(y)
    v = torch.zeros_like(y)
    step = torch.ones(1, dtype=torch.int32, device="cuda")
    loss = b.metamer_step(y, tgt, m, v, step, 0.1)
    torch.cuda.synchronize()
    for i, (c, t) in enumerate(zip(y0, targets)):
        E, g = O.loss_and_grad_reflect(torch.tensor(c, dtype=torch.float64), t, dict(TINY))
        assert _rel([loss[i].item()], [E.item()]) <= TOL
        s0, s1 = b.sample_offsets[i], b.sample_offsets[i + 1]
        # Adam's first moment after one step is 0.1 g: the folded gradient itself.
        assert _rel(m[s0:s1].double().cpu().numpy(), (0.1 * g).numpy()) <= TOL, i
        upd = y[s0:s1].double().cpu() - torch.tensor(c, dtype=torch.float64)
        big = g.abs() > 1e-3 * g.abs().max()
        assert torch.allclose(upd[big], (-0.1 * g / (g.abs() + 1e-8))[big], rtol=0, atol=1e-4)
