"""Pins of the unpooled variants in the oracle (average_local / average_local_fr = False, reading R21).

The FFT-and-decimation oracle against the brute-force route (direct time-domain
convolution, retyped schedule) for every combination, exact frame shifts of
every block at its own stride, the zeroth order equal to the signal,
central finite differences of the gradient, and the pooled transform
recovered from the unpooled one by the averaging it skips.
"""

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from oracle.bruteforce import jtfs_bruteforce

SMALL = [
    dict(N=256, J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2),
    dict(N=512, J=5, Q=3, Q2=2, J_fr=2, Q_fr=2, T=32, F=3),    # phi_F stride 2 > log2 F = 1
    dict(N=256, J=5, Q=2, Q2=1, J_fr=2, Q_fr=1, T=8, F=4),     # j1, j2 up to 4 > log2 T = 3
]
MODES = [(False, True), (True, False), (False, False)]


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("params", SMALL)
def test_unpooled_oracle_equals_bruteforce(params, mode):
    p = O.Plan(**params, average_local=mode[0], average_local_fr=mode[1])
    x = np.random.default_rng(3).standard_normal((2, p.N))
    a = O.jtfs(torch.tensor(x), p)["phi"].numpy()
    b = jtfs_bruteforce(x, p)["phi"]
    assert a.shape == b.shape == (2, p.phi_size)
    assert _rel(a, b) < 1e-12


@pytest.mark.parametrize("mode", MODES)
def test_every_block_shifts_by_whole_frames(mode):
    """Periodic boundary: shifting x by 2^m (m >= every stride) shifts each block by 2^m / its stride frames."""
    params = SMALL[2]
    p = O.Plan(**params, average_local=mode[0], average_local_fr=mode[1])
    shift = 2 ** max([p.lT] + [f.j for f in p.psi2])
    x = torch.tensor(np.random.default_rng(7).standard_normal((1, p.N)))
    a = O.phi_blocks(O.jtfs(x, p)["phi"], p)
    b = O.phi_blocks(O.jtfs(torch.roll(x, shift, -1), p)["phi"], p)
    s0 = p.N if not p.average_local else p.n_frames
    assert torch.allclose(b["S0"], torch.roll(a["S0"], shift * s0 // p.N, -1), atol=1e-12)
    nf = p.n_frames
    assert torch.allclose(b["first"].reshape(-1, nf), torch.roll(a["first"].reshape(-1, nf), shift // p.T, -1),
                          atol=1e-12)
    for n2 in p.active:
        fr = p.frames2(n2)
        got = b[f"n2={n2}"].reshape(-1, fr)
        want = torch.roll(a[f"n2={n2}"].reshape(-1, fr), shift * fr // p.N, -1)
        assert torch.allclose(got, want, atol=1e-12), n2


def test_time_unpooled_zeroth_order_is_the_signal():
    p = O.Plan(**SMALL[0], average_local=False)
    x = torch.tensor(np.random.default_rng(1).standard_normal((2, p.N)))
    assert torch.equal(O.phi_blocks(O.jtfs(x, p)["phi"], p)["S0"], x)


def test_pooling_the_unpooled_recovers_the_transform():
    """Where the strides agree (every j2 and frequential j within the caps), phi_T and phi_F applied to the
    unpooled second-order blocks give the default transform's blocks."""
    params = SMALL[0]
    base = O.Plan(**params)
    assert all(f.j <= base.lT for f in base.psi1 + base.psi2)
    assert all(b[2] <= base.lF for b in base.beta_second)
    un = O.Plan(**params, average_local=False, average_local_fr=False)
    x = torch.tensor(np.random.default_rng(2).standard_normal((1, base.N)))
    ref = O.phi_blocks(O.jtfs(x, base)["phi"], base)
    got = O.phi_blocks(O.jtfs(x, un)["phi"], un)
    phiT = O.gauss_hat(base.N, base.sigma_phiT)
    phiF = O.gauss_hat(base.N_fr, base.sigma_phiF)
    for n2 in base.active:
        s2 = un.s2[n2]
        blocks, o = [], 0
        rows_all = got[f"n2={n2}"].reshape(-1, un.frames2(n2))
        for beta in un.beta_second:
            R = un.rows(beta)
            u = rows_all[o:o + R][None]
            o += R
            a = O.decimate(O.conv_circ(u.to(O.C128), O.periodise(phiT, s2), 2), base.lT - s2, 2).real
            v = O.decimate(O.conv_circ(a.to(O.C128), O.periodise(phiF, beta[2]), 1), base.lF - beta[2], 1).real
            blocks.append(v.reshape(-1))
        assert _rel(torch.cat(blocks), ref[f"n2={n2}"].reshape(-1)) < 1e-12, n2


def test_unpooled_gradient_matches_central_differences():
    params = SMALL[2]
    p = O.Plan(**params, average_local=False, average_local_fr=False)
    rng = np.random.default_rng(6)
    y = torch.tensor(rng.standard_normal((1, p.N)))
    tgt = O.jtfs(torch.tensor(rng.standard_normal((1, p.N))), p)["phi"]
    E, g = O.loss_and_grad(y, tgt, p)
    h = 1e-6
    for i in rng.choice(p.N, 8, replace=False):
        e = torch.zeros(1, p.N, dtype=torch.float64)
        e[0, i] = h
        fd = (O.loss(y + e, tgt, p) - O.loss(y - e, tgt, p)) / (2 * h)
        assert abs(float(fd) - float(g[0, i])) <= 1e-6 * max(1.0, abs(float(g[0, i])))
