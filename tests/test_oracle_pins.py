"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a special case or an independent brute-force evaluation.
"""

import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from oracle.bruteforce import jtfs_bruteforce

GOLD = os.path.join(os.path.dirname(__file__), "golden", "filterbank_counts.json")

TINY = [
    dict(N=256, J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2),
    dict(N=512, J=5, Q=3, Q2=2, J_fr=2, Q_fr=2, T=32, F=3),
    dict(N=256, J=3, Q=2, Q2=1, J_fr=1, Q_fr=1, T=8, F=1),
]
CFG1 = dict(N=2 ** 13, J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4)


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# --------------------------------------------------------------------------- filterbank (§3.1)

def test_filterbank_counts_closed_form():
    """Counts of the §3.1 generator equal the hand-derived closed form."""
    gold = json.load(open(GOLD))
    for c in gold["cases"]:
        fb = O.morlet_filterbank(c["J"], c["Q"])
        assert len(fb) == c["count"], c
        # Constant-Q part: xi/sigma constant; constant-bandwidth part: sigma = sigma0/2^J.
        smin = 0.1 / 2 ** c["J"]
        ncq = sum(1 for _, s in fb if s != smin)
        assert ncq == c["constant_q"], c


def test_filterbank_first_filter_and_progressions():
    """xi_0, sigma_0 from the listing's formulas; geometric then arithmetic steps."""
    for J, Q in [(6, 8), (12, 12), (6, 1), (5, 2)]:
        fb = O.morlet_filterbank(J, Q)
        xi0 = max(1.0 / (1.0 + 2.0 ** (3.0 / Q)), 0.35)
        s0 = (1 - 2 ** (-1 / Q)) / (1 + 2 ** (-1 / Q)) * xi0 / math.sqrt(math.log(2.0))
        assert abs(fb[0][0] - xi0) < 1e-15 and abs(fb[0][1] - s0) < 1e-15
        smin = 0.1 / 2 ** J
        cq = [f for f in fb if f[1] != smin]
        cb = [f for f in fb if f[1] == smin]
        for (xa, sa), (xb, sb) in zip(cq, cq[1:]):
            assert abs(xb / xa - 2 ** (-1 / Q)) < 1e-12 and abs(sb / sa - 2 ** (-1 / Q)) < 1e-12
        assert len(cb) == Q - 1
        if cb:
            elbow = cq[-1][0]
            for q, (x, _) in enumerate(cb, start=1):
                assert abs(x - elbow * (1 - q / Q)) < 1e-14
        xs = [x for x, _ in fb]
        assert all(a > b for a, b in zip(xs, xs[1:])) and xs[-1] > 0


def test_phi_sizes_of_named_workloads():
    gold = json.load(open(GOLD))["phi_size"]
    assert O.Plan(**CFG1).phi_size == gold["tones8k_n8192"]
    p2 = O.Plan(N=2 ** 16, J=12, Q=12, Q2=1, J_fr=5, Q_fr=2, T=2 ** 11, F=12)
    assert p2.phi_size == gold["chirps22k_b8_n65536"]


# --------------------------------------------------------------------------- subsampling j (reading R2)

SUBS = os.path.join(os.path.dirname(__file__), "golden", "subsampling_j.json")


def _subsampling_mismatches():
    """Differences between the oracle's schedule and the hand-derived tables (empty when they agree)."""
    gold = json.load(open(SUBS))["configs"]
    bad = []
    for name, g in gold.items():
        p = O.Plan(**g["params"])
        for key, fb in (("psi1", p.psi1), ("psi2", p.psi2), ("psi_fr", p.psi_fr)):
            if [f.j for f in fb] != [e["j"] for e in g[key]]:
                bad.append((name, key))
        if p.j_phiT != g["phi_T"]["j"] or p.j_phiT != p.lT:
            bad.append((name, "phi_T"))
        if p.j_phiF != g["phi_F"]["j"]:
            bad.append((name, "phi_F"))
        if p.n1_max != g["n1_max"]:
            bad.append((name, "n1_max"))
    return bad


def test_subsampling_matches_hand_derived_tables():
    """Every filter's j, j(phi_T) = log2 T and the row counts n1_max of the tone and chirp plans equal
    the tables derived in 50-digit arithmetic from the closed forms (tests/golden/subsampling_j.json)."""
    assert _subsampling_mismatches() == []
    gold = json.load(open(SUBS))["configs"]
    from oracle.bruteforce import schedule
    for g in gold.values():
        p = O.Plan(**g["params"])
        for key, fb in (("psi1", p.psi1), ("psi2", p.psi2), ("psi_fr", p.psi_fr)):
            for f, e in zip(fb, g[key]):      # the restated filterbank against the closed form
                assert abs(f.xi - e["xi"]) <= 1e-14 and abs(f.sigma - e["sigma"]) <= 1e-14
        sch = schedule(p)                     # the brute force's own schedule
        assert sch["j1"] == [e["j"] for e in g["psi1"]] and sch["j2"] == [e["j"] for e in g["psi2"]]
        assert [len(r) for r in sch["rows2"]] == g["n1_max"]


def test_phi_T_subsampling_is_log2_T():
    """phi_T of width 0.1 / T (reading R3) has j = log2 T: 3 x 0.1 lies in (1/4, 1/2]."""
    for lT in range(0, 16):
        T = 2 ** lT
        assert O.max_subsampling(0.0, 0.1 / T) == lT
        assert O.Plan(N=max(T, 16), J=2, Q=1, Q2=1, J_fr=1, Q_fr=1, T=T, F=1).j_phiT == lT


@pytest.mark.parametrize("plant", ["xi_plus_2_sigma", "round"])
def test_pins_catch_wrong_subsampling(monkeypatch, plant):
    """Plant a misreading of R2 in the oracle: the hand-derived tables and the brute force (which derives
    its own schedule) must both disagree."""
    p0 = O.Plan(**TINY[1])
    x = np.random.default_rng(13).standard_normal((1, p0.N))

    def two_sigma(xi, sigma):
        return max(0, int(math.floor(math.log2(0.5 / (xi + 2.0 * sigma)))))

    def rounded(xi, sigma):
        return max(0, int(round(math.log2(0.5 / (xi + 3.0 * sigma)))))

    monkeypatch.setattr(O, "max_subsampling", two_sigma if plant == "xi_plus_2_sigma" else rounded)
    assert _subsampling_mismatches() != []
    p = O.Plan(**TINY[1])
    a = O.jtfs(torch.tensor(x), p)["phi"].numpy()
    b = jtfs_bruteforce(x, p)["phi"]
    assert a.shape != b.shape or _rel(a, b) > 1e-3


# --------------------------------------------------------------------------- filters (Eq. 1)

def test_morlet_zero_mean_and_peak():
    """kappa gives psi_hat(0) = 0 (one vanishing moment, Eq. (1)); time-domain sum is 0."""
    p = O.Plan(**CFG1)
    for f in p.psi1 + p.psi2:
        h = O.morlet_hat(p.N, f.xi, f.sigma)
        assert abs(h[0].item()) < 1e-15
        assert abs(torch.fft.ifft(h.to(O.C128)).sum().item()) < 1e-12
    for f in p.psi_fr:
        for s in (+1, -1):
            h = O.morlet_hat(p.N_fr, s * f.xi, f.sigma)
            assert abs(h[0].item()) < 1e-15


def test_littlewood_paley_bounds():
    """Energy cover of the first-order filterbank (standard frame property).

    r_psi = sqrt(1/2) makes neighbours cross at |psi_hat|^2 = 1/2, so inside
    the constant-Q band the LP sum stays within about [1, 1 + 2 r^4]; a wrong
    bandwidth formula moves it out.  Over all positive frequencies A > 0.
    """
    p = O.Plan(**CFG1)
    w = O.fourier_grid(p.N)
    lp = O.gauss_hat(p.N, p.sigma_phiT) ** 2
    for f in p.psi1:
        lp = lp + O.morlet_hat(p.N, f.xi, f.sigma) ** 2
    ncq = sum(1 for f in p.psi1 if f.sigma != 0.1 / 2 ** p.J)
    band = (w >= p.psi1[ncq - 1].xi) & (w <= p.psi1[0].xi)
    A, B = lp[band].min().item(), lp[band].max().item()
    assert 0.99 <= A <= B <= 1.0 + 2 * 0.5 ** 2 + 0.01
    assert lp[w > 0].min().item() > 0


# --------------------------------------------------------------------------- brute force

@pytest.mark.parametrize("params", TINY)
def test_oracle_equals_bruteforce(params):
    """FFT + decimation route == direct convolution with time-domain level filters."""
    p = O.Plan(**params)
    x = np.random.default_rng(3).standard_normal((2, p.N))
    a = O.jtfs(torch.tensor(x), p)["phi"].numpy()
    b = jtfs_bruteforce(x, p)["phi"]
    assert a.shape == (2, p.phi_size)
    assert _rel(a, b) < 1e-12


def test_strided_U1_is_decimated_full_rate():
    """U1 at stride 2^k1 equals |x * psi| computed at full rate, decimated."""
    p = O.Plan(**TINY[0])
    x = torch.tensor(np.random.default_rng(5).standard_normal((1, p.N)))
    o = O.jtfs(x, p, keep=True)
    from oracle.bruteforce import circ_conv, idft_explicit, _morlet
    for n1, f in enumerate(p.psi1):
        full = np.abs(circ_conv(x.numpy().astype(np.complex128), idft_explicit(_morlet(p.N, f.xi, f.sigma))))
        assert np.abs(o["U1"][n1].numpy() - full[:, :: 2 ** p.k1[n1]]).max() < 1e-12


# --------------------------------------------------------------------------- invariants

def test_positive_homogeneity_and_sign():
    """Phi(c x) = |c| Phi(x) on the scattering paths (linear maps and moduli,
    Eqs. (2), (4), (5)); S0 = x * phi_T has no modulus and scales by c."""
    p = O.Plan(**TINY[1])
    x = torch.tensor(np.random.default_rng(7).standard_normal((1, p.N)))
    a = O.jtfs(x, p)["phi"]
    nf = p.n_frames
    for c in (-2.5, 0.3):
        b = O.jtfs(c * x, p)["phi"]
        assert _rel(b[:, nf:], abs(c) * a[:, nf:]) < 1e-13
        assert _rel(b[:, :nf], c * a[:, :nf]) < 1e-13


@pytest.mark.parametrize("params", [TINY[0], TINY[1], CFG1])
def test_shift_by_T_shifts_frames(params):
    """Periodic boundary and strides dividing T: shifting x by T shifts every frame by one."""
    p = O.Plan(**params)
    x = torch.tensor(np.random.default_rng(11).standard_normal((1, p.N)))
    a = O.jtfs(x, p)["phi"].reshape(-1)
    b = O.jtfs(torch.roll(x, p.T, -1), p)["phi"].reshape(-1)
    nf = p.n_frames
    a_fr = a.reshape(-1, nf)      # every Phi block is [..., frame]
    b_fr = b.reshape(-1, nf)
    assert _rel(b_fr, torch.roll(a_fr, 1, -1)) < 1e-12


def test_small_shifts_change_phi_little():
    """Averaging by phi_T makes Phi nearly invariant to shifts tau << T (§1.2, §2.2)."""
    p = O.Plan(**CFG1)
    x = torch.tensor(np.random.default_rng(0).standard_normal((1, p.N)))
    a = O.jtfs(x, p)["phi"]
    d = []
    for tau in (1, 4, 16, 64):
        d.append(_rel(O.jtfs(torch.roll(x, tau, -1), p)["phi"], a))
    assert d[0] < 0.01
    assert all(u < v for u, v in zip(d, d[1:]))
    assert d[-1] < 0.2


def test_pure_tone_closed_form():
    """x = cos(2 pi xi0 t), xi0 on the DFT grid: U1 = |a e^{i th} + b e^{-i th}|.

    a = psi_hat(xi0)/2, b = psi_hat(-xi0)/2.  At xi0 = 1/4, b vanishes for every
    first-order filter, so U1 is constant, S1 = |a| (phi_T has unit DC gain),
    S0 = phi_hat_T(xi0) cos(2 pi xi0 T t) ~ 0, and every second-order path
    vanishes because psi_alpha has a null average (Eq. (1)).
    """
    p = O.Plan(**CFG1)
    n = p.N
    for m0, check_b in ((n // 4, False), (3, True), (41, True)):
        xi0 = m0 / n
        t = torch.arange(n, dtype=torch.float64)
        x = torch.cos(2 * math.pi * xi0 * t)[None]
        o = O.jtfs(x, p, keep=True)
        for n1, f in enumerate(p.psi1):
            a = 0.5 * O.morlet_hat(n, f.xi, f.sigma)[m0].item()
            b = 0.5 * O.morlet_hat(n, f.xi, f.sigma)[n - m0].item()
            tt = torch.arange(0, n, 2 ** p.k1[n1], dtype=torch.float64)
            th = 2 * math.pi * xi0 * tt
            cf = torch.abs(a * torch.exp(1j * th) + b * torch.exp(-1j * th))
            assert (o["U1"][n1][0] - cf).abs().max().item() < 1e-12
        if not check_b:
            for n1, f in enumerate(p.psi1):
                a = 0.5 * abs(O.morlet_hat(n, f.xi, f.sigma)[m0].item())
                assert (o["S1"][0, n1] - a).abs().max().item() < 1e-12
            phiT0 = math.exp(-xi0 ** 2 / (2 * p.sigma_phiT ** 2))
            s0 = phiT0 * torch.cos(2 * math.pi * xi0 * p.T * torch.arange(p.n_frames, dtype=torch.float64))
            assert (o["S0"][0] - s0).abs().max().item() < 1e-13
            assert o["Phi2"].abs().max().item() < 1e-12 * o["Phi1"].abs().max().item() + 1e-13


def test_kappa_matters_for_low_filters():
    """The corrective term is not negligible for the constant-bandwidth filters."""
    p = O.Plan(**CFG1)
    f = p.psi1[-1]
    kappa = math.exp(-f.xi ** 2 / (2 * f.sigma ** 2))
    assert kappa > 1e-2


# --------------------------------------------------------------------------- gradient (§2.3)

def test_gradient_matches_central_differences():
    p = O.Plan(**TINY[0])
    rng = np.random.default_rng(1)
    y = torch.tensor(rng.standard_normal((1, p.N)))
    tgt = O.jtfs(torch.tensor(rng.standard_normal((1, p.N))), p)["phi"]
    E, g = O.loss_and_grad(y, tgt, p)
    h = 1e-5
    for k in range(4):
        d = torch.tensor(rng.standard_normal((1, p.N)))
        d = d / d.norm()
        fd = (O.loss(y + h * d, tgt, p) - O.loss(y - h * d, tgt, p)).item() / (2 * h)
        an = (g * d).sum().item()
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * g.norm().item())
    for i in rng.choice(p.N, 4, replace=False):
        e = torch.zeros_like(y)
        e[0, i] = 1.0
        fd = (O.loss(y + h * e, tgt, p) - O.loss(y - h * e, tgt, p)).item() / (2 * h)
        assert abs(fd - g[0, i].item()) <= 1e-6 * g.abs().max().item()


def test_gradient_null_for_metamers():
    """∇E vanishes when Phi(y) equals the target (the remark closing §2.3)."""
    p = O.Plan(**TINY[1])
    y = torch.tensor(np.random.default_rng(2).standard_normal((1, p.N)))
    E, g = O.loss_and_grad(y, O.jtfs(y, p)["phi"], p)
    assert E.item() == 0.0 and g.abs().max().item() == 0.0


def test_checkpointed_gradient_identical():
    p = O.Plan(**TINY[0])
    rng = np.random.default_rng(4)
    y = torch.tensor(rng.standard_normal((2, p.N)))
    tgt = O.jtfs(torch.tensor(rng.standard_normal((2, p.N))), p)["phi"]
    _, g1 = O.loss_and_grad(y, tgt, p)
    _, g2 = O.loss_and_grad(y, tgt, p, checkpoint_blocks=True)
    assert (g1 - g2).abs().max().item() <= 1e-13 * g1.abs().max().item()


def test_selected_second_order_paths_equal_the_full_transform():
    """The path-subset evaluation (used to sample long signals) returns exactly the
    blocks of the full transform."""
    p = O.Plan(**TINY[1])
    x = torch.tensor(np.random.default_rng(6).standard_normal((2, p.N)))
    full = O.jtfs(x, p, keep=True)
    sel = O.jtfs(x, p, active=[0, len(p.active) - 1])
    assert torch.equal(sel["S0"], full["S0"]) and torch.equal(sel["Phi1"], full["Phi1"])
    for a, blk in sel["Phi2_sel"].items():
        assert torch.equal(blk, full["Phi2"][:, a])


def test_second_order_frames_equal_the_full_transform():
    """The frame-restricted second order (phi_T as its sum over the columns where the taps are not
    negligible) equals the whole transform's frames, on a plan where that is a small part of the columns."""
    p = O.Plan(N=2 ** 13, J=5, Q=4, Q2=2, J_fr=2, Q_fr=1, T=16, F=2)
    x = torch.tensor(np.random.default_rng(11).standard_normal((2, p.N)))
    full = O.jtfs(x, p, keep=True)["Phi2"]
    frames = [0, 3, p.n_frames - 1]
    for a in range(len(p.active)):
        got = O.second_order_frames(x, p, a, frames)
        assert got.shape == (2, 1 + 2 * p.K, p.R_out, len(frames))
        assert (got - full[:, a][..., frames]).abs().max().item() <= 1e-12 * full[:, a].abs().max().item()


# --------------------------------------------------------------------------- planted mistakes

def test_pins_catch_dropped_kappa(monkeypatch):
    """Plant a mistake in the oracle (drop kappa): the closed-form pin must fail."""
    p = O.Plan(**CFG1)
    n = p.N

    def no_kappa(nn, xi, sigma):
        w = O.fourier_grid(nn)
        return torch.exp(-(w - xi) ** 2 / (2.0 * sigma * sigma))

    m0 = 41
    x = torch.cos(2 * math.pi * m0 / n * torch.arange(n, dtype=torch.float64))[None]
    f = p.psi1[-1]
    a = 0.5 * O.morlet_hat(n, f.xi, f.sigma)[m0].item()
    b = 0.5 * O.morlet_hat(n, f.xi, f.sigma)[n - m0].item()
    monkeypatch.setattr(O, "morlet_hat", no_kappa)
    o = O.jtfs(x, p, keep=True)
    tt = torch.arange(0, n, 2 ** p.k1[-1], dtype=torch.float64)
    th = 2 * math.pi * m0 / n * tt
    cf = torch.abs(a * torch.exp(1j * th) + b * torch.exp(-1j * th))
    assert (o["U1"][-1][0] - cf).abs().max().item() > 1e-4


def test_pins_catch_wrong_decimation_phase(monkeypatch):
    """Plant a mistake (decimate starting at sample 1): shift-by-T and brute force must fail."""
    p = O.Plan(**TINY[0])
    x = np.random.default_rng(3).standard_normal((1, p.N))
    ref = jtfs_bruteforce(x, p)["phi"]

    def bad_decimate(z, k, dim):
        if k == 0:
            return z
        idx = torch.arange(1, z.shape[dim], 2 ** k)
        return z.index_select(dim, idx)

    monkeypatch.setattr(O, "decimate", bad_decimate)
    a = O.jtfs(torch.tensor(x), p)["phi"].numpy()
    assert _rel(a, ref) > 1e-3


def test_pins_catch_wrong_spin(monkeypatch):
    """Plant a mistake (frequential wavelets spun the wrong way, §3.4): brute force must fail.

    (Time-reversing every filter at once is not a mistake this can see: for a
    real input each stage then only conjugates, and the moduli hide it.)
    """
    p = O.Plan(**TINY[0])
    x = np.random.default_rng(9).standard_normal((1, p.N))
    ref = jtfs_bruteforce(x, p)["phi"]
    orig = O.freq_filter_hat
    monkeypatch.setattr(O, "freq_filter_hat", lambda n, xi, sigma: orig(n, -xi, sigma))
    a = O.jtfs(torch.tensor(x), p)["phi"].numpy()
    assert _rel(a, ref) > 1e-3


# --------------------------------------------------------------------------- uneven lengths (R15)

def test_uneven_length_power_of_two_is_plain_phi():
    """For L a power of two the pad and the crop are identities."""
    p = dict(TINY[0])
    x = torch.tensor(np.random.default_rng(21).standard_normal(p["N"]))
    a = O.jtfs_uneven(x, p)
    b = O.jtfs(x[None], O.Plan(**p))["phi"][0]
    assert torch.equal(a, b)


def test_uneven_length_is_padded_and_cropped():
    """Phi of a clip of length L equals Phi of its zero-padded copy, cropped to ceil(L/T) frames;
    the gradient never touches the padding (it has no samples there)."""
    p = dict(TINY[0])
    L = 200
    x = torch.tensor(np.random.default_rng(22).standard_normal(L))
    a = O.jtfs_uneven(x, p)
    plan = O.Plan(**p)
    xp = torch.cat([x, torch.zeros(p["N"] - L, dtype=torch.float64)])[None]
    full = O.jtfs(xp, plan)["phi"].reshape(-1, plan.n_frames)
    nf = -(-L // p["T"])
    assert nf < plan.n_frames
    assert torch.equal(a, full[:, :nf].reshape(-1))
    tgt = torch.zeros_like(a)
    E, g = O.loss_and_grad_uneven(x, tgt, p)
    assert g.shape == (L,)
    assert abs(E.item() - (a ** 2).sum().item()) <= 1e-12 * E.item()


# --------------------------------------------------------------------------- decoder layers

def test_decoder_conv_transpose_reference_is_the_defining_sum():
    from oracle import decoder_oracle as D
    rng = np.random.default_rng(8)
    x = rng.standard_normal((2, 3, 7))
    w = rng.standard_normal((3, 4, 9))
    b = rng.standard_normal(4)
    a = D.conv_transpose(torch.tensor(x), torch.tensor(w), torch.tensor(b)).numpy()
    assert a.shape == (2, 4, 14)
    assert np.abs(a - D.conv_transpose_direct(x, w, b)).max() < 1e-12


def test_decoder_gelu_closed_form_points():
    from oracle import decoder_oracle as D
    z = torch.tensor([0.0, 1.0, -1.0, 3.0])
    g = D.gelu(z)
    assert g[0].item() == 0.0
    assert abs(g[1].item() - 0.8413447460685429) < 1e-12          # Phi_N(1)
    assert abs(g[2].item() + 0.15865525393145707) < 1e-12          # -(1 - Phi_N(1))
    assert abs(g[3].item() - 3 * 0.9986501019683699) < 1e-12
