"""Brute-force JTFS for tiny inputs: direct O(n^2) circular convolution.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

It evaluates the same discrete definition as ``jtfs_oracle.jtfs`` by a
different route, so that a transposed operand, a wrong sign, a dropped
alias or a wrong decimation phase in either one shows up as a mismatch:

* time-domain filters are built from their Fourier samples by an explicit
  inverse-DFT sum written with cos/sin (no FFT);
* a filter at resolution level k is its full-rate impulse response
  decimated and scaled, 2^k h[2^k t] (the time-domain reading of
  "levels[k]", §3.2-§3.3), not a periodised spectrum;
* every convolution is the direct sum y[t] = sum_s x[s] h[(t - s) mod n].

* the multirate schedule is derived here from the filters' (xi, sigma)
  alone: the subsampling j of a filter (reading R2: the largest k >= 0 with
  2^k (xi + 3 sigma) <= 1/2) by counting doublings, the strides k1, s2, k_fr,
  the second-order row sets (j1 < j2), N_fr and R_out, so that a misreading
  of the schedule in ``jtfs_oracle`` shows up here too.

Only the filterbank values (xi, sigma of every filter, pinned separately by
the closed-form counts and progressions of §3.1) and the configuration are
taken from the oracle's ``Plan``.
"""

from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

from .jtfs_oracle import Plan


def _grid(n: int) -> np.ndarray:
    m = np.arange(n, dtype=np.float64)
    return np.where(m < n / 2, m, m - n) / n


def _morlet(n: int, xi: float, sigma: float) -> np.ndarray:
    w = _grid(n)
    if xi == 0.0:
        return np.exp(-w * w / (2 * sigma * sigma))
    kappa = math.exp(-xi * xi / (2 * sigma * sigma))
    return np.exp(-(w - xi) ** 2 / (2 * sigma * sigma)) - kappa * np.exp(-w * w / (2 * sigma * sigma))


def idft_explicit(h_hat: np.ndarray) -> np.ndarray:
    """h[t] = (1/n) sum_m h_hat[m] exp(+2 pi i m t / n), summed term by term."""
    n = h_hat.shape[0]
    t = np.arange(n)[:, None]
    m = np.arange(n)[None, :]
    ang = 2.0 * math.pi * ((m * t) % n) / n
    return (np.cos(ang) + 1j * np.sin(ang)) @ h_hat / n


def level(h: np.ndarray, k: int) -> np.ndarray:
    """Time-domain filter at resolution level k: 2^k h[2^k t]."""
    return (2 ** k) * h[:: 2 ** k]


def circ_conv(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Direct circular convolution along the last axis of x (any leading shape)."""
    n = x.shape[-1]
    assert h.shape[0] == n
    idx = (np.arange(n)[:, None] - np.arange(n)[None, :]) % n   # [t, s] -> t - s
    H = h[idx]                                                   # H[t, s] = h[t - s]
    return x @ H.T


def _along(a: np.ndarray, axis: int, fn) -> np.ndarray:
    return np.moveaxis(fn(np.moveaxis(a, axis, -1)), -1, axis)


def subsampling(xi: float, sigma: float) -> int:
    """Reading R2 by counting: double the band edge xi + 3 sigma while it stays <= 1/2."""
    edge, k = xi + 3.0 * sigma, 0
    while 2.0 * edge <= 0.5:
        edge *= 2.0
        k += 1
    return k


def _log2_floor(v: int) -> int:
    k = 0
    while (2 << k) <= v:
        k += 1
    return k


def schedule(plan: Plan) -> Dict:
    """Strides and row sets of the multirate schedule (readings R2, R3, R7, R8, R10, R21)."""
    lT, lF = _log2_floor(plan.T), _log2_floor(plan.F)
    j1 = [subsampling(f.xi, f.sigma) for f in plan.psi1]
    j2 = [subsampling(f.xi, f.sigma) for f in plan.psi2]
    jfr = [subsampling(f.xi, f.sigma) for f in plan.psi_fr]
    sig_phiF = 0.1 / plan.F
    jphiF = subsampling(0.0, sig_phiF)
    nfr = 1
    while nfr < len(plan.psi1) + 2 ** (plan.J_fr + 1):
        nfr *= 2
    kfr = (lambda j: min(j, lF)) if plan.average_local_fr else (lambda j: j)
    phi = (0.0, sig_phiF, kfr(jphiF))
    plus = [(f.xi, f.sigma, kfr(j)) for f, j in zip(plan.psi_fr, jfr)]
    minus = [(-f.xi, f.sigma, kfr(j)) for f, j in zip(plan.psi_fr, jfr)]
    rows2 = [[n1 for n1 in range(len(j1)) if j1[n1] < jj] for jj in j2]
    return {
        "lT": lT, "lF": lF, "N_fr": nfr, "sigma_phiT": 0.1 / plan.T, "sigma_phiF": sig_phiF,
        "j1": j1, "j2": j2,
        "k1": [min(j, lT) for j in j1],                                     # first order (R7)
        "k1_2": [min(j, lT) if plan.average_local else j for j in j1],     # rows feeding the second order
        "s2": [min(j, lT) if plan.average_local else j for j in j2],       # second order total stride
        "rows2": rows2, "active": [n2 for n2, r in enumerate(rows2) if r],
        "beta_first": [phi] + plus, "beta_second": [phi] + plus + minus,
    }


def jtfs_bruteforce(x: np.ndarray, plan: Plan, keep: bool = False) -> Dict[str, np.ndarray]:
    """Phi of x [N] or [B, N] by direct convolution; returns {'phi': [B, size]}."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    B, N = x.shape
    sch = schedule(plan)
    lT, lF, Nfr = sch["lT"], sch["lF"], sch["N_fr"]
    phiT = idft_explicit(_morlet(N, 0.0, sch["sigma_phiT"]))
    phiF = idft_explicit(_morlet(Nfr, 0.0, sch["sigma_phiF"]))

    # Unpooled variants (reading R21): plan.average_local / plan.average_local_fr.
    S0 = circ_conv(x.astype(np.complex128), phiT).real[:, :: 2 ** lT] if plan.average_local else x.copy()

    U1: List[np.ndarray] = []
    U1_2: List[np.ndarray] = []
    for n1, f in enumerate(plan.psi1):
        h = idft_explicit(_morlet(N, f.xi, f.sigma))
        full = circ_conv(x.astype(np.complex128), h)
        U1.append(np.abs(full[:, :: 2 ** sch["k1"][n1]]))
        U1_2.append(np.abs(full[:, :: 2 ** sch["k1_2"][n1]]))

    S1 = np.stack([
        circ_conv(U1[n1].astype(np.complex128), level(phiT, k1)).real[:, :: 2 ** (lT - k1)]
        for n1, k1 in enumerate(sch["k1"])], axis=1)                   # [B, N1, N/T]

    def freq_path(Z: np.ndarray, xi_b: float, sig_b: float, k_b: int) -> np.ndarray:
        """|Z *_n1 psi_beta| decimated, then *_n1 phi_F decimated; Z [B, N_fr, L]."""
        hb = idft_explicit(_morlet(Nfr, xi_b, sig_b))
        y = _along(Z, 1, lambda a: circ_conv(a, hb))[:, :: 2 ** k_b, :]
        u = np.abs(y)
        if not plan.average_local_fr:
            return u
        v = _along(u.astype(np.complex128), 1, lambda a: circ_conv(a, level(phiF, k_b))).real
        return v[:, :: 2 ** (lF - k_b), :]

    S1p = np.zeros((B, Nfr, S1.shape[2]), dtype=np.complex128)
    S1p[:, : len(plan.psi1)] = S1
    Phi1 = np.concatenate([freq_path(S1p, *b) for b in sch["beta_first"]], axis=1)

    blocks = []
    for n2 in sch["active"]:
        f2 = plan.psi2[n2]
        s2 = sch["s2"][n2]
        h2 = idft_explicit(_morlet(N, f2.xi, f2.sigma))
        rows = []
        for n1 in sch["rows2"][n2]:
            k1 = sch["k1_2"][n1]
            rows.append(circ_conv(U1_2[n1].astype(np.complex128), level(h2, k1))[:, :: 2 ** (s2 - k1)])
        Y2 = np.stack(rows, axis=1)
        Y2p = np.zeros((B, Nfr, Y2.shape[2]), dtype=np.complex128)
        Y2p[:, : Y2.shape[1]] = Y2
        per_beta = []
        for xi_b, sig_b, k_b in sch["beta_second"]:
            hb = idft_explicit(_morlet(Nfr, xi_b, sig_b))
            y = _along(Y2p, 1, lambda a: circ_conv(a, hb))[:, :: 2 ** k_b, :]
            a = np.abs(y)
            if plan.average_local:
                a = circ_conv(a.astype(np.complex128), level(phiT, s2)).real[:, :, :: 2 ** (lT - s2)]   # *_t phi_T
            if plan.average_local_fr:
                a = _along(a.astype(np.complex128), 1,
                           lambda z: circ_conv(z, level(phiF, k_b))).real[:, :: 2 ** (lF - k_b), :]
            per_beta.append(a)
        blocks.append(np.concatenate(per_beta, axis=1))

    parts = [S0, Phi1.reshape(B, -1)] + [blk.reshape(B, -1) for blk in blocks]
    out = {"phi": np.concatenate(parts, axis=1)}
    if keep:
        out.update(S0=S0, U1=U1, S1=S1, Phi1=Phi1)
    return out
