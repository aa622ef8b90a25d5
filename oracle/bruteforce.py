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

Filter construction (Eq. (1), §3.1) and the schedule follow the same
readings as ``jtfs_oracle`` and are retyped here on purpose.
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


def jtfs_bruteforce(x: np.ndarray, plan: Plan, keep: bool = False) -> Dict[str, np.ndarray]:
    """Phi of x [N] or [B, N] by direct convolution; returns {'phi': [B, size]}."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    B, N = x.shape
    lT, lF, Nfr = plan.lT, plan.lF, plan.N_fr
    phiT = idft_explicit(_morlet(N, 0.0, plan.sigma_phiT))
    phiF = idft_explicit(_morlet(Nfr, 0.0, plan.sigma_phiF))

    # Unpooled variants (reading R21): plan.average_local / plan.average_local_fr.
    S0 = circ_conv(x.astype(np.complex128), phiT).real[:, :: 2 ** lT] if plan.average_local else x.copy()

    U1: List[np.ndarray] = []
    U1_2: List[np.ndarray] = []
    for n1, f in enumerate(plan.psi1):
        h = idft_explicit(_morlet(N, f.xi, f.sigma))
        full = circ_conv(x.astype(np.complex128), h)
        U1.append(np.abs(full[:, :: 2 ** plan.k1[n1]]))
        U1_2.append(np.abs(full[:, :: 2 ** (plan.k1[n1] if plan.average_local else f.j)]))

    S1 = np.stack([
        circ_conv(U1[n1].astype(np.complex128), level(phiT, k1)).real[:, :: 2 ** (lT - k1)]
        for n1, k1 in enumerate(plan.k1)], axis=1)                     # [B, N1, N/T]

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
    S1p[:, : plan.N1] = S1
    Phi1 = np.concatenate([freq_path(S1p, *b) for b in plan.beta_first], axis=1)

    blocks = []
    for n2 in plan.active:
        f2 = plan.psi2[n2]
        s2 = min(f2.j, lT) if plan.average_local else f2.j
        h2 = idft_explicit(_morlet(N, f2.xi, f2.sigma))
        rows = []
        for n1 in range(plan.n1_max[n2]):
            k1 = plan.k1[n1] if plan.average_local else plan.psi1[n1].j
            rows.append(circ_conv(U1_2[n1].astype(np.complex128), level(h2, k1))[:, :: 2 ** (s2 - k1)])
        Y2 = np.stack(rows, axis=1)
        Y2p = np.zeros((B, Nfr, Y2.shape[2]), dtype=np.complex128)
        Y2p[:, : Y2.shape[1]] = Y2
        per_beta = []
        for xi_b, sig_b, k_b in plan.beta_second:
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
