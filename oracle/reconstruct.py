"""FP64 oracle: the paper's own reconstruction variant (§2.3).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.  The product path
never imports this module.

§2.3 reconstructs a signal from its JTFS by gradient descent that starts from
coloured Gaussian noise whose power spectral density follows the target's
first-order scattering S1x(t, lambda), and refines it by additive momentum
updates whose step size follows the "bold driver" heuristic.  The paper gives
neither construction in formulas; the readings taken here are

  R18 Coloured initialisation.  With the first-layer operators of §3.2,
      Psi_l w = decimate_{k1}(w * psi_l)  (complex, at the U1 rate of band l)
      and the phi_T pooling P_l u = decimate_{lT-k1}(u * phi_T) that turns U1
      into S1 (Eq. (4)), the initial signal is

        y~ = sum_l c_l Psi_l^T ( A_l . Psi_l w ),  A_l = 2^(lT-k1) P_l^T S1x(., l),
        y0 = y~ * ||x|| / ||y~||   (y0 = 0 when y~ = 0),

      where w is white Gaussian noise (drawn by the caller), ^T is the real
      adjoint, A_l is the target's S1 envelope interpolated back to the U1
      rate (the scaled adjoint of the pooling is an interpolation: a constant
      envelope comes back as the same constant), and
      c_l = 2^(k1+1) / sqrt(mean_m psi_hat_l(m)^6) makes the band-l term of
      y~ have E|Psi_l y~|^2 = A_l^2 for a slowly varying A_l.  y~ is linear in
      w, so y0 is Gaussian given the target; its local power in band l is
      proportional to A_l^2 = S1x^2.  The final scale matches the target's
      energy.
  R19 Momentum with bold driver (reading of the recursion printed in §2.3,
      whose u_n appears on both sides and whose sign is ambiguous):
        u_n = m u_{n-1} - mu_n grad E(y_n),  y_{n+1} = y_n + u_n,  m = 0.9,
      mu_0 = 0.1.  At each evaluation, per clip: if E(y_n) <= E_acc (the loss
      at the last accepted point; +inf before the first) the point is
      accepted, mu grows by 1.1 (except at the first evaluation), E_acc and
      the stored gradient take the new values and the momentum step is taken.
      Otherwise (E increased, or is NaN) the point is rejected: mu halves,
      y returns to the last accepted point, the momentum is reset and a plain
      step -mu * (gradient at the accepted point) is taken from there.
"""

from __future__ import annotations

import math
from typing import Dict

import numpy as np
import torch

from .jtfs_oracle import C128, F64, Plan, conv_circ, decimate, gauss_hat, morlet_hat, periodise

GROW = 1.1     # bold driver: step-size factor after a decrease (R19)
SHRINK = 0.5   # bold driver: step-size factor after an increase (R19)


# ---------------------------------------------------------------------------
# First-layer operators of §3.2 and their adjoints
# ---------------------------------------------------------------------------

def zero_insert(z: torch.Tensor, k: int) -> torch.Tensor:
    """Adjoint of ``decimate`` by 2^k along the last axis: samples at multiples of 2^k."""
    if k == 0:
        return z
    out = torch.zeros(z.shape[:-1] + (z.shape[-1] << k,), dtype=z.dtype)
    out[..., ::2 ** k] = z
    return out


def analysis(w: torch.Tensor, plan: Plan, n1: int) -> torch.Tensor:
    """Psi_l w = decimate_{k1}(w * psi_l): band n1 of the first layer before the modulus (§3.2)."""
    f = plan.psi1[n1]
    z = torch.fft.ifft(torch.fft.fft(w.to(C128), dim=-1) * morlet_hat(plan.N, f.xi, f.sigma), dim=-1)
    return decimate(z, plan.k1[n1], -1)


def synthesis(g: torch.Tensor, plan: Plan, n1: int) -> torch.Tensor:
    """Real adjoint Psi_l^T g = Re(zero_insert(g) correlated with psi_l) (transpose of ``analysis``)."""
    f = plan.psi1[n1]
    G = torch.fft.fft(zero_insert(g.to(C128), plan.k1[n1]), dim=-1)
    return torch.fft.ifft(G * morlet_hat(plan.N, f.xi, f.sigma).conj(), dim=-1).real


def pool_T(u: torch.Tensor, plan: Plan, n1: int) -> torch.Tensor:
    """S1 row of band n1 from its U1 row: phi_T at the U1 rate, decimated to stride T (Eq. (4))."""
    k1 = plan.k1[n1]
    h = periodise(gauss_hat(plan.N, plan.sigma_phiT), k1)
    return decimate(conv_circ(u.to(C128), h, -1), plan.lT - k1, -1).real


def pool_T_adjoint(s: torch.Tensor, plan: Plan, n1: int) -> torch.Tensor:
    """Transpose of ``pool_T``: zero insertion to the U1 rate, then correlation with phi_T."""
    k1 = plan.k1[n1]
    h = periodise(gauss_hat(plan.N, plan.sigma_phiT), k1)
    return conv_circ(zero_insert(s.to(C128), plan.lT - k1), h.conj(), -1).real


def band_gain(plan: Plan, n1: int) -> float:
    """c_l = 2^(k1+1) / sqrt(mean_m psi_hat_l(m)^6) (R18)."""
    f = plan.psi1[n1]
    p = morlet_hat(plan.N, f.xi, f.sigma)
    return 2.0 ** (plan.k1[n1] + 1) / math.sqrt(float((p ** 6).mean()))


# ---------------------------------------------------------------------------
# Coloured initialisation (§2.3, R18)
# ---------------------------------------------------------------------------

def first_order(x: torch.Tensor, plan: Plan) -> torch.Tensor:
    """S1x [B, N1, N/T] = P_l |Psi_l x| (§3.2 then Eq. (4))."""
    x = x.to(F64).reshape(-1, plan.N)
    return torch.stack([pool_T(analysis(x, plan, n1).abs(), plan, n1) for n1 in range(plan.N1)], 1)


def envelope(S1: torch.Tensor, plan: Plan, n1: int) -> torch.Tensor:
    """A_l = 2^(lT-k1) P_l^T S1(., l): the S1 row interpolated to the U1 rate (R18)."""
    return 2.0 ** (plan.lT - plan.k1[n1]) * pool_T_adjoint(S1[:, n1], plan, n1)


def coloured_init(x: torch.Tensor, w: torch.Tensor, plan: Plan, raw: bool = False) -> torch.Tensor:
    """Initial signal y0 [B, N] of the reconstruction (R18) from target x and white noise w.

    With ``raw`` the unscaled y~ is returned (linear in w).
    """
    x = x.to(F64).reshape(-1, plan.N)
    w = w.to(F64).reshape(-1, plan.N)
    S1 = first_order(x, plan)
    y = torch.zeros_like(w)
    for n1 in range(plan.N1):
        g = envelope(S1, plan, n1) * analysis(w, plan, n1)
        y = y + band_gain(plan, n1) * synthesis(g, plan, n1)
    if raw:
        return y
    nx = x.norm(dim=-1, keepdim=True)
    ny = y.norm(dim=-1, keepdim=True)
    return torch.where(ny > 0, y * nx / torch.where(ny > 0, ny, torch.ones_like(ny)), torch.zeros_like(y))


# ---------------------------------------------------------------------------
# Momentum descent with the bold-driver step size (§2.3, R19)
# ---------------------------------------------------------------------------

def bold_driver_step(y: np.ndarray, u: np.ndarray, g_acc: np.ndarray, mu: np.ndarray, E_acc: np.ndarray,
                     E: np.ndarray, g: np.ndarray, m: float = 0.9) -> Dict[str, np.ndarray]:
    """One update of every clip (arrays [B, N] and [B]); E, g are E(y) and grad E(y).

    Returns the new y, u, g_acc, mu, E_acc and the per-clip accept flags.
    """
    y, u, g_acc = (np.array(a, dtype=np.float64, copy=True) for a in (y, u, g_acc))
    mu, E_acc = (np.array(a, dtype=np.float64, copy=True) for a in (mu, E_acc))
    E = np.asarray(E, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    accepted = np.zeros(len(E), dtype=bool)
    for b in range(len(E)):
        if E[b] <= E_acc[b]:                       # no increase: accept y_n
            accepted[b] = True
            if math.isfinite(E_acc[b]):
                mu[b] *= GROW
            E_acc[b] = E[b]
            g_acc[b] = g[b]
            u[b] = m * u[b] - mu[b] * g[b]
        else:                                      # increase: reject y_n
            mu[b] *= SHRINK
            y[b] -= u[b]                           # back to the accepted point
            u[b] = -mu[b] * g_acc[b]               # momentum reset
        y[b] += u[b]
    return {"y": y, "u": u, "g_acc": g_acc, "mu": mu, "E_acc": E_acc, "accepted": accepted}
