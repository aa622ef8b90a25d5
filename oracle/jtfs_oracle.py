"""FP64 oracle: joint time-frequency scattering, JTFS loss and its gradient.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.  The product path
never imports this module.

What it computes (Lostanlen & Han, "Musical Metamerism with Time-Frequency
Scattering"):

* Filterbanks: the generator of §3.1 (constant-Q progression down to an
  elbow, then Q-1 constant-bandwidth filters), used for the first-order time
  filters (J, Q), the second-order time filters (J, Q2) and the frequential
  filters (J_fr, Q_fr), the latter spun to +xi and -xi (§3.4).
* Morlet wavelets of Eq. (1) in the Fourier domain, with the corrective term
  kappa giving a null average; Gaussian low-pass phi_T, phi_F (§2.1, §2.2).
* The multirate schedule of §3.2-§3.5: first layer U1 = |x * psi| at stride
  2^k1 (§3.2), width-first second layer over n2 then n1 (§3.3), frequential
  scattering along n1 with zero padding to N_fr (§3.4), the order of yielded
  paths of the main algorithm (§3.5), and Gaussian averaging in time and
  log-frequency after the modulus, Eqs. (4)-(5).
* Loss E = ||Phi(y) - Phi(x)||^2 (§1.2, §2.3) and its gradient by
  reverse-mode automatic differentiation, the route §2.3 describes
  (Eqs. (6)-(8) are the structure autograd realises).

Route: every filtering step is a circular convolution evaluated as
ifft(fft(z) * h_hat) (a library FFT as a step) followed by time-domain
decimation z[::2^k].  The CUDA path instead decimates in the Fourier domain
(periodisation) with band-limited alias sums; the two agree because
periodising a spectrum by 2^k is exactly decimating the signal by 2^k.

Readings of passages that are silent or ambiguous (each is listed with its
reason in the repository's design notes):
  R1  listing §3.1 uses an undefined ``r``: read as r_psi = sqrt(1/2).
  R2  filter field 'j' (§3.2-§3.4) is undefined: j = max(0, floor(log2(
      0.5 / (xi + 3 sigma)))), the largest dyadic subsampling that keeps
      xi + 3 sigma below the new Nyquist frequency.
  R3  phi_T has sigma = sigma0 / T cycles/sample and phi_F has
      sigma = sigma0 / F cycles/bin; output strides are T in time and
      2^floor(log2 F) along n1.
  R4  Filters are sampled in the Fourier domain at omega_m = m/n for
      m < n/2 and (m - n)/n otherwise (the Nyquist bin is -1/2); peak value
      1 before the kappa correction; no periodisation at full rate.
  R5  levels[k] of a filter = its full-rate spectrum periodised onto n/2^k
      bins (sum of the 2^k aliases).
  R6  subsample_fourier = exact time-domain decimation (keep every 2^k-th
      sample, starting at sample 0).
  R7  k1 = min(j1, log2 T); second order keeps rows with j1 < j2 at total
      stride s2 = min(j2, log2 T), i.e. k2 = s2 - k1; frequential stride
      k_fr = min(j_fr, floor(log2 F)).
  R8  N_fr = next power of two >= N1 + 2^(J_fr + 1); rows zero-padded on the
      right; all N_fr / 2^floor(log2 F) pooled rows are kept.
  R9  Time boundary: periodic (power-of-two N, no padding).
  R10 Frequential filter set: first order {phi_F} + {+xi_n}; second order
      {phi_F} + {+xi_n} + {-xi_n}; phi_F is the beta = 0 member.
  R11 First-order frequential paths: |S1 *_n1 psi_beta| *_n1 phi_F
      (S1 = U1 *_t phi_T already at stride T).  Second-order paths:
      |U1 *_t psi_alpha *_n1 psi_beta| *_t phi_T *_n1 phi_F.
  R12 Phi layout per clip: S0 [N/T]; first order [1+K][R_out][N/T];
      second order per active n2 ascending [1+2K][R_out][N/T].
  R13 E = sum over all Phi entries of (Phi(y) - Phi(x))^2; modulus
      derivative at 0 is 0 (torch's convention for |z|).
  R15 Clips whose length L is not a power of two: zero-padded on the right
      to the next power of two, Phi computed there, and only the first
      ceil(L/T) frames of each row kept (the crop's adjoint fills zeros).
  R21 Unpooled outputs (average_local / average_local_fr of §3.3-§3.5 set
      to False).  average_local = False: the zeroth-order output is U0 = x
      at full rate; the rows U1 that feed the second order are taken at
      stride k1 = j1 and the second order at total stride j2 (k2 = j2 - k1,
      §3.3), with no phi_T averaging of |Y2_fr|; the first order keeps S1 at
      stride T (the main algorithm scatters S1 along n1, which needs one
      time grid).  average_local_fr = False: frequential stride k = j_fr for
      every beta (phi_F included, §3.4) and no phi_F averaging: each beta
      yields N_fr / 2^k rows of |Y_fr|.  Outputs are concatenated in the
      path order of R12, rows per beta, then frames.
  R20 Reflect boundary (the padding "on both sides" of §3.2 as an option):
      P = ceil(sqrt(ln(1000) / 2) / (pi sigma_min)) samples per side, the
      half-width beyond which the slowest time envelope exp(-2 pi^2 sigma^2
      t^2) among psi1, psi2 and phi_T is below 1e-3 of its peak; padded
      length n = next power of two >= L + 2P; left pad p0 = T floor((n - L) /
      (2T)) (frames stay on the stride-T grid), the rest on the right; the
      padding mirrors the clip without repeating its edge samples (x[-t] =
      x[t], x[L-1+t] = x[L-1-t], repeated with period 2(L-1)); Phi is
      computed on the padded clip and the ceil(L/T) frames starting at
      frame p0 / T are kept.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import torch

SIGMA0 = 0.1                 # §3.1 listing: sigma0
R_PSI = math.sqrt(0.5)       # §3.1 listing: r_psi (reading R1)
F64 = torch.float64
C128 = torch.complex128


# ---------------------------------------------------------------------------
# Filterbank design (§3.1)
# ---------------------------------------------------------------------------

def morlet_filterbank(J: int, Q: int) -> List[Tuple[float, float]]:
    """(xi, sigma) of the filterbank §3.1 generates, highest centre frequency first.

    Written from what the generator computes, not from its loop:

    * Constant-Q part.  The first centre frequency is xi_0 = max(1/(1 + 2^(3/Q)),
      0.35).  Neighbours sit a factor f = 2^(-1/Q) apart, and the width is the
      one at which a filter and its lower neighbour (width scaled by f too)
      have both fallen to r_psi where they meet:
          xi_0 - c sigma_0 = f (xi_0 + c sigma_0),   c = sqrt(2 ln(1/r_psi)),
      so sigma_0 = (1 - f) / (1 + f) * xi_0 / c.  Filter k has
      (xi_0 f^k, sigma_0 f^k); k runs from 0 to K, K being the number of
      k >= 0 whose width sigma_0 f^k still exceeds sigma_min / f, with
      sigma_min = sigma_0' / 2^J the elbow width (sigma_0' = 0.1 of §3.1).
    * Constant-bandwidth part.  Below the elbow xi_e = xi_0 f^K, Q - 1 filters
      of width sigma_min at xi_e (1 - m/Q), m = 1 .. Q - 1.
    * If sigma_0 <= sigma_min there is no constant-Q part and xi_e = sigma_0
      (the generator's literal branch, reading of §3.1).
    """
    f = math.pow(2.0, -1.0 / Q)
    xi0 = max(1.0 / (1.0 + math.pow(2.0, 3.0 / Q)), 0.35)
    c = math.sqrt(2.0 * math.log(1.0 / R_PSI))
    sigma0 = (1.0 - f) / (1.0 + f) * xi0 / c
    sigma_min = SIGMA0 / 2 ** J
    if sigma0 <= sigma_min:
        constant_q: List[Tuple[float, float]] = []
        xi_elbow = sigma0
    else:
        K = 0
        while sigma0 * math.pow(f, K) > sigma_min / f:
            K += 1
        constant_q = [(xi0 * math.pow(f, k), sigma0 * math.pow(f, k)) for k in range(K + 1)]
        xi_elbow = constant_q[-1][0]
    constant_bw = [(xi_elbow * (1.0 - m / Q), sigma_min) for m in range(1, Q)]
    return constant_q + constant_bw


def max_subsampling(xi: float, sigma: float) -> int:
    """Filter field 'j' (reading R2): largest k with 2^k (xi + 3 sigma) <= 1/2."""
    return max(0, int(math.floor(math.log2(0.5 / (xi + 3.0 * sigma)))))


def _next_pow2(n: int) -> int:
    return 1 << (int(n) - 1).bit_length()


@dataclass
class Filter:
    xi: float
    sigma: float
    j: int


@dataclass
class Plan:
    """Filterbanks and multirate schedule of one JTFS configuration."""

    N: int
    J: int
    Q: int
    Q2: int
    J_fr: int
    Q_fr: int
    T: int
    F: int
    average_local: bool = True
    average_local_fr: bool = True
    psi1: List[Filter] = field(init=False)
    psi2: List[Filter] = field(init=False)
    psi_fr: List[Filter] = field(init=False)

    def __post_init__(self) -> None:
        if self.N <= 0 or self.N & (self.N - 1):
            raise ValueError("N must be a power of two")
        if self.T <= 0 or self.T & (self.T - 1) or self.T > self.N:
            raise ValueError("T must be a power of two <= N")
        if self.F < 1:
            raise ValueError("F must be >= 1")
        self.lT = self.T.bit_length() - 1
        self.lF = int(math.floor(math.log2(self.F)))
        self.psi1 = [Filter(x, s, max_subsampling(x, s)) for x, s in morlet_filterbank(self.J, self.Q)]
        self.psi2 = [Filter(x, s, max_subsampling(x, s)) for x, s in morlet_filterbank(self.J, self.Q2)]
        self.psi_fr = [Filter(x, s, max_subsampling(x, s)) for x, s in morlet_filterbank(self.J_fr, self.Q_fr)]
        self.sigma_phiT = SIGMA0 / self.T
        self.sigma_phiF = SIGMA0 / self.F
        self.j_phiT = max_subsampling(0.0, self.sigma_phiT)
        self.j_phiF = max_subsampling(0.0, self.sigma_phiF)
        self.N1 = len(self.psi1)
        self.K = len(self.psi_fr)
        self.N_fr = _next_pow2(self.N1 + 2 ** (self.J_fr + 1))
        if (1 << self.lF) > self.N_fr:
            raise ValueError("2^floor(log2 F) exceeds the frequential length")
        self.k1 = [min(f.j, self.lT) for f in self.psi1]
        self.n1_max = [sum(1 for f1 in self.psi1 if f1.j < f2.j) for f2 in self.psi2]
        self.active = [n2 for n2 in range(len(self.psi2)) if self.n1_max[n2] > 0]
        # Frequential filter sets (reading R10): (xi, sigma, k_fr); xi = 0 is phi_F.
        # Frequential strides capped at log2 F unless the output is unpooled (R21).
        kcap = (lambda j: min(j, self.lF)) if self.average_local_fr else (lambda j: j)
        phi = (0.0, self.sigma_phiF, kcap(self.j_phiF))
        plus = [(f.xi, f.sigma, kcap(f.j)) for f in self.psi_fr]
        minus = [(-f.xi, f.sigma, kcap(f.j)) for f in self.psi_fr]
        self.beta_first = [phi] + plus
        self.beta_second = [phi] + plus + minus
        self.R_out = self.N_fr >> self.lF
        self.n_frames = self.N >> self.lT
        # Time strides of the rows feeding the second order and of the second order (R7, R21).
        self.k1_2 = [min(f.j, self.lT) if self.average_local else f.j for f in self.psi1]
        self.s2 = [min(f.j, self.lT) if self.average_local else f.j for f in self.psi2]

    def rows(self, beta: Tuple[float, float, int]) -> int:
        """Rows n1 of one frequential path: R_out pooled, else N_fr / 2^k (R21)."""
        return self.R_out if self.average_local_fr else self.N_fr >> beta[2]

    def frames2(self, n2: int) -> int:
        """Time frames of the second-order paths of n2: N/T pooled, else N / 2^j2 (R21)."""
        return self.n_frames if self.average_local else self.N >> self.s2[n2]

    @property
    def phi_size(self) -> int:
        """Floats per clip in the flat Phi vector (readings R12, R21)."""
        s0 = self.n_frames if self.average_local else self.N
        first = sum(self.rows(b) for b in self.beta_first) * self.n_frames
        second = sum(sum(self.rows(b) for b in self.beta_second) * self.frames2(n2) for n2 in self.active)
        return s0 + first + second


# ---------------------------------------------------------------------------
# Fourier-domain filters (Eq. (1); §2.1-§2.2)
# ---------------------------------------------------------------------------

def fourier_grid(n: int) -> torch.Tensor:
    """omega_m in cycles per sample on [-1/2, 1/2) (reading R4)."""
    m = torch.arange(n, dtype=F64)
    return torch.where(m < n / 2, m, m - n) / n


def morlet_hat(n: int, xi: float, sigma: float) -> torch.Tensor:
    """Morlet wavelet of Eq. (1) in the Fourier domain, sampled on n bins.

    psi_hat(w) = exp(-(w - xi)^2 / 2 sigma^2) - kappa exp(-w^2 / 2 sigma^2),
    kappa = exp(-xi^2 / 2 sigma^2), so psi_hat(0) = 0 (one vanishing moment).
    """
    w = fourier_grid(n)
    kappa = math.exp(-xi * xi / (2.0 * sigma * sigma))
    return torch.exp(-(w - xi) ** 2 / (2.0 * sigma * sigma)) - kappa * torch.exp(-w * w / (2.0 * sigma * sigma))


def gauss_hat(n: int, sigma: float) -> torch.Tensor:
    """Gaussian low-pass phi_hat(w) = exp(-w^2 / 2 sigma^2) on n bins."""
    w = fourier_grid(n)
    return torch.exp(-w * w / (2.0 * sigma * sigma))


def freq_filter_hat(n: int, xi: float, sigma: float) -> torch.Tensor:
    """Frequential filter: phi_F when xi == 0, else the (spun) Morlet."""
    return gauss_hat(n, sigma) if xi == 0.0 else morlet_hat(n, xi, sigma)


def periodise(h_hat: torch.Tensor, k: int) -> torch.Tensor:
    """levels[k] (reading R5): sum of the 2^k aliases onto n / 2^k bins."""
    n = h_hat.shape[-1]
    return h_hat.reshape(2 ** k, n >> k).sum(0)


# ---------------------------------------------------------------------------
# Multirate primitives
# ---------------------------------------------------------------------------

def decimate(z: torch.Tensor, k: int, dim: int) -> torch.Tensor:
    """Keep every 2^k-th sample along ``dim``, starting at 0 (reading R6)."""
    if k == 0:
        return z
    idx = torch.arange(0, z.shape[dim], 2 ** k)
    return z.index_select(dim, idx)


def conv_circ(z: torch.Tensor, h_hat: torch.Tensor, dim: int) -> torch.Tensor:
    """Circular convolution along ``dim`` with the filter whose DFT is h_hat."""
    shape = [1] * z.dim()
    shape[dim] = h_hat.shape[0]
    return torch.fft.ifft(torch.fft.fft(z, dim=dim) * h_hat.reshape(shape), dim=dim)


def pad_rows(z: torch.Tensor, n: int, dim: int) -> torch.Tensor:
    """Zero-pad ``dim`` on the right to length n (§3.4 listing, pad_frequency)."""
    extra = n - z.shape[dim]
    if extra <= 0:
        return z
    shape = list(z.shape)
    shape[dim] = extra
    return torch.cat([z, torch.zeros(shape, dtype=z.dtype)], dim=dim)


# ---------------------------------------------------------------------------
# The transform
# ---------------------------------------------------------------------------

def jtfs(x: torch.Tensor, plan: Plan, keep: bool = False,
         checkpoint_blocks: bool = False, active: Optional[Sequence[int]] = None) -> Dict[str, torch.Tensor]:
    """JTFS of x [B, N] (float64).  Returns {'phi': [B, phi_size], ...}.

    With ``keep`` the intermediates U1 (list over n1), S1 and Y2 (list over
    active n2) are returned too.  ``checkpoint_blocks`` recomputes each
    second-order block in the backward pass instead of storing it (same
    arithmetic; only bounds autograd memory for long signals).  ``active``
    (positions in ``plan.active``) restricts the second order to those paths:
    the result then has S0, Phi1 and {'Phi2_sel': {position: [B, 1+2K, R_out, N/T]}}
    instead of 'phi' (for sampling long signals).
    """
    if x.dim() == 1:
        x = x[None]
    B, N = x.shape
    assert N == plan.N
    lT, lF = plan.lT, plan.lF
    X = torch.fft.fft(x.to(C128), dim=-1)
    phiT = gauss_hat(N, plan.sigma_phiT)
    phiF = gauss_hat(plan.N_fr, plan.sigma_phiF)

    # Zeroth order: x * phi_T at stride T (first yield of the main algorithm), or x itself (R21).
    if plan.average_local:
        S0 = decimate(torch.fft.ifft(X * phiT, dim=-1).real, lT, -1)
    else:
        S0 = x.to(F64)

    # First layer (§3.2): U1 = |x * psi_n1| at stride 2^k1; the second order reads
    # its rows at stride 2^k1_2 (equal to k1 unless unpooled in time, R21).
    U1, U1_2 = [], []
    for f, k1, k12 in zip(plan.psi1, plan.k1, plan.k1_2):
        z = torch.fft.ifft(X * morlet_hat(N, f.xi, f.sigma), dim=-1)
        U1.append(decimate(z, k1, -1).abs())
        U1_2.append(U1[-1] if k12 == k1 else decimate(z, k12, -1).abs())

    # First-order time averaging, S_1 of the main algorithm (§3.5), Eq. (4)'s phi_T.
    S1 = torch.stack([
        decimate(conv_circ(U1[n1], periodise(phiT, k1), -1), lT - k1, -1).real
        for n1, k1 in enumerate(plan.k1)], dim=1)                         # [B, N1, N/T]

    # First-order frequential scattering (spinned=False, §3.4) then phi_F averaging.
    def pool_F(u: torch.Tensor, k_b: int) -> torch.Tensor:
        """*_n1 phi_F decimated to 2^lF (Eq. (5)), or the rows as they are (unpooled, R21)."""
        if not plan.average_local_fr:
            return u
        return decimate(conv_circ(u, periodise(phiF, k_b), 1), lF - k_b, 1).real

    def join(blocks: List[torch.Tensor]) -> torch.Tensor:
        """[B, paths, R_out, frames] when every path has R_out rows, else rows concatenated."""
        return torch.stack(blocks, 1) if plan.average_local_fr else torch.cat(blocks, 1)

    S1p = pad_rows(S1, plan.N_fr, 1)
    phi1 = []
    for xi_b, sig_b, k_b in plan.beta_first:
        yfr = decimate(conv_circ(S1p, freq_filter_hat(plan.N_fr, xi_b, sig_b), 1), k_b, 1)
        phi1.append(pool_F(yfr.abs(), k_b))
    Phi1 = join(phi1)                                                    # [B, 1+K, R_out, N/T]

    def second_order_block(U1_rows: List[torch.Tensor], n2: int) -> Tuple[torch.Tensor, torch.Tensor]:
        f2 = plan.psi2[n2]
        s2 = plan.s2[n2]
        psi2 = morlet_hat(N, f2.xi, f2.sigma)
        # Second layer, time variable (§3.3): rows n1 with j1 < j2, stacked.
        rows = []
        for n1 in range(plan.n1_max[n2]):
            k1 = plan.k1_2[n1]
            rows.append(decimate(conv_circ(U1_rows[n1], periodise(psi2, k1), -1), s2 - k1, -1))
        Y2 = torch.stack(rows, 1)                                        # [B, n1_max, N/2^s2]
        # Second layer, frequency variable (§3.4, spinned=True), modulus, Eq. (5).
        Y2p = pad_rows(Y2, plan.N_fr, 1)
        blocks = []
        for xi_b, sig_b, k_b in plan.beta_second:
            yfr = decimate(conv_circ(Y2p, freq_filter_hat(plan.N_fr, xi_b, sig_b), 1), k_b, 1)
            u2 = yfr.abs()
            if plan.average_local:
                u2 = decimate(conv_circ(u2, periodise(phiT, s2), 2), lT - s2, 2).real     # *_t phi_T
            blocks.append(pool_F(u2, k_b))                                           # *_n1 phi_F
        return join(blocks), Y2                                          # [B, 1+2K, R_out, N/T]

    if active is not None:
        sel = {int(a): second_order_block(U1_2, plan.active[int(a)])[0] for a in active}
        return {"S0": S0, "Phi1": Phi1, "Phi2_sel": sel}

    phi2, Y2s = [], []
    for n2 in plan.active:
        if checkpoint_blocks and torch.is_grad_enabled():
            from torch.utils.checkpoint import checkpoint
            blk = checkpoint(lambda *rows, _n2=n2: second_order_block(list(rows), _n2)[0],
                             *U1_2[:plan.n1_max[n2]], use_reentrant=False)
        else:
            blk, Y2 = second_order_block(U1_2, n2)
            if keep:
                Y2s.append(Y2)
        phi2.append(blk)

    parts = [S0, Phi1.reshape(B, -1)] + [blk.reshape(B, -1) for blk in phi2]
    out = {"phi": torch.cat(parts, 1)}
    if keep:
        pooled = plan.average_local and plan.average_local_fr
        out.update(S0=S0, U1=U1, S1=S1, Phi1=Phi1, Y2=Y2s,
                   Phi2=(torch.stack(phi2, 1) if phi2 else None) if pooled else phi2)
    return out


def second_order_frames(x: torch.Tensor, plan: Plan, a: int, frames: Sequence[int],
                        tail: float = 1e-13) -> torch.Tensor:
    """Second-order paths of active group ``a`` at the pooled frames ``frames`` only:
    [B, 1+2K, R_out, len(frames)], for clips too long for the whole transform (the
    un-pooled second order of a 2^20-sample clip is hundreds of GB).

    The same steps as ``jtfs`` for that group -- U1 rows with j1 < j2 (§3.2), Y2
    (§3.3), frequential filtering, modulus, phi_F (§3.4, Eq. (5)) -- with the
    phi_T average of Eq. (5) written as the sum it is at the kept frames:
        Phi[f] = sum_t g[(f D - t) mod L] u[t],   g = ifft(levels[s2] of phi_T),
    D = 2^(lT - s2), L = N / 2^s2, over the columns t where |g| exceeds ``tail``
    times its peak (the Gaussian's taps beyond are below it); only those columns
    are scattered along n1.  Pooled in time only (average_local and
    average_local_fr on).
    """
    if x.dim() == 1:
        x = x[None]
    assert plan.average_local and plan.average_local_fr
    B, N = x.shape
    n2 = plan.active[int(a)]
    f2 = plan.psi2[n2]
    s2, lT = plan.s2[n2], plan.lT
    L, D = N >> s2, 1 << (lT - s2)
    X = torch.fft.fft(x.to(C128), dim=-1)
    psi2 = morlet_hat(N, f2.xi, f2.sigma)
    rows = []
    for n1 in range(plan.n1_max[n2]):
        f, k1 = plan.psi1[n1], plan.k1_2[n1]
        u1 = decimate(torch.fft.ifft(X * morlet_hat(N, f.xi, f.sigma), dim=-1), k1, -1).abs()
        rows.append(decimate(conv_circ(u1, periodise(psi2, k1), -1), s2 - k1, -1))
    Y2 = torch.stack(rows, 1)                                            # [B, n1_max, L]
    g = torch.fft.ifft(periodise(gauss_hat(N, plan.sigma_phiT), s2).to(C128)).real
    lag = torch.nonzero(g.abs() > tail * g.abs().max()).flatten()        # lags (f D - t) mod L kept
    cols = torch.unique(torch.cat([(int(fr) * D - lag) % L for fr in frames]))
    Yc = pad_rows(Y2[:, :, cols], plan.N_fr, 1)                           # the columns that matter
    G = torch.stack([g[(int(fr) * D - cols) % L] for fr in frames], 1)   # [columns, frames]
    phiF = gauss_hat(plan.N_fr, plan.sigma_phiF)
    out = []
    for xi_b, sig_b, k_b in plan.beta_second:
        u = decimate(conv_circ(Yc, freq_filter_hat(plan.N_fr, xi_b, sig_b), 1), k_b, 1).abs()
        v = u @ G.to(u.dtype)                                             # *_t phi_T at the frames
        out.append(decimate(conv_circ(v.to(C128), periodise(phiF, k_b), 1), plan.lF - k_b, 1).real)
    return torch.stack(out, 1)


def phi_blocks(phi: torch.Tensor, plan: Plan) -> Dict[str, torch.Tensor]:
    """Split a flat [B, phi_size] Phi into S0, first-order and per-n2 blocks."""
    B = phi.shape[0]
    nf = plan.n_frames
    o = 0
    n = nf if plan.average_local else plan.N
    out = {"S0": phi[:, o:o + n]}
    o += n
    n = sum(plan.rows(b) for b in plan.beta_first) * nf
    out["first"] = phi[:, o:o + n]
    o += n
    for n2 in plan.active:
        n = sum(plan.rows(b) for b in plan.beta_second) * plan.frames2(n2)
        out[f"n2={n2}"] = phi[:, o:o + n]
        o += n
    assert o == phi.shape[1] == plan.phi_size and B == phi.shape[0]
    return out


def loss(y: torch.Tensor, phi_target: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Per-clip E(y) = ||Phi(y) - Phi_target||^2 (§1.2; reading R13)."""
    phi = jtfs(y, plan)["phi"]
    return ((phi - phi_target) ** 2).sum(-1)


def loss_and_grad(y: torch.Tensor, phi_target: torch.Tensor, plan: Plan,
                  checkpoint_blocks: bool = False) -> Tuple[torch.Tensor, torch.Tensor]:
    """(E [B], dE/dy [B, N]) by reverse-mode autodiff (§2.3)."""
    y = y.detach().to(F64)
    if y.dim() == 1:
        y = y[None]
    y = y.clone().requires_grad_(True)
    with torch.enable_grad():
        phi = jtfs(y, plan, checkpoint_blocks=checkpoint_blocks)["phi"]
        E = ((phi - phi_target.to(F64)) ** 2).sum(-1)
        (g,) = torch.autograd.grad(E.sum(), y)
    return E.detach(), g.detach()


# ---------------------------------------------------------------------------
# Clips of any length (reading R15): zero-pad on the right to the next power
# of two (the padding of §3.2 with a periodic boundary), compute Phi at that
# length, keep the first ceil(L / T) frames of every row.
# ---------------------------------------------------------------------------

def padded_length(L: int) -> int:
    """Next power of two >= L."""
    return _next_pow2(L)


def jtfs_uneven(y: torch.Tensor, params: Dict[str, int]) -> torch.Tensor:
    """Phi of one clip y [L] (any L >= 1): flat vector of rows x ceil(L/T) frames.

    Every Phi block is [..., frame] with n_frames = N_pad / T frames per row;
    the crop keeps frames [0, ceil(L/T)) of each row (S0 counts as one row).
    """
    L = y.shape[-1]
    plan = Plan(N=padded_length(max(L, params["T"])), **{k: v for k, v in params.items() if k != "N"})
    yp = torch.cat([y.reshape(1, L).to(F64), torch.zeros(1, plan.N - L, dtype=F64)], dim=1)
    phi = jtfs(yp, plan)["phi"].reshape(-1, plan.n_frames)
    nf = -(-L // plan.T)
    return phi[:, :nf].reshape(-1)


def loss_and_grad_uneven(y: torch.Tensor, phi_target: torch.Tensor,
                         params: Dict[str, int]) -> Tuple[torch.Tensor, torch.Tensor]:
    """E = ||Phi_cropped(y) - target||^2 and dE/dy for one clip of any length."""
    y = y.detach().to(F64).clone().requires_grad_(True)
    with torch.enable_grad():
        E = ((jtfs_uneven(y, params) - phi_target.to(F64)) ** 2).sum()
        (g,) = torch.autograd.grad(E, y)
    return E.detach(), g.detach()


# ---------------------------------------------------------------------------
# Reflect boundary (reading R20): pad on both sides by reflection, compute
# Phi on the padded clip, keep the frames over the clip (§3.2's padding and
# unpadding).
# ---------------------------------------------------------------------------

def reflect_pad_width(params: Dict[str, int]) -> int:
    """P of R20 from the filterbanks the parameters define (they do not depend on N)."""
    plan = Plan(**{**params, "N": max(params["T"], 2 ** (params["J"] + 1))})
    sig = min([f.sigma for f in plan.psi1] + [f.sigma for f in plan.psi2] + [plan.sigma_phiT])
    return int(math.ceil(math.sqrt(math.log(1000.0) / 2.0) / (math.pi * sig)))


def reflect_layout(L: int, params: Dict[str, int]) -> Tuple[int, int, int, int]:
    """(n, p0, first kept frame, kept frames) of a clip of L samples (R20)."""
    T = params["T"]
    n = _next_pow2(L + 2 * reflect_pad_width(params))
    p0 = T * ((n - L) // (2 * T))
    return n, p0, p0 // T, -(-L // T)


def reflect_index(u: torch.Tensor, L: int) -> torch.Tensor:
    """Index into a clip of L samples of position u relative to its first sample, mirrored (R20)."""
    if L == 1:
        return torch.zeros_like(u)
    per = 2 * (L - 1)
    r = torch.remainder(u, per)
    return torch.where(r < L, r, per - r)


def jtfs_reflect(y: torch.Tensor, params: Dict[str, int]) -> torch.Tensor:
    """Phi of one clip y [L] with the reflect boundary: rows x ceil(L/T) frames, flattened."""
    L = y.shape[-1]
    n, p0, f0, nf = reflect_layout(L, params)
    plan = Plan(**{**params, "N": n})
    yp = y.reshape(L).to(F64)[reflect_index(torch.arange(n) - p0, L)][None]
    phi = jtfs(yp, plan)["phi"].reshape(-1, plan.n_frames)
    return phi[:, f0:f0 + nf].reshape(-1)


def loss_and_grad_reflect(y: torch.Tensor, phi_target: torch.Tensor,
                          params: Dict[str, int]) -> Tuple[torch.Tensor, torch.Tensor]:
    """E = ||Phi_reflect(y) - target||^2 and dE/dy for one clip."""
    y = y.detach().to(F64).clone().requires_grad_(True)
    with torch.enable_grad():
        E = ((jtfs_reflect(y, params) - phi_target.to(F64)) ** 2).sum()
        (g,) = torch.autograd.grad(E, y)
    return E.detach(), g.detach()
