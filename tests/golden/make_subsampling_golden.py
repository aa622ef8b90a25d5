"""Write subsampling_j.json: the subsampling j of every filter of the tone and
chirp configurations, and the second-order row counts n1_max, derived by hand
from the closed forms of §3.1 and reading R2 -- not by calling the oracle.

Run from the repository root:  python tests/golden/make_subsampling_golden.py

Derivation (50-digit arithmetic, mpmath):
* §3.1 filterbank in closed form: f = 2^(-1/Q), xi_0 = max(1/(1+2^(3/Q)), 0.35),
  sigma_0 = (1-f)/(1+f) xi_0 / sqrt(ln 2) (r_psi = sqrt(1/2)), filter k of the
  constant-Q part (xi_0 f^k, sigma_0 f^k) for k = 0..K with K = #{k >= 0:
  sigma_0 f^k > sigma_min / f}, sigma_min = 0.1 / 2^J; then Q-1 filters
  (xi_0 f^K (1 - m/Q), sigma_min).
* Reading R2: j = the largest integer k >= 0 with 2^k (xi + 3 sigma) <= 1/2,
  found by comparing powers of two (exact in this precision); each entry keeps
  the two margins 2^j (xi + 3 sigma) <= 1/2 < 2^(j+1) (xi + 3 sigma) (the
  first fails only where the floor at 0 applies: xi + 3 sigma > 1/2).
* Low-pass filters (reading R3): phi_T has xi = 0, sigma = 0.1 / T;
  phi_F has xi = 0, sigma = 0.1 / F.  Since 3 * 0.1 = 0.3 lies in (1/4, 1/2],
  j(phi_T) = log2 T exactly.
* n1_max[n2] = number of first-order filters with j1 < j2 (reading R7).
"""

from __future__ import annotations

import json
import os

import mpmath as mp

mp.mp.dps = 50

CONFIGS = {
    "tones8k_n8192": dict(N=2 ** 13, J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4),
    "chirps22k_b8_n65536": dict(N=2 ** 16, J=12, Q=12, Q2=1, J_fr=5, Q_fr=2, T=2 ** 11, F=12),
}


def bank(J, Q):
    f = mp.power(2, mp.mpf(-1) / Q)
    xi0 = max(1 / (1 + mp.power(2, mp.mpf(3) / Q)), mp.mpf("0.35"))
    s0 = (1 - f) / (1 + f) * xi0 / mp.sqrt(mp.log(2))
    smin = mp.mpf("0.1") / mp.power(2, J)
    out = []
    if s0 <= smin:
        xe = s0
    else:
        K = 0
        while s0 * mp.power(f, K) > smin / f:
            K += 1
        out = [(xi0 * mp.power(f, k), s0 * mp.power(f, k)) for k in range(K + 1)]
        xe = out[-1][0]
    out += [(xe * (1 - mp.mpf(m) / Q), smin) for m in range(1, Q)]
    return out


def subsampling(xi, sigma):
    edge = xi + 3 * sigma
    j = 0
    while mp.power(2, j + 1) * edge <= mp.mpf("0.5"):
        j += 1
    return j, float(mp.power(2, j) * edge), float(mp.power(2, j + 1) * edge)


def entries(fb):
    out = []
    for xi, sg in fb:
        j, lo, hi = subsampling(xi, sg)
        assert (lo <= 0.5 or j == 0) and hi > 0.5
        out.append({"xi": float(xi), "sigma": float(sg), "j": j, "2^j(xi+3s)": lo, "2^(j+1)(xi+3s)": hi})
    return out


def main():
    gold = {"_source": "Derivation " + __doc__.split("Derivation ")[1].strip(), "configs": {}}
    for name, c in CONFIGS.items():
        psi1 = entries(bank(c["J"], c["Q"]))
        psi2 = entries(bank(c["J"], c["Q2"]))
        psifr = entries(bank(c["J_fr"], c["Q_fr"]))
        phiT = entries([(mp.mpf(0), mp.mpf("0.1") / c["T"])])[0]
        phiF = entries([(mp.mpf(0), mp.mpf("0.1") / c["F"])])[0]
        n1_max = [sum(1 for a in psi1 if a["j"] < b["j"]) for b in psi2]
        gold["configs"][name] = {"params": c, "psi1": psi1, "psi2": psi2, "psi_fr": psifr,
                                 "phi_T": phiT, "phi_F": phiF, "n1_max": n1_max}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "subsampling_j.json")
    with open(path, "w") as fh:
        json.dump(gold, fh, indent=1)
    print(path)


if __name__ == "__main__":
    main()
