"""Operand tables of the tensor-core frequential kernels against the oracle (CPU).

The tensor-core path writes the frequential filtering along n1 (§3.4: psi_beta,
then decimation by 2^k) as a fixed complex matrix H_beta, and the phi_F
averaging after the modulus (Eq. (5)) as a fixed real matrix P_k.  Here both
are rebuilt column by column from the oracle's own steps (circular convolution
of a unit column with the filter, then time-domain decimation) and compared
with the BF16 hi + lo tables the library uploads.  Host-only plans: no GPU.
"""

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from workloads import get_workload

CASES = ["tones8k_n8192", "chirps22k_b8_n65536", "notes22k_b4_n1048576"]


def _plans(name):
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload(name)
    return JTFSPlan(**wl.params, batch=1, host_only=True), O.Plan(**wl.params)


def _oracle_H(op, xi, sig, k, nmax):
    """Columns n < nmax of H_beta: decimate_k(unit column n convolved with psi_beta) (§3.4)."""
    eye = torch.zeros(nmax, op.N_fr, dtype=torch.complex128)
    eye[torch.arange(nmax), torch.arange(nmax)] = 1.0
    z = O.decimate(O.conv_circ(eye, O.freq_filter_hat(op.N_fr, xi, sig), 1), k, 1)   # [n][r]
    return z.T.numpy()                                                                  # [r][n]


def _oracle_P(op, k):
    """P_k[ro][r]: phi_F (periodised to level k) then decimation to R_out rows (Eq. (5))."""
    R = op.N_fr >> k
    eye = torch.eye(R, dtype=torch.complex128)
    phiF = O.gauss_hat(op.N_fr, op.sigma_phiF)
    v = O.decimate(O.conv_circ(eye, O.periodise(phiF, k), 1), op.lF - k, 1).real   # [r][ro]
    return v.T.numpy()


@pytest.mark.parametrize("name", CASES)
def test_filter_matrix_matches_oracle(name):
    plan, op = _plans(name)
    H = plan.tc_table(0).astype(np.float64)
    off = 0
    for xi, sig, k in op.beta_second:
        R = op.N_fr >> k
        Ho = _oracle_H(op, xi, sig, k, 64)                       # [R][64] complex
        scale = np.abs(Ho).max()
        blk = H[2 * off:2 * (off + R)]                            # rows (r, x), columns (n, y)
        Zr_from_Yr, Zr_from_Yi = blk[0::2, 0::2], blk[0::2, 1::2]
        Zi_from_Yr, Zi_from_Yi = blk[1::2, 0::2], blk[1::2, 1::2]
        # Z = H Y with complex H = Hr + i Hi: Zr = Hr Yr - Hi Yi, Zi = Hi Yr + Hr Yi.
        for got, want in ((Zr_from_Yr, Ho.real), (Zr_from_Yi, -Ho.imag), (Zi_from_Yr, Ho.imag),
                          (Zi_from_Yi, Ho.real)):
            assert np.abs(got - want).max() <= 2e-5 * scale, (xi, k)
        off += R
    assert H.shape[0] == 2 * off


@pytest.mark.parametrize("name", CASES)
def test_pooling_matrix_matches_oracle(name):
    plan, op = _plans(name)
    P = plan.tc_table(1).astype(np.float64)
    for k in range(op.lF + 1):
        R = op.N_fr >> k
        Po = _oracle_P(op, k)                                     # [R_out][R]
        assert np.abs(P[k, :, :R] - Po).max() <= 2e-5 * np.abs(Po).max(), k
        assert not P[k, :, R:].any()
