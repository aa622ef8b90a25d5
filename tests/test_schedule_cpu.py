"""Host logic of the launch schedules (no GPU): the work tables a plan builds, read through
jtfs_plan_schedule on host-only plans and checked against the oracle's plan and brute force."""

import math

import numpy as np
import pytest

from oracle import jtfs_oracle as O
from workloads import get_workload

NAMES = ["tones8k_n8192", "chirps22k_b8_n65536", "notes22k_b4_n1048576"]


def _plans(name):
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload(name)
    return wl, JTFSPlan(**wl.params, batch=wl.batch, host_only=True), O.Plan(**wl.params)


@pytest.mark.parametrize("name", NAMES)
def test_u1_gradient_blocks_cover_every_row_once(name):
    """k_dU1's block table: every U1 row (one per clip and first-order filter, N / 2^k1 samples, k1 from
    the oracle) gets blocks 0 .. max(1, length / 256) - 1, each exactly once."""
    wl, plan, ref = _plans(name)
    tab = plan.schedule(0)
    rows = {}
    for r, blk, lg in tab:
        rows.setdefault(int(r), (int(lg), []))[1].append(int(blk))
    for r, (lg, blks) in rows.items():
        assert sorted(blks) == list(range(max(1, (1 << lg) // 256))), r
    lengths = sorted(1 << lg for lg, _ in rows.values())
    assert lengths == sorted(wl.batch * [wl.N >> k for k in ref.k1])


@pytest.mark.parametrize("name", NAMES)
def test_tensor_core_groups_follow_their_rule(name):
    """Per active second-order group: rows n1max agree with the oracle; the forward takes the tensor cores
    with ceil(n1max / 32) K atoms up to 5 (160 rows) when the group has at least one 128-column tile, and
    for more than 2 atoms at least 148 tiles; the adjoint only up to 2 atoms."""
    wl, plan, ref = _plans(name)
    g = plan.schedule(2)
    assert len(g) == len(ref.active)
    for a, (s2, rows, n1max, w, s_band, kf, kb) in enumerate(g):
        n2 = ref.active[a]
        assert s2 == min(ref.psi2[n2].j, ref.lT)
        assert n1max == ref.n1_max[n2]
        L2 = wl.N >> s2
        ka = (n1max + 31) // 32 if (L2 >= 128 and n1max <= 160) else 0
        if ka >= 3 and wl.batch * L2 < 148 * 128:
            ka = 0
        assert kf == ka, a
        assert kb == (ka if ka <= 2 else 0), a


def _phi_t_reach_ok(ref, s, W):
    """The taps of phi_T at level s beyond W samples are below 2^-40 of its peak (Gaussian of width
    sigma_phiT cycles per sample: the time envelope exp(-2 pi^2 sigma^2 tau^2) at tau = W 2^s)."""
    c = 2.0 * math.pi ** 2 * ref.sigma_phiT ** 2
    return math.exp(-c * float(W << s) ** 2) < 2.0 ** -40


@pytest.mark.parametrize("name", ["tones8k_n8192", "notes22k_b4_n1048576"])
def test_banded_adjoint_ctas_hold_every_frame_within_reach(name):
    """The banded phi_T adjoint on the tensor cores: for every group with band samples S > 0, the CTAs tile
    rows in 128s and samples in S-sample steps exactly once per clip; every frame within reach W of a CTA's
    samples (circular distance of f D and t at most W) is among the 64 frames from floor((t0 - W) / D),
    checked by brute force on the first, a middle and the last CTA of each group; and W is where phi_T has
    fallen below 2^-40 of its peak."""
    wl, plan, ref = _plans(name)
    groups = plan.schedule(2)
    ctas = plan.schedule(1)
    nf = wl.N // wl.T
    for a, (s2, rows, _n1, W, S, _kf, _kb) in enumerate(groups):
        sel = ctas[ctas[:, 1] == a]
        if S == 0:
            assert len(sel) == 0
            continue
        assert W > 0 and _phi_t_reach_ok(ref, int(s2), int(W))
        L = wl.N >> int(s2)
        D = 1 << (ref.lT - int(s2))
        want = sorted((b, r0, t0) for b in range(wl.batch) for r0 in range(0, int(rows), 128)
                      for t0 in range(0, L, int(S)))
        got = sorted((int(b), int(r0), int(t0)) for b, _, r0, t0 in sel)
        assert got == want, a
        t0s = sorted({int(t0) for _, _, _, t0 in sel})
        for t0 in (t0s[0], t0s[len(t0s) // 2], t0s[-1]):
            fa = (t0 - int(W)) // D
            t = np.arange(t0, min(t0 + int(S), L))[:, None]
            f = np.arange(nf)[None, :]
            d = np.abs(f * D - t) % L
            d = np.minimum(d, L - d)
            reach = (d <= W).any(axis=0)
            window = ((np.arange(nf) - fa) % nf) < 64
            assert not (reach & ~window).any(), (a, t0)
