"""Host table of the coloured initialisation (§2.3) against the oracle (CPU, host-only plans)."""

import numpy as np
import pytest

from oracle import jtfs_oracle as O
from oracle import reconstruct as R
from workloads import get_workload


@pytest.mark.parametrize("name", ["tones8k_n8192", "chirps22k_b8_n65536", "notes22k_b4_n1048576"])
def test_band_gains_match_oracle(name):
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload(name)
    plan = JTFSPlan(**wl.params, batch=1, host_only=True)
    op = O.Plan(**wl.params)
    got = plan.init_gains().astype(np.float64)
    want = np.array([R.band_gain(op, n1) * 2.0 ** (op.lT - op.k1[n1]) for n1 in range(op.N1)])
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=2e-7)
