"""Learned initialiser workload: 32 tone clips of 2^16 samples at 8 kHz.

Parity of the JTFS path in this launch configuration (every second-order
level on banded time pooling, 1024 frames per row) on sampled clips, and the
trained decoder's proposal against white-noise initialisation.
"""

import os

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from workloads import get_workload

pytestmark = pytest.mark.gpu

TOL = 1e-4
WL = get_workload("tones8k_b32_n65536")
WEIGHTS = os.path.join(os.path.dirname(__file__), "..", "paper_2602_11896_gb300", "weights",
                       "decoder_tones8k_n65536.npz")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.fixture(scope="module")
def batch():
    from paper_2602_11896_gb300 import JTFSPlan
    plan = JTFSPlan(**WL.params, batch=WL.batch)
    return plan, WL.targets(), WL.inits()


def test_forward_and_gradient_parity_sampled_clips(batch):
    plan, targets, inits = batch
    ref = O.Plan(**WL.params)
    phi = plan.forward(torch.tensor(targets, device="cuda")).cpu().numpy()
    for b in (0, 31):
        phi_ref = O.jtfs(torch.tensor(targets[b:b + 1], dtype=torch.float64), ref)["phi"].numpy()[0]
        assert _rel(phi[b], phi_ref) <= TOL, b
    y = torch.tensor(inits, device="cuda")
    loss, grad = plan.loss_grad(y, torch.tensor(phi, device="cuda"))
    E, g = O.loss_and_grad(torch.tensor(inits[:1], dtype=torch.float64),
                           torch.tensor(phi[:1], dtype=torch.float64), ref)
    assert _rel([loss[0].item()], [float(E)]) <= TOL
    assert _rel(grad[0].cpu().numpy(), g.numpy()) <= TOL


def test_learned_initialiser_reaches_the_noise_runs_final_loss_sooner(batch):
    from paper_2602_11896_gb300 import JTFSPlan
    from paper_2602_11896_gb300.initialiser import Decoder, compare_initialisations
    _, targets, inits = batch
    B = 8
    plan = JTFSPlan(**WL.params, batch=B)
    dec = Decoder.load(WEIGHTS)
    phi_t = plan.forward(torch.tensor(targets[:B], device="cuda"))
    ev = compare_initialisations(dec, plan, phi_t, torch.tensor(inits[:B], device="cuda"), steps=200, lr=0.1)
    print({k: v for k, v in ev.items() if not k.endswith("_curve")})
    assert ev["learned_initial_loss"] < ev["plain_initial_loss"] / 20
    assert ev["learned_steps_to_plain_final"] is not None and ev["learned_steps_to_plain_final"] <= 60
    assert ev["learned_final_loss"] < ev["plain_final_loss"]
