"""Autotuned execution choices change speed, not results."""

import itertools
import json

import numpy as np
import pytest
import torch

from workloads import get_workload, signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


@pytest.mark.parametrize("pool_tc", [0, 1])
@pytest.mark.parametrize("name", ["tones8k_n8192", "chirps22k_b8_n65536"])
def test_every_tuning_choice_gives_the_same_gradient(name, pool_tc):
    """Only the pooling split reorders a sum.  The FMA pooling accumulates in FP32 (differences ~1e-7);
    the tensor-core pooling accumulates each split's BF16 hi/lo products inside the MMA, so moving the
    split boundaries changes the result at ~1e-6 (tolerance 1e-5, ten times below the parity bound)."""
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload(name)
    B = 2
    plan = JTFSPlan(**wl.params, batch=B)
    plan.set_tuning(list(plan.tuning()[:4]) + [pool_tc])
    tol = 1e-5 if plan.tuning()[4] else 1e-6
    y = torch.tensor(np.stack([signals.white_noise(wl.N, 7 + b) for b in range(B)]), device="cuda")
    tgt = plan.forward(torch.tensor(np.stack([signals.white_noise(wl.N, 17 + b) for b in range(B)]), device="cuda"))
    ref_choice = plan.tuning()
    l0, g0 = plan.loss_grad(y, tgt)
    for wide, split, pts in itertools.product((0, 1), (1024, 2048, 4096), (1024, 8192)):
        plan.set_tuning((wide, split, pts))
        assert plan.tuning()[:3] == (wide, split, pts)
        l1, g1 = plan.loss_grad(y, tgt)
        assert _rel(l1, l0) <= tol and _rel(g1, g0) <= tol, (wide, split, pts)
        if split == ref_choice[1]:   # only the pooling split reorders a sum
            assert torch.equal(l1, l0) and torch.equal(g1, g0), (wide, split, pts)
    plan.set_tuning(ref_choice)


def test_autotune_picks_a_valid_choice_and_caches_it(tmp_path):
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload("tones8k_n8192")
    plan = JTFSPlan(**wl.params, batch=4)
    y = torch.tensor(np.stack([signals.white_noise(wl.N, b) for b in range(4)]), device="cuda")
    tgt = plan.forward(y.flip(0).contiguous())
    cache = tmp_path / "tune.json"
    choice = plan.autotune(y, tgt, cache=str(cache))
    assert choice[0] in (0, 1) and choice[1] in (1024, 2048, 4096) and choice[2] in (1024, 2048, 4096, 8192)
    assert choice[3] in (0, 1)
    table = json.load(open(cache))
    assert list(table.values()) == [list(choice)]
    other = JTFSPlan(**wl.params, batch=4)
    assert other.autotune(y, tgt, cache=str(cache)) == choice


@pytest.mark.parametrize("name", ["tones8k_n8192", "chirps22k_b8_n65536"])
def test_time_fft_engines_agree(name):
    """Tuning choice 6: the in-place radix-16 / cluster time-axis FFT engine and the batched / four-step
    kernels compute the same transforms (§3.2-§3.3) up to FP32 rounding, forward and gradient; the
    four-step kernels with every small-FFT batching give one result."""
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload(name)
    B = 2
    plan = JTFSPlan(**wl.params, batch=B)
    base = list(plan.tuning())
    assert base[5] == 1
    x = torch.tensor(np.stack([signals.harmonic_tones(wl.N, wl.sr, 5 + b) for b in range(B)]), device="cuda")
    y = torch.tensor(np.stack([signals.white_noise(wl.N, 9 + b) for b in range(B)]), device="cuda")
    res = {}
    for eng in (1, 0):
        plan.set_tuning(base[:5] + [eng])
        assert plan.tuning()[5] == eng
        phi = plan.forward(x)
        loss, g = plan.loss_grad(y, phi.flip(0).contiguous())
        res[eng] = (phi.clone(), loss.clone(), g.clone())
    for a, b in zip(res[1], res[0]):
        assert _rel(a, b) <= 2e-6, name
    plan.set_tuning(base[:2] + [1024] + base[3:5] + [0])
    l1, g1 = plan.loss_grad(y, res[0][0].flip(0).contiguous())
    assert _rel(g1, res[0][2]) <= 1e-6
    plan.set_tuning(base)
    plan.check_status("engine comparison")


@pytest.mark.parametrize("name", ["tones8k_n8192", "chirps22k_b8_n65536"])
def test_concurrent_frequential_launches_match_in_order_ones(name):
    """The second-order frequential stage runs its independent launches (the two tensor-core kernels, the
    FFT kernels of the larger groups, the first-order adjoint) on forked streams; with stage events
    registered they run in order on the caller's stream.  They write disjoint data, so both schedules
    give the same bits, eagerly and replayed from a CUDA graph."""
    import ctypes

    from paper_2602_11896_gb300 import JTFSPlan, _native
    wl = get_workload(name)
    B = 2
    plan = JTFSPlan(**wl.params, batch=B)
    y = torch.tensor(np.stack([signals.white_noise(wl.N, 31 + b) for b in range(B)]), device="cuda")
    tgt = plan.forward(torch.tensor(np.stack([signals.white_noise(wl.N, 41 + b) for b in range(B)]),
                                    device="cuda"))
    lib = _native.load()
    l_conc, g_conc = plan.loss_grad(y, tgt)
    ws = plan.workspace(y.device)
    loss = torch.empty(B, device="cuda")
    grad = torch.empty_like(y)
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            plan.loss_grad(y, tgt, loss_out=loss, grad_out=grad, workspace=ws)
    torch.cuda.current_stream().wait_stream(cap)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(loss, l_conc) and torch.equal(grad, g_conc)
    # In-order schedule: stage events registered (one begin/end pair per stage, used by the first call).
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(12)]
    for e in evs:
        e.record()
    arrs = []
    for st in range(6):
        arr = (ctypes.c_void_p * 2)(ctypes.c_void_p(evs[2 * st].cuda_event), ctypes.c_void_p(evs[2 * st + 1].cuda_event))
        arrs.append(arr)
        assert lib.jtfs_profile_stage(plan._h, st, arr, 2) == 0
    try:
        l_ord, g_ord = plan.loss_grad(y, tgt)
        torch.cuda.synchronize()
    finally:
        for st in range(6):
            lib.jtfs_profile_stage(plan._h, st, None, 0)
    assert torch.equal(l_ord, l_conc) and torch.equal(g_ord, g_conc)
