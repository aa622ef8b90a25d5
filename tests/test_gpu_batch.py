"""Ragged batches (clips of uneven length) through the C ABI against the oracle.

Each clip is padded to the next power of two and its Phi cropped to
ceil(L/T) frames (oracle reading R15); tolerance as the other parity tests.
"""

import numpy as np
import pytest
import torch

from oracle import jtfs_oracle as O
from workloads import signals, uneven_lengths

pytestmark = pytest.mark.gpu

TOL = 1e-4
TINY = dict(J=4, Q=4, Q2=1, J_fr=2, Q_fr=1, T=16, F=2)
TONES = dict(J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _batch(lengths, params):
    from paper_2602_11896_gb300 import JTFSBatch
    return JTFSBatch(lengths, **params)


def _clips(lengths, seed):
    return [signals.white_noise(int(L), seed + i) for i, L in enumerate(lengths)]


def test_batch_forward_matches_oracle_per_clip():
    lengths = [200, 256, 97, 512, 300, 16, 1]
    b = _batch(lengths, TINY)
    clips = _clips(lengths, 5)
    x = torch.tensor(np.concatenate(clips), device="cuda")
    phi = b.forward(x).cpu().numpy()
    for i, c in enumerate(clips):
        ref = O.jtfs_uneven(torch.tensor(c, dtype=torch.float64), dict(TINY)).numpy()
        got = phi[b.phi_offsets[i]:b.phi_offsets[i + 1]]
        assert got.shape == ref.shape, (i, got.shape, ref.shape)
        assert _rel(got, ref) <= TOL, i


def test_batch_metamer_step_matches_oracle_gradient():
    lengths = [200, 97, 512]
    b = _batch(lengths, TINY)
    y0 = _clips(lengths, 30)
    tg = _clips(lengths, 40)
    targets = [O.jtfs_uneven(torch.tensor(c, dtype=torch.float64), dict(TINY)) for c in tg]
    y = torch.tensor(np.concatenate(y0), device="cuda")
    tgt = torch.cat(targets).float().cuda()
    m = torch.zeros_like(y)
    v = torch.zeros_like(y)
    step = torch.ones(1, dtype=torch.int32, device="cuda")
    loss = b.metamer_step(y, tgt, m, v, step, 0.1)
    torch.cuda.synchronize()
    assert step.item() == 2
    for i, (c, t) in enumerate(zip(y0, targets)):
        E, g = O.loss_and_grad_uneven(torch.tensor(c, dtype=torch.float64), t, dict(TINY))
        assert _rel([loss[i].item()], [E.item()]) <= TOL
        # Adam's first step moves every sample by lr * g / (|g| + eps): compare the update direction
        s0, s1 = b.sample_offsets[i], b.sample_offsets[i + 1]
        upd = (y[s0:s1].double().cpu() - torch.tensor(c, dtype=torch.float64))
        expect = -0.1 * g / (g.abs() + 1e-8)
        big = g.abs() > 1e-3 * g.abs().max()
        assert torch.allclose(upd[big], expect[big], rtol=0, atol=1e-4)
        assert _rel(m[s0:s1].double().cpu().numpy(), (0.1 * g).numpy()) <= TOL


def test_batch_graph_replay_equals_eager():
    """The whole ragged step recorded once in a CUDA graph and replayed gives the
    same iterates as calling it eagerly (the step index lives on the device)."""
    lengths = [3000, 8192, 5000, 1024]
    b = _batch(lengths, TONES)
    y0 = torch.tensor(np.concatenate(_clips(lengths, 50)), device="cuda")
    tgt = b.forward(torch.tensor(np.concatenate(_clips(lengths, 60)), device="cuda"))

    def run(use_graph, steps=4):
        y = y0.clone()
        m = torch.zeros_like(y)
        v = torch.zeros_like(y)
        step = torch.ones(1, dtype=torch.int32, device="cuda")
        loss = torch.empty(len(lengths), device="cuda")
        if not use_graph:
            for _ in range(steps):
                b.metamer_step(y, tgt, m, v, step, 0.1, loss_out=loss)
        else:
            b.metamer_step(y, tgt, m, v, step, 0.1, loss_out=loss)   # warm-up outside the capture
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    b.metamer_step(y, tgt, m, v, step, 0.1, loss_out=loss)
            torch.cuda.current_stream().wait_stream(s)
            for _ in range(steps - 1):   # capturing records the step without running it
                g.replay()
        torch.cuda.synchronize()
        return y.clone(), loss.clone(), step.item()

    ye, le, se = run(False)
    yg, lg, sg = run(True)
    assert se == sg == 5
    assert torch.equal(ye, yg) and torch.equal(le, lg)


def test_uneven_workload_longest_clip_of_every_bucket():
    """The 64-clip uneven workload: in every padded-length group (2^15 .. 2^18, the largest taking the
    biggest four-step FFTs) its longest clip's cropped Phi against the oracle."""
    lengths = [int(v) for v in uneven_lengths(64, 300)]
    b = _batch(lengths, TONES)
    clips = [signals.harmonic_tones(L, 8000.0, 1000 + i) for i, L in enumerate(lengths)]
    phi = b.forward(torch.tensor(np.concatenate(clips), device="cuda")).cpu().numpy()
    longest = {}
    for i, L in enumerate(lengths):
        n = O.padded_length(L)
        if n not in longest or L > lengths[longest[n]]:
            longest[n] = i
    assert max(longest) == 2 ** 18
    for n, i in sorted(longest.items()):
        ref = O.jtfs_uneven(torch.tensor(clips[i], dtype=torch.float64), dict(TONES)).numpy()
        assert _rel(phi[b.phi_offsets[i]:b.phi_offsets[i + 1]], ref) <= TOL, (n, i)


def test_uneven_workload_lengths_sampled_clip():
    """64 log-uniform lengths in [2^14, 2^18] with the 8 kHz tone parameters: the
    shortest clip's cropped Phi against the oracle (the oracle's cost bounds the sample)."""
    lengths = uneven_lengths(64, 300)
    b = _batch(lengths, TONES)
    clips = [signals.harmonic_tones(int(L), 8000.0, 1000 + i) for i, L in enumerate(lengths)]
    x = torch.tensor(np.concatenate(clips), device="cuda")
    phi = b.forward(x).cpu().numpy()
    i = int(np.argmin(lengths))
    ref = O.jtfs_uneven(torch.tensor(clips[i], dtype=torch.float64), dict(TONES)).numpy()
    assert _rel(phi[b.phi_offsets[i]:b.phi_offsets[i + 1]], ref) <= TOL
    assert np.isfinite(phi).all()
