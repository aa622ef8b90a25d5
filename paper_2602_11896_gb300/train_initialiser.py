"""Train the learned initialiser and compare it with noise initialisation.

    python -m paper_2602_11896_gb300.train_initialiser --out decoder.npz

Training clips: 20k harmonic-tone clips of 2^16 samples at 8 kHz (the tone
generator of the single-clip workload, seeds 10^6 + i), JTFS parameters
J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=2^6, F=2^2, so each clip's Phi is 801 rows
x 1024 frames.  The decoder is fitted with the JTFS loss (Eq. 5) through the
library's adjoint.  Evaluation: 32 held-out targets (seeds 2*10^6 + i),
metamers from white noise (seeds 3*10^6 + i) and from the decoder, each
refined by 200 Adam steps at lr 0.1.
"""

from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import time

import numpy as np
import torch

from workloads import get_workload, signals
from workloads.configs import TRAIN_CLIPS, TRAIN_SEED0

from . import JTFSPlan
from .initialiser import Decoder, channel_scale, compare_initialisations, phi_shape, train

EVAL = "tones8k_b32_n65536"


def _tones(args):
    n, sr, seeds = args
    return np.stack([signals.harmonic_tones(n, sr, s) for s in seeds])


def make_clips(n_clips: int, n: int, sr: float, seed0: int, workers: int, device: str) -> torch.Tensor:
    """[n_clips][n] float32 on the device, generated on the host in a spawn pool."""
    out = torch.empty(n_clips, n, dtype=torch.float32, device=device)
    chunk = 250
    jobs = [(n, sr, list(range(seed0 + i, seed0 + min(i + chunk, n_clips)))) for i in range(0, n_clips, chunk)]
    with mp.get_context("spawn").Pool(workers) as pool:
        for j, arr in enumerate(pool.imap(_tones, jobs)):
            out[j * chunk:j * chunk + arr.shape[0]].copy_(torch.from_numpy(arr))
    return out


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--clips", type=int, default=TRAIN_CLIPS)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--epochs", type=float, default=10.0)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=min(16, mp.cpu_count()))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="decoder.npz")
    ap.add_argument("--report", default=None, help="write the evaluation as JSON here")
    ap.add_argument("--no-eval", action="store_true")
    a = ap.parse_args(argv)

    wl = get_workload(EVAL)
    t0 = time.time()
    clips = make_clips(a.clips, wl.N, wl.sr, TRAIN_SEED0, a.workers, "cuda")
    torch.cuda.synchronize()
    print(f"generated {a.clips} training clips in {time.time() - t0:.1f} s", flush=True)

    plan = JTFSPlan(**wl.params, batch=a.batch)
    rows, frames = phi_shape(plan)
    sample = torch.cat([plan.forward(clips[i:i + a.batch]).view(a.batch, rows, frames)
                        for i in range(0, min(a.clips, 8 * a.batch) - a.batch + 1, a.batch)])
    dec = Decoder(rows, frames, seed=a.seed, row_scale=channel_scale(sample))
    del sample
    steps = max(1, int(a.epochs * a.clips / a.batch))
    print(f"decoder: {dec.n_params} parameters, {rows} x {frames} -> {frames << dec.layers}; {steps} steps",
          flush=True)
    t0 = time.time()
    history = train(dec, plan, clips, steps, lr=a.lr, seed=a.seed, log_every=max(1, steps // 40),
                    log=lambda s: print(s, flush=True))
    torch.cuda.synchronize()
    train_s = time.time() - t0
    print(f"trained in {train_s:.1f} s ({1e3 * train_s / steps:.2f} ms/step)", flush=True)
    dec.save(a.out)
    del clips

    report = {"train_clips": a.clips, "batch": a.batch, "train_steps": steps, "train_seconds": train_s,
              "history": history}
    if not a.no_eval:
        eplan = JTFSPlan(**wl.params, batch=wl.batch)
        phi_t = eplan.forward(torch.tensor(wl.targets(), device="cuda"))
        noise = torch.tensor(wl.inits(), device="cuda")
        ev = compare_initialisations(dec, eplan, phi_t, noise)
        report["eval"] = ev
        print(json.dumps({k: v for k, v in ev.items() if not k.endswith("_curve")}), flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f)
    return report


if __name__ == "__main__":
    main()
