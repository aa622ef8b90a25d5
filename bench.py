"""Benchmark: JTFS metamer step throughput (audio samples/s) on GB300.

One step = metamer_step on the batch-8, 2^16-sample chirp workload (J=12,
Q=12, Q2=1, J_fr=5, Q_fr=2, T=2^11, F=12): JTFS forward, loss against the
target Phi, hand-written adjoint, Adam update, all in the library's CUDA
kernels.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun, one rank per GPU): every rank solves its own batch of
clips (independent metamers, no data-path collective; weak scaling).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import get_workload  # noqa: E402

WORKLOAD = "chirps22k_b8_n65536"
METRIC = "JTFS fwd+bwd audio-samples/s"
UNIT = "audio-samples/s"
L2_FLUSH_BYTES = 256 << 20
# FP32 ALU peak of a GB300 from unit counts: 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one clip's launches of each profiling stage (the
# tensor-core frequential forward = 4 and adjoint = 5, both kernels of a stage summed), from the capture
# of the 1-clip case summarised in profiles/top_kernels_chirps22k_b1_n65536.md; the traffic of a launch
# grows with the clips it processes.  Valid for the kernel versions it was taken on; emptied when those
# kernels change.
DRAM_BYTES_PER_CLIP = {4: (10.712064 + 83.598592 + 7.814400 + 0.015616) * 1e6,
                       5: (155.660800 + 4.626432 + 52.681216 + 0.058880) * 1e6}


def bf16_peak():
    """Measured dense BF16 tensor peak of the GB300s (sustained figure: the kernel is timed
    inside a long run of steps), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        mp = json.load(open(path))
        return float(mp["bf16_tflops_sustained"]), "measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    except (OSError, ValueError, KeyError):
        return 1700.0, "fallback (sustained BF16, no MEASURED_PEAKS.json)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip autotuning at set-up")
    ap.add_argument("--workload", default="chirps",
                    choices=["chirps", "uneven64", "initialiser", "decoder", "long", "reconstruct", "reflect"],
                    help="chirps: the 8 x 2^16 benchmark (default); uneven64: 64 clips of 2^14..2^18 samples; "
                         "initialiser: 32 tone clips of 2^16 samples from the learned decoder vs white noise; "
                         "decoder: the learned initialiser's training step on the tensor cores; "
                         "long: 4 clips of 2^20 samples, forward + loss + gradient; "
                         "reconstruct: the paper's coloured-noise start and bold-driver momentum against "
                         "white-noise Adam on the chirp batch, 200 evaluations each; "
                         "reflect: the chirp batch with mirror padding on both sides")
    ap.add_argument("--unpooled", default="none", choices=list(VARIANTS),
                    help="chirps workload only: unpooled outputs (average_local / average_local_fr off): "
                         "time, freq or both")
    ap.add_argument("--batch", type=int, default=0,
                    help="clips per GPU (default: the workload's 8); smaller values only for ncu captures")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# Algorithmic FLOP model (5 n log2 n per complex FFT, 2.5 n log2 n per real
# FFT, 2 per real-filter product, 3 per modulus, 6 per modulus adjoint).
# ---------------------------------------------------------------------------
def _lg(n):
    return math.log2(n) if n > 1 else 0.0


def freq_flops_per_column(plan, adjoint: bool) -> float:
    info = plan.info
    Nfr, Rout, lF = info["N_fr"], info["R_out"], info["log2_F"]
    pooled = getattr(plan, "average_local_fr", True)
    cap = (lambda j: min(int(j), lF)) if pooled else int
    _, _, jf = plan.filters(2)
    _, _, jl = plan.filters(3)
    ks = [cap(jl[1])] + [cap(j) for j in jf] * 2
    f = 5 * Nfr * _lg(Nfr)
    for k in ks:
        R = Nfr >> k
        pool = 2.5 * R * _lg(R) + 2 * R + 2.5 * Rout * _lg(Rout) if pooled else 0.0   # phi_F and its adjoint
        if not adjoint:
            f += 2 * Nfr + 5 * R * _lg(R) + 3 * R + pool
        else:
            f += 2 * Nfr + 5 * R * _lg(R) + pool + 6 * R + 5 * R * _lg(R) + 2 * Nfr
    if adjoint:
        f += 5 * Nfr * _lg(Nfr)
    return f


def tc_groups(plan):
    """Second-order groups the tensor-core frequential kernels take: (n1max, columns per clip)."""
    info = plan.info
    _, _, j2 = plan.filters(1)
    _, _, j1 = plan.filters(0)
    lT = info["log2_T"]
    out = []
    if info["R_out"] not in (16, 32) or info["N_fr"] < 64:
        return out
    for jj in j2:
        n1 = int((j1 < jj).sum())
        L2 = info["N"] >> min(int(jj), lT)
        if 0 < n1 <= 64 and L2 >= 128:
            out.append((n1, L2))
    return out


def tc_tensor_flops(plan, adjoint: bool) -> float:
    """Tensor FLOPs the tensor-core frequential launches issue per call (three BF16 products per
    FP32 product: hi.hi + lo.hi + hi.lo), M = 128 columns per tile."""
    info = plan.info
    Nfr, RO, lF = info["N_fr"], info["R_out"], info["log2_F"]
    _, _, jf = plan.filters(2)
    _, _, jl = plan.filters(3)
    ks = [min(int(jl[1]), lF)] + [min(int(j), lF) for j in jf] * 2
    chunks = []
    for k in ks:
        R = Nfr >> k
        rc = min(R, 32)
        chunks += [rc] * (R // rc)
    total = 0.0
    for n1, L2 in tc_groups(plan):
        kp = 16 * ((2 * n1 + 15) // 16)
        tiles = info["batch"] * ((L2 + 127) // 128)
        per_tile = 0.0
        for rc in chunks:
            per_tile += 2 * 128 * (2 * rc) * kp + 2 * 128 * RO * rc      # GEMM1 (recomputed in the adjoint), pooling
            if adjoint:
                per_tile += 2 * 128 * kp * (2 * rc)                        # GEMM3
        total += 3 * per_tile * tiles
    return total


def compulsory_bytes_per_clip(plan) -> float:
    """HBM bytes a fused forward + loss + adjoint cannot avoid, per clip: x read twice, U1 written and read
    once (it is recomputed, not stored, for the adjoint), dU1 written and read, Phi written, the target Phi
    read, dy written (FP32).  Y2 and the un-pooled second order are not counted: a fused design keeps them
    on chip."""
    info = plan.info
    N, lT = info["N"], info["log2_T"]
    _, _, j1 = plan.filters(0)
    u1 = sum(N >> min(int(j), lT) for j in j1)
    return 4.0 * (2 * N + 2 * u1 + 2 * u1 + 2 * plan.phi_size + N)


def hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def columns_per_launch(plan) -> int:
    """Time columns the second-order frequential kernels process per launch."""
    info = plan.info
    _, _, j2 = plan.filters(1)
    _, _, j1 = plan.filters(0)
    lT = info["log2_T"]
    cols = 0
    for jj in j2:
        if (j1 < jj).sum() > 0:
            cols += info["N"] >> min(int(jj), lT)
    return cols * info["batch"]


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        self.proc = subprocess.Popen([exe, f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Reference arm: the FP64 oracle on the host cores.
# ---------------------------------------------------------------------------
# Output variant of the chirp step (--unpooled): average_local, average_local_fr.
VARIANTS = {"none": (True, True), "time": (False, True), "freq": (True, False), "both": (False, False)}
VARIANT = {"name": "none"}


def variant_kw():
    al, alf = VARIANTS[VARIANT["name"]]
    return dict(average_local=al, average_local_fr=alf)


def rank_inputs(wl, rank: int):
    """(targets, initial iterates) [batch][N] of one rank: rank 0 runs the workload's own seeds, rank r
    the same recipe with seeds offset by 1000 r (independent clips per GPU: weak scaling, no collective)."""
    import dataclasses
    off = 1000 * rank
    w = dataclasses.replace(wl, target_seeds=[s + off for s in wl.target_seeds],
                            init_seeds=[s + off for s in wl.init_seeds])
    return w.targets(), w.inits()


def job_throughput(ms_local: float, world: int, clips_per_rank: int, N: int, steps: int, dist=None, device=None):
    """(slowest rank's ms for `steps` steps, whole-job audio-samples/s): every rank processed
    clips_per_rank x N samples per step; the job's time is the maximum over ranks."""
    ms = ms_local
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * clips_per_rank * N * steps / (ms / 1e3)


def oracle_clip_seconds(wl, clip: int):
    from oracle import jtfs_oracle as O
    ref = O.Plan(**wl.params, **variant_kw())
    y = torch.tensor(wl.inits()[clip:clip + 1], dtype=torch.float64)
    tgt = O.jtfs(torch.tensor(wl.targets()[clip:clip + 1], dtype=torch.float64), ref)["phi"]
    t0 = time.perf_counter()
    O.loss_and_grad(y, tgt, ref, checkpoint_blocks=True)
    return time.perf_counter() - t0


def run_reference(args, wl):
    from oracle import jtfs_oracle as O
    small = get_workload("tones8k_n8192")
    sp = O.Plan(**small.params, **variant_kw())
    ys = torch.tensor(small.inits(), dtype=torch.float64)
    ts = O.jtfs(torch.tensor(small.targets(), dtype=torch.float64), sp)["phi"]
    for _ in range(args.warmup):
        O.loss_and_grad(ys, ts, sp)
    steps = max(1, min(args.steps, 3))
    total = 0.0
    for k in range(steps):
        total += oracle_clip_seconds(wl, k % wl.batch)
    value = steps * wl.N / total
    cores = torch.get_num_threads()
    sample = (f"{steps} step(s), each the oracle's FP64 forward+loss+adjoint (autograd) of one "
              f"{wl.N}-sample clip of the {wl.name} workload; warm-up on 8192-sample clips")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def device_status(what: str) -> None:
    """Fail the run if, since the last check, a tensor-core kernel gave up on a barrier (its outputs, and
    so the timed work, are invalid) or a loss was NaN / Inf (jtfs_status; synchronises the stream)."""
    from paper_2602_11896_gb300 import _native
    _native.check_status(what, torch.cuda.current_stream().cuda_stream)


def config_dict(wl):
    cfg = {"workload": wl.name, "batch": wl.batch, "N": wl.N, "J": wl.J, "Q": wl.Q, "Q2": wl.Q2,
           "J_fr": wl.J_fr, "Q_fr": wl.Q_fr, "T": wl.T, "F": wl.F, "sample_rate_hz": wl.sr,
           "step": "metamer_step: JTFS forward + loss + hand-written adjoint + Adam (lr 0.1)",
           "l2": f"{L2_FLUSH_BYTES >> 20} MiB buffer written between timed steps (outside the events)",
           "parallelism": "replicas (independent clips per GPU)"}
    if VARIANT["name"] != "none":
        cfg["workload"] = f"{wl.name}_unpooled_{VARIANT['name']}"
        cfg["outputs"] = {"time": "second order at stride 2^j2 without phi_T, zeroth order = x",
                          "freq": "frequential stride 2^j without phi_F",
                          "both": "no phi_T on the second order and no phi_F"}[VARIANT["name"]]
    return cfg


# ---------------------------------------------------------------------------
# Native arm.
# ---------------------------------------------------------------------------
def run_uneven(args):
    """64 clips with log-uniform lengths in [2^14, 2^18] (seed 300), 8 kHz tone parameters, all
    solved together: one ragged metamer step recorded in a CUDA graph and replayed."""
    from paper_2602_11896_gb300 import JTFSBatch
    from workloads import signals, uneven_lengths
    params = dict(J=6, Q=8, Q2=1, J_fr=3, Q_fr=1, T=64, F=4)
    lengths = [int(v) for v in uneven_lengths(64, 300)]
    b = JTFSBatch(lengths, **params)
    x = torch.tensor(np.concatenate([signals.harmonic_tones(L, 8000.0, 1000 + i) for i, L in enumerate(lengths)]),
                     device="cuda")
    y = torch.tensor(np.concatenate([signals.white_noise(L, 2000 + i) for i, L in enumerate(lengths)]),
                     device="cuda")
    tgt = b.forward(x)
    m = torch.zeros_like(y)
    v = torch.zeros_like(y)
    step = torch.ones(1, dtype=torch.int32, device="cuda")
    loss = torch.empty(len(lengths), device="cuda")
    for _ in range(max(args.warmup, 1)):
        b.metamer_step(y, tgt, m, v, step, 0.1, loss_out=loss)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.metamer_step(y, tgt, m, v, step, 0.1, loss_out=loss)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(0)
    clocks.start()
    for e0, e1 in ev:
        e0.record()
        g.replay()
        e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    device_status("timed steps")
    lat = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
    total = sum(lengths)
    line = {"metric": "batched uneven metamer step audio-samples/s", "value": total / (lat.mean() / 1e3),
            "unit": "audio-samples/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": float(lat.mean()), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "uneven64_tones8k", "clips": len(lengths), "samples": total,
                       "min_len": min(lengths), "max_len": max(lengths), **params,
                       "groups": sorted(set(1 << (max(L, 64) - 1).bit_length() for L in lengths)),
                       "step": "one ragged metamer step for all clips (pad to 2^k, crop frames), CUDA-graph replay",
                       "l2": "inputs and intermediates exceed L2 (GBs of workspace)"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "note": "every clip of the batch finishes with the step: per-clip latency = step latency"},
            "clocks": clk, "final_loss_mean": float(loss.mean().item())}
    print(json.dumps(line), flush=True)


def run_reflect(args):
    """The chirp batch (8 x 2^16 samples) with the reflect boundary: each clip mirrored on both sides to
    2^17 samples, Phi over the clip's frames; one metamer step (ragged-batch API) recorded in a CUDA graph."""
    from paper_2602_11896_gb300 import JTFSBatch
    wl = get_workload(WORKLOAD)
    lengths = [wl.N] * wl.batch
    b = JTFSBatch(lengths, **{k: v for k, v in wl.params.items() if k != "N"}, boundary="reflect")
    x = torch.tensor(wl.targets().reshape(-1), device="cuda")
    y = torch.tensor(wl.inits().reshape(-1), device="cuda")
    tgt = b.forward(x)
    m = torch.zeros_like(y)
    v = torch.zeros_like(y)
    step = torch.ones(1, dtype=torch.int32, device="cuda")
    loss = torch.empty(wl.batch, device="cuda")
    for _ in range(max(args.warmup, 3)):
        b.metamer_step(y, tgt, m, v, step, 0.1, loss_out=loss)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.metamer_step(y, tgt, m, v, step, 0.1, loss_out=loss)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(0)
    clocks.start()
    for e0, e1 in ev:
        e0.record()
        g.replay()
        e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    device_status("timed steps")
    lat = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
    total = sum(lengths)
    line = {"metric": "JTFS fwd+bwd audio-samples/s (reflect boundary)", "value": total / (lat.mean() / 1e3),
            "unit": "audio-samples/s", "n_gpus": 1, "steps": K, "warmup": max(args.warmup, 3),
            "ms_per_step": float(lat.mean()), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name + "_reflect", "clips": wl.batch, "samples": total, **wl.params,
                       "padded_length": 2 * wl.N,
                       "step": "metamer step (Adam, lr 0.1) with mirror padding on both sides, CUDA-graph replay",
                       "l2": "inputs and intermediates exceed L2 (GBs of workspace)"},
            "clocks": clk, "final_loss_mean": float(loss.mean().item())}
    print(json.dumps(line), flush=True)


def run_initialiser(args):
    """32 held-out tone clips (2^16 samples, 8 kHz parameters): 200 Adam steps (lr 0.1) from white noise,
    then from the trained decoder's proposal; wall time for the latter to reach the former's final loss."""
    from paper_2602_11896_gb300 import JTFSPlan
    from paper_2602_11896_gb300.initialiser import Decoder, compare_initialisations
    wl = get_workload("tones8k_b32_n65536")
    weights = os.path.join(ROOT, "paper_2602_11896_gb300", "weights", "decoder_tones8k_n65536.npz")
    plan = JTFSPlan(**wl.params, batch=wl.batch)
    dec = Decoder.load(weights)
    phi_t = plan.forward(torch.tensor(wl.targets(), device="cuda"))
    noise = torch.tensor(wl.inits(), device="cuda")
    for _ in range(max(args.warmup, 1)):   # warm-up: one short run of each arm
        compare_initialisations(dec, plan, phi_t, noise, steps=3)
    clocks = ClockSampler(0)
    clocks.start()
    ev = compare_initialisations(dec, plan, phi_t, noise, steps=200, lr=0.1)
    clk = clocks.stop()
    line = {"metric": "learned-initialiser wall time to the noise run's 200-step loss", "unit": "ms",
            "value": ev["learned_ms_to_plain_final"], "n_gpus": 1, "steps": 200, "warmup": max(args.warmup, 1),
            "ms_per_step": ev["plain_ms"] / 200, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (decoder: bf16 operands, f32 accumulate)", "data": "synthetic",
            "config": {"workload": wl.name, "batch": wl.batch, **wl.params, "sample_rate_hz": wl.sr,
                       "decoder": "6 transposed convs, 128 channels, kernel 9, GELU; 801 x 1024 -> 65536",
                       "train": "20k tone clips (seeds 1e6 + i), JTFS loss, 6250 Adam steps of 32 (10 epochs)",
                       "l2": "each arm's 200 steps timed as one region; inputs and workspace exceed L2"},
            "noise_ms_200_steps": ev["plain_ms"], "decoder_ms": ev["decoder_ms"],
            "learned_steps_to_noise_final": ev["learned_steps_to_plain_final"],
            "noise_loss": [ev["plain_initial_loss"], ev["plain_final_loss"]],
            "learned_loss": [ev["learned_initial_loss"], ev["learned_final_loss"]],
            "speedup_wall": (ev["plain_ms"] / ev["learned_ms_to_plain_final"]
                             if ev["learned_ms_to_plain_final"] else None),
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_reconstruct(args):
    """The chirp batch (8 x 2^16): the paper's reconstruction of §2.3 (coloured noise following S1x, momentum
    0.9 with bold-driver step size from 0.1) against white-noise Adam (lr 0.1), and the two crossed arms,
    200 gradient evaluations each; wall time for each arm to reach the white-noise Adam run's final loss."""
    from paper_2602_11896_gb300 import JTFSPlan
    from paper_2602_11896_gb300.reconstruct import compare_reconstruction
    wl = get_workload(WORKLOAD)
    plan = JTFSPlan(**wl.params, batch=wl.batch)
    if not args.no_tune:
        plan.autotune(torch.tensor(wl.inits(), device="cuda"), plan.forward(torch.tensor(wl.targets(), device="cuda")))
    x = torch.tensor(wl.targets(), device="cuda")
    phi_t = plan.forward(x)
    noise = torch.tensor(wl.inits(), device="cuda")
    for _ in range(max(args.warmup, 1)):   # warm-up: a short run of every arm
        compare_reconstruction(plan, x, phi_t, noise, steps=3)
    steps = 200
    clocks = ClockSampler(0)
    clocks.start()
    ev = compare_reconstruction(plan, x, phi_t, noise, steps=steps)
    clk = clocks.stop()
    marks = [0, 9, 24, 49, 99, 149, 199]
    arms = {k: {"initial_loss": a["initial_loss"], "final_loss": a["final_loss"], "ms": a["ms"],
                "init_ms": a["init_ms"], "steps_to_target": a["steps_to_target"], "ms_to_target": a["ms_to_target"],
                "curve_at": {str(i + 1): a["curve"][i] for i in marks},
                **{k2: a[k2] for k2 in ("rejected", "final_mu") if k2 in a}}
            for k, a in ev["arms"].items()}
    paper = ev["arms"]["coloured_momentum"]
    line = {"metric": "wall time of the paper's reconstruction (coloured init + bold-driver momentum) to the "
                      "white-noise Adam run's 200-step loss", "unit": "ms",
            "value": paper["ms_to_target"], "n_gpus": 1, "steps": steps, "warmup": max(args.warmup, 1),
            "ms_per_step": paper["ms_per_step"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "batch": wl.batch, **wl.params, "sample_rate_hz": wl.sr,
                       "adam": {"lr": ev["lr"]}, "momentum": {"m": ev["m"], "mu0": ev["mu0"],
                                                              "bold_driver": [1.1, 0.5]},
                       "curves": "per-clip running minimum of the loss, summed over the batch",
                       "l2": "each arm's evaluations timed as one region; inputs and workspace exceed L2"},
            "target_loss": ev["target_loss"], "arms": arms, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_long(args):
    """4 clips of 2^20 samples (polyphonic notes + pink noise at 22.05 kHz; J=14, Q=16, Q2=2, J_fr=6,
    Q_fr=2, T=2^13, F=16): one step = forward, loss against the targets' Phi and the hand-written adjoint
    (jtfs_loss_grad; U1's phase and every un-pooled second-order column are recomputed, never stored)."""
    from paper_2602_11896_gb300 import JTFSPlan
    wl = get_workload("notes22k_b4_n1048576")
    torch.cuda.reset_peak_memory_stats()
    plan = JTFSPlan(**wl.params, batch=wl.batch)
    phi_t = plan.forward(torch.tensor(wl.targets(), device="cuda"))
    y = torch.tensor(wl.inits(), device="cuda")
    loss = torch.empty(wl.batch, device="cuda")
    grad = torch.empty_like(y)
    ws = plan.workspace(y.device)
    for _ in range(max(args.warmup, 3)):
        plan.loss_grad(y, phi_t, loss_out=loss, grad_out=grad, workspace=ws)
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(0)
    clocks.start()
    for e0, e1 in ev:
        e0.record()
        plan.loss_grad(y, phi_t, loss_out=loss, grad_out=grad, workspace=ws)
        e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    device_status("timed steps")
    ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in ev]))
    peak = torch.cuda.max_memory_allocated()
    line = {"metric": METRIC, "value": wl.batch * wl.N / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**config_dict(wl), "step": "jtfs_loss_grad: forward + loss + hand-written adjoint",
                       "l2": "workspace and inputs exceed L2 (tens of GB)"},
            "peak_hbm_gib": peak / 2 ** 30, "workspace_gib": plan.workspace_bytes / 2 ** 30,
            "gpu_launches": int(plan._lib.jtfs_launch_count(plan._h, 2)) * K, "clocks": clk,
            "loss_mean": float(loss.mean().item())}
    print(json.dumps(line), flush=True)


def run_decoder(args):
    """The learned initialiser's own training step without the JTFS loss: decoder forward, backward from a
    fixed waveform gradient, Adam and BF16 repacking, on B clips of Phi (801 rows x 1024 frames, the 2^16-
    sample tone plan).  Throughput in algorithmic FLOP/s; roofline of the busiest tensor-core kernel."""
    from paper_2602_11896_gb300.initialiser import Decoder
    B = args.batch or 32
    dec = Decoder(801, 1024, seed=0)
    g = torch.Generator(device="cuda").manual_seed(0)
    phi = torch.rand(B, 801, 1024, device="cuda", generator=g)
    dy = torch.randn(B, 1024 << dec.layers, device="cuda", generator=g)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")

    def step():
        dec.forward(phi)
        dec.backward(dy)
        dec.step(1e-5)

    for _ in range(max(args.warmup, 3)):
        step()
    dec.check_errors()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    dec.profile = []
    clocks = ClockSampler(0)
    clocks.start()
    for e0, e1 in ev:
        flush.fill_(1.0)
        e0.record()
        step()
        e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    dec.check_errors()
    ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in ev]))
    lf = dec.layer_flops(B)
    L = dec.layers
    # forward: every layer; weight gradient: every layer; data gradient: layers 1 .. L-1
    step_flops = sum(lf) * 2 + sum(lf[1:])
    kinds = {"fwd": ("k_umma<FwdOp> (forward, layers 0-4)", sum(lf[:L - 1])),
             "dw": ("k_umma<DwOp> (weight gradient, layers 0-4)", sum(lf[:L - 1])),
             "dx": ("k_umma<BwdDataOp> (data gradient, layers 1-4)", sum(lf[1:L - 1]))}
    per_kind = {}
    for kind, li, e0, e1 in dec.profile:
        t = e0.elapsed_time(e1)
        per_kind.setdefault(kind, [0.0, 0])
        per_kind[kind][0] += t
        per_kind[kind][1] += 1
    dec.profile = None
    top = max(kinds, key=lambda k: per_kind.get(k, [0.0])[0])
    top_ms = per_kind[top][0] / K  # per step, summed over the kind's launches
    peak = None
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak = json.load(open(peaks_path)).get("bf16_tflops")
    achieved = kinds[top][1] / (top_ms / 1e3) / 1e12
    line = {"metric": "learned-initialiser training step TFLOP/s (algorithmic)", "unit": "TFLOP/s",
            "value": step_flops / (ms / 1e3) / 1e12, "n_gpus": 1, "steps": K, "warmup": max(args.warmup, 3),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 operands, f32 accumulate", "data": "synthetic",
            "config": {"workload": f"decoder_801x1024_b{B}", "batch": B, "layers": L, "width": 128,
                       "step": "decoder forward + backward (fixed dL/dy) + Adam + bf16 repack",
                       "l2": f"{L2_FLUSH_BYTES >> 20} MiB buffer written between timed steps (outside the events)"},
            "roofline": {"bound": "tensor", "kernel": kinds[top][0], "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if peak else None,
                         "peak_note": "measured bf16 burst (MEASURED_PEAKS.json), of measured",
                         "traffic": None},
            "kernel_ms_per_step": {k: v[0] / K for k, v in per_kind.items()},
            # per step: forward 1 pack + (L-1) GEMMs + 1 output layer; backward 1 + 2 (output layer)
            # + (L-1) x (2 weight-gradient + 2 bias) + (L-2) data-gradient; Adam 2 L + (2 L - 3) repacks
            "gpu_launches": K * ((L + 1) + 3 + 4 * (L - 1) + (L - 2) + 2 * L + (2 * L - 3)), "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    VARIANT["name"] = args.unpooled
    if args.workload == "long":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the chirps workload"}))
            return
        run_long(args)
        return
    if args.workload == "decoder":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the chirps workload"}))
            return
        run_decoder(args)
        return
    if args.workload == "initialiser":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the chirps workload"}))
            return
        run_initialiser(args)
        return
    if args.workload == "reflect":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the chirps workload"}))
            return
        run_reflect(args)
        return
    if args.workload == "reconstruct":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the chirps workload"}))
            return
        run_reconstruct(args)
        return
    if args.workload == "uneven64":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the chirps workload"}))
            return
        run_uneven(args)
        return
    wl = get_workload(WORKLOAD)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        if dist:
            dist.destroy_process_group()
        return

    from paper_2602_11896_gb300 import JTFSPlan, _native
    if args.batch:
        import dataclasses
        wl = dataclasses.replace(wl, batch=args.batch, target_seeds=wl.target_seeds[:args.batch],
                                 init_seeds=wl.init_seeds[:args.batch])
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    plan = JTFSPlan(**wl.params, batch=wl.batch, **variant_kw())
    targets, inits = rank_inputs(wl, rank)
    x = torch.tensor(targets, device=dev)
    y0 = torch.tensor(inits, device=dev)
    phi_t = plan.forward(x)
    y = y0.clone()
    m = torch.zeros_like(y)
    v = torch.zeros_like(y)
    loss = torch.empty(wl.batch, device=dev)
    ws = plan.workspace(dev)
    tuning = plan.tuning() if args.no_tune else plan.autotune(y0, phi_t)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    step_t = torch.ones(1, dtype=torch.int32, device=dev)   # Adam's step index, on the device

    def step():
        plan.metamer_step_counted(y, phi_t, m, v, step_t, 0.1, loss_out=loss, workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    lib = _native.load()
    # Per-stage kernel durations: the library's event hooks around its launches, on K eager steps
    # (outside the timed region; the kernels are the same ones the graph replays).
    stage_events = {}
    for st in range(6):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
        for e in evs:           # torch creates the CUDA event on its first record
            e.record()
        arr = (ctypes_void_p * (2 * K))(*[ctypes_void_p(e.cuda_event) for e in evs])
        _native.check(lib.jtfs_profile_stage(plan._h, st, arr, 2 * K), "jtfs_profile_stage")
        stage_events[st] = (evs, arr)
    for k in range(K):
        flush.fill_(float(k))
        step()
    torch.cuda.synchronize()
    for st in range(6):
        lib.jtfs_profile_stage(plan._h, st, None, 0)

    # The timed steps: one metamer step recorded in a CUDA graph and replayed (the step index lives on the
    # device, so every replay is the next Adam step).
    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            step()
    torch.cuda.current_stream().wait_stream(cap)
    graph.replay()              # warm replay
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    hist = torch.empty(K, wl.batch, device=dev)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for k in range(K):
        flush.fill_(float(k))
        starts[k].record()
        graph.replay()
        ends[k].record()
        hist[k].copy_(loss)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    device_status("timed steps")
    adam_steps = int(step_t.item()) - 1
    if dist:
        dist.barrier()
    ms, value = job_throughput(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world, wl.batch, wl.N, K,
                               dist if dist else None, dev)
    ms_per_step = ms / K

    # Per-stage average launch duration (CUDA events on the library's stream).
    stage_ms = {}
    for st, (evs, _) in stage_events.items():
        d = [evs[2 * i].elapsed_time(evs[2 * i + 1]) for i in range(K)] if tuning[3] or st < 4 else [0.0]
        stage_ms[st] = float(np.mean(d))
    # Kernels of the step: tensor-core frequential launches (stages 4, 5), the FFT kernels of the
    # remaining groups (stage 0 / 1 minus the tensor-core part), time pooling (2, 3).
    kern = {"k_freq_tc_adj (tensor-core adjoint of the second-order frequential scattering)": stage_ms[5],
            "k_freq_tc_fwd (tensor-core second-order frequential scattering + modulus + phi_F)": stage_ms[4],
            "k_freq_adj_ct (FFT adjoint, groups with n1max > 64)": stage_ms[1] - stage_ms[5],
            "k_freq_fwd_ct (FFT forward, groups with n1max > 64)": stage_ms[0] - stage_ms[4],
            "k_pool_fwd + k_pool_reduce (phi_T averaging)": stage_ms[2],
            "k_pool_adj (adjoint of phi_T averaging)": stage_ms[3]}
    dom = max(kern, key=kern.get)
    launch_ms = kern[dom]
    roofline = None
    if dom.startswith("k_freq_tc"):
        # The method's own work in these kernels is the FFT-count FLOPs of the frequential step (the
        # algorithmic count of the scope table: 5 n log2 n per complex FFT ...) on the columns of the groups
        # they take; they run it as dense BF16 GEMMs on the tensor cores, which is reported beside it as
        # useful dense FLOPs (one product per FP32-accurate product) and as issued FLOPs (three).
        adj = dom.startswith("k_freq_tc_adj")
        cols = wl.batch * sum(L2 for _, L2 in tc_groups(plan))
        flops = freq_flops_per_column(plan, adjoint=adj) * cols
        ach = flops / (launch_ms / 1e3) / 1e12
        issued = tc_tensor_flops(plan, adjoint=adj)
        t_ach = issued / (launch_ms / 1e3) / 1e12
        peak, peak_src = bf16_peak()
        per_clip = (DRAM_BYTES_PER_CLIP or {}).get(5 if adj else 4) if VARIANT["name"] == "none" else None
        roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP32_PEAK_TFLOPS,
                    "traffic": per_clip * wl.batch if per_clip is not None else None,
                    "traffic_note": "ncu dram bytes of the 1-clip capture x clips per launch",
                    "flops_per_launch": flops,
                    "flops_note": "algorithmic FFT-count FLOPs of the frequential step (5 n log2 n per complex "
                                  "FFT, 2 per filter product, 3 per modulus, 6 per modulus adjoint) on the "
                                  f"{cols} tensor-core columns of one launch",
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (no measured FP32 peak)",
                    "tensor": {"useful_flops_per_launch": issued / 3, "achieved": t_ach / 3, "peak": peak,
                               "frac": t_ach / 3 / peak, "issued_flops_per_launch": issued,
                               "issued_achieved": t_ach, "issued_frac": t_ach / peak, "peak_source": peak_src,
                               "note": "dense BF16 GEMM formulation (M = 128 columns per tile); each FP32-accurate "
                                       "product is three BF16 products (hi.hi + lo.hi + hi.lo)"},
                    "launch_ms": launch_ms,
                    "stage_ms": {k.split(" ")[0]: round(v, 4) for k, v in kern.items()},
                    "step_share": launch_ms / ms_per_step}
    elif dom.startswith("k_freq_"):
        adj = dom.startswith("k_freq_adj")
        cols = columns_per_launch(plan) - wl.batch * sum(L2 for _, L2 in (tc_groups(plan) if tuning[3] else []))
        flops = freq_flops_per_column(plan, adjoint=adj) * cols
        ach = flops / (launch_ms / 1e3) / 1e12
        per_clip = (DRAM_BYTES_PER_CLIP or {}).get(1 if adj else 0) if VARIANT["name"] == "none" else None
        roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                    "traffic": per_clip * wl.batch if per_clip is not None else None,
                    "flops_per_launch": flops, "launch_ms": launch_ms,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz (no measured FP32 peak)",
                    "stage_ms": {k.split(" ")[0]: round(v, 4) for k, v in kern.items()},
                    "step_share": launch_ms / ms_per_step}

    # Step-level HBM roofline: the compulsory bytes of a fused step against the measured copy bandwidth.
    if roofline is not None:
        cb = compulsory_bytes_per_clip(plan) * wl.batch
        hp, hsrc = hbm_peak()
        gbs = cb / (ms_per_step / 1e3) / 1e9
        roofline["step_hbm"] = {"compulsory_bytes_per_step": cb, "achieved_gbs": gbs, "peak_gbs": hp,
                                "frac": gbs / hp, "peak_source": hsrc,
                                "note": "x twice, U1 and dU1 written and read, Phi, target Phi, dy; the fused path "
                                        "does thousands of FLOPs per compulsory byte, so it is compute-bound and "
                                        "this fraction is small by design"}

    # End to end through the public API from pinned host memory.
    y_host = torch.tensor(inits, dtype=torch.float32).pin_memory()
    t_host = phi_t.cpu().pin_memory()
    l_host = torch.empty(wl.batch, dtype=torch.float32).pin_memory()
    yo_host = torch.empty_like(y_host).pin_memory()
    y_dev = torch.empty_like(y)
    t_dev = torch.empty_like(phi_t)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    Ke = max(1, min(K, 50))
    m.zero_()
    v.zero_()
    e0.record()
    for k in range(Ke):
        y_dev.copy_(y_host, non_blocking=True)
        t_dev.copy_(t_host, non_blocking=True)
        plan.metamer_step(y_dev, t_dev, m, v, k + 1, 0.1, loss_out=loss, workspace=ws)
        l_host.copy_(loss, non_blocking=True)
        yo_host.copy_(y_dev, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    device_status("end-to-end steps")
    e2e_ms, e2e_value = job_throughput(e0.elapsed_time(e1) / Ke, world, wl.batch, wl.N, 1, dist if dist else None, dev)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(y_host.numel() * 4 + t_host.numel() * 4),
           "d2h_bytes_per_step": int(l_host.numel() * 4 + yo_host.numel() * 4), "ms_per_step": e2e_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs = oracle_clip_seconds(wl, 0)
        cpu = {"value": wl.N / secs, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
               "sample": f"one {wl.N}-sample clip of {wl.name}: FP64 forward + loss + autograd adjoint, "
                         f"{secs:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {**config_dict(wl), "step": "metamer step (JTFS forward + loss + hand-written adjoint + "
                           "Adam, lr 0.1) replayed from a CUDA graph"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": (int(lib.jtfs_launch_count(plan._h, 3)) + 1) * K,
                "clocks": clk, "wall_s_timed": t_wall,
                "tuning": {"wide_forward_tiles": tuning[0], "pool_split": tuning[1], "fft_points_per_cta": tuning[2],
                           "tensor_core_frequential": tuning[3], "tensor_core_pooling": tuning[4],
                           "time_fft_engine": tuning[5] if len(tuning) > 5 else None},
                "metamer_loss": {"first_timed_step": float(hist[0].mean().item()),
                                 "last_timed_step": float(hist[-1].mean().item()),
                                 "adam_steps_before_last": adam_steps - 1},
                "timing": "each timed step is one replay of a CUDA graph of metamer_step_counted (forward + loss + "
                          "adjoint + Adam, step index on the device); stage_ms from the library's event hooks "
                          "on eager steps"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


from ctypes import c_void_p as ctypes_void_p  # noqa: E402

if __name__ == "__main__":
    main()
