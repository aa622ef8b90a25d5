"""Learned initialiser: a transposed-convolution decoder from Phi to a waveform.

Six transposed 1-D convolutions (stride 2, kernel 9; 128 channels; GELU
between layers) map the Phi of a clip, read as (rows of Phi) channels x
(frames) time steps and scaled per channel (``row_scale``), to
N = frames * 2^6 samples.  With T = 2^6 this is
exactly the clip length.  Operands are BF16 and products accumulate in FP32
on the tensor cores (library kernels ``jtfs_convt_*``: tcgen05 MMA with TMEM
accumulators fed by TMA); parameters are kept in FP32, updated with the
library's Adam kernel and repacked to BF16 after every update.  It is trained with the
JTFS loss itself: the gradient reaching the waveform comes from
``jtfs_loss_grad`` (the hand-written adjoint).  Its proposal replaces the
noise initialisation of metamer descent; plain noise initialisation stays the
fallback.
"""

from __future__ import annotations

import ctypes
import math
from ctypes import c_void_p
from typing import List, Optional, Tuple

import numpy as np
import torch

from . import _native

KERNEL = 9


def _p(t: torch.Tensor) -> c_void_p:
    return c_void_p(t.data_ptr())


def _s() -> c_void_p:
    return c_void_p(torch.cuda.current_stream().cuda_stream)


class Decoder:
    """Transposed-convolution decoder; see the module docstring.

    ``in_channels`` = rows of Phi, ``frames`` = Phi frames per clip; the output
    has frames * 2^layers samples.  Hidden width 128 (the tensor-core layers);
    activations are kept channels-last [B][T][C].
    """

    WIDTH = 128

    def __init__(self, in_channels: int, frames: int, channels: int = 128, layers: int = 6, seed: int = 0,
                 row_scale: Optional[np.ndarray] = None, device: str = "cuda"):
        if channels != self.WIDTH or layers < 2:
            raise ValueError("the decoder's hidden width is 128 and it has at least 2 layers")
        self._lib = _native.load()
        self.dims = [in_channels] + [channels] * (layers - 1) + [1]
        self.frames = frames
        self.layers = layers
        self.device = torch.device(device)
        self.cip0 = int(self._lib.jtfs_convt_padded_channels(in_channels))
        rng = np.random.default_rng(seed)
        self.w: List[torch.Tensor] = []
        self.b: List[torch.Tensor] = []
        for li in range(layers):
            ci, co = self.dims[li], self.dims[li + 1]
            std = math.sqrt(2.0 / (ci * KERNEL / 2.0))
            w = rng.standard_normal((ci, co, KERNEL)) * std
            self.w.append(torch.tensor(w, dtype=torch.float32, device=self.device))
            self.b.append(torch.zeros(co, dtype=torch.float32, device=self.device))
        scale = np.ones(in_channels) if row_scale is None else np.asarray(row_scale, dtype=np.float64)
        if scale.shape != (in_channels,):
            raise ValueError("row_scale must have one entry per input channel")
        self.row_scale = torch.tensor(scale, dtype=torch.float32, device=self.device)
        # When a list, every layer call appends (kind, layer, start event, end event) to it.
        self.profile: Optional[list] = None
        self._alloc_state()

    def _call(self, kind: str, li: int, name: str, *args) -> None:
        fn = getattr(self._lib, name)
        if self.profile is None:
            _native.check(fn(*args), name)
            return
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _native.check(fn(*args), name)
        e1.record()
        self.profile.append((kind, li, e0, e1))

    def _cip(self, li: int) -> int:
        return self.cip0 if li == 0 else self.WIDTH

    def _alloc_state(self):
        C = self.WIDTH
        self.wf = [torch.empty(2 * C, 5 * self._cip(li), dtype=torch.int16, device=self.device)
                   for li in range(self.layers - 1)]
        self.wd = [None] + [torch.empty(C, 9 * C, dtype=torch.int16, device=self.device)
                            for _ in range(1, self.layers - 1)]
        self.mw = [torch.zeros_like(w) for w in self.w]
        self.vw = [torch.zeros_like(w) for w in self.w]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.gw = [torch.zeros_like(w) for w in self.w]
        self.gb = [torch.zeros_like(b) for b in self.b]
        self.t = 0
        self._a: List[torch.Tensor] = []
        self._z: List[torch.Tensor] = []
        self._pack()

    def _pack(self):
        for li in range(self.layers - 1):
            wd = self.wd[li]
            _native.check(self._lib.jtfs_convt_pack_weights(_p(self.w[li]), _p(self.wf[li]),
                                                            _p(wd) if wd is not None else c_void_p(0),
                                                            self.dims[li], self.WIDTH, _s()),
                          "jtfs_convt_pack_weights")

    def layer_flops(self, batch: int) -> List[float]:
        """Algorithmic FLOPs of each layer's forward product: 2 x outputs x Co x Ci x 4.5
        (a kernel-9, stride-2 transposed convolution reaches each output from 4.5 taps on average)."""
        out, T = [], self.frames
        for li in range(self.layers):
            out.append(2.0 * batch * 2 * T * self.dims[li + 1] * self.dims[li] * KERNEL / 2.0)
            T *= 2
        return out

    @property
    def n_params(self) -> int:
        return sum(w.numel() for w in self.w) + sum(b.numel() for b in self.b)

    def forward(self, phi: torch.Tensor, keep: bool = True) -> torch.Tensor:
        """phi [B][in_channels][frames] float32 (CUDA) -> waveform [B][frames * 2^layers] float32."""
        if phi.dtype != torch.float32 or not phi.is_cuda or phi.dim() != 3 or phi.shape[1] != self.dims[0]:
            raise ValueError("phi must be a float32 CUDA tensor [B][in_channels][frames]")
        phi = phi.contiguous()
        B, _, T = phi.shape
        C = self.WIDTH
        x = torch.empty(B, T, self.cip0, dtype=torch.int16, device=self.device)
        _native.check(self._lib.jtfs_convt_pack_input(_p(phi), _p(self.row_scale), _p(x), B, self.dims[0], T, _s()),
                      "jtfs_convt_pack_input")
        a, zs = [x], []
        for li in range(self.layers - 1):
            z = torch.empty(B, 2 * T, C, dtype=torch.float32, device=self.device) if keep else None
            h = torch.empty(B, 2 * T, C, dtype=torch.int16, device=self.device)
            self._call("fwd", li, "jtfs_convt_forward", _p(a[-1]), _p(self.wf[li]), _p(self.b[li]),
                       _p(z) if z is not None else c_void_p(0), _p(h), B, self._cip(li), C, T, _s())
            if keep:
                a.append(h)
                zs.append(z)
            else:
                a = [h]
            T *= 2
        y = torch.empty(B, 2 * T, dtype=torch.float32, device=self.device)
        self._call("out_fwd", self.layers - 1, "jtfs_convt_out_forward", _p(a[-1]), _p(self.w[-1]), _p(self.b[-1]),
                   _p(y), B, C, T, _s())
        self._a, self._z = (a, zs) if keep else ([], [])
        return y

    def backward(self, dy: torch.Tensor) -> None:
        """Parameter gradients (written into gw, gb) from dL/dy [B][N] of the last forward."""
        if not self._a:
            raise RuntimeError("backward needs a forward with keep=True")
        C = self.WIDTH
        dy = dy.contiguous().float()
        B = dy.shape[0]
        L = self.layers
        T = self._a[-1].shape[1]  # input length of the output layer
        g32 = torch.empty(B, T, C, dtype=torch.float32, device=self.device)
        g16 = torch.empty(B, T, C, dtype=torch.int16, device=self.device)
        self._call("out_dx", L - 1, "jtfs_convt_out_backward_data", _p(dy), _p(self.w[-1]), _p(self._z[-1]), _p(g32),
                   _p(g16), B, C, T, _s())
        ws = torch.empty(max(int(self._lib.jtfs_convt_out_workspace_bytes(B, T)), 16), dtype=torch.uint8,
                         device=self.device)
        self._call("out_dw", L - 1, "jtfs_convt_out_backward_weight", _p(self._a[-1]), _p(dy), _p(self.gw[-1]),
                   _p(self.gb[-1]), B, C, T, _p(ws), _s())
        for li in reversed(range(L - 1)):
            T = self._a[li].shape[1]
            cip = self._cip(li)
            wsz = int(self._lib.jtfs_convt_weight_workspace_bytes(B, cip, C, T))
            ws = torch.empty(max(wsz, 16), dtype=torch.uint8, device=self.device)
            self._call("dw", li, "jtfs_convt_backward_weight", _p(self._a[li]), _p(g16), _p(self.gw[li]), B,
                       self.dims[li], cip, C, T, _p(ws), _s())
            rows = B * 2 * T
            ws = torch.empty(max(int(self._lib.jtfs_convt_bias_workspace_bytes(rows)), 16), dtype=torch.uint8,
                             device=self.device)
            self._call("db", li, "jtfs_convt_bias_grad", _p(g32), _p(self.gb[li]), rows, C, _p(ws), _s())
            if li > 0:
                n32 = torch.empty(B, T, C, dtype=torch.float32, device=self.device)
                n16 = torch.empty(B, T, C, dtype=torch.int16, device=self.device)
                self._call("dx", li, "jtfs_convt_backward_data", _p(g16), _p(self.wd[li]), _p(self._z[li - 1]),
                           _p(n32), _p(n16), B, C, C, T, _s())
                g32, g16 = n32, n16

    def step(self, lr: float) -> None:
        """One Adam update of every parameter from the gradients of the last backward."""
        self.t += 1
        for li in range(self.layers):
            _native.check(self._lib.jtfs_adam_update(_p(self.w[li]), _p(self.gw[li]), _p(self.mw[li]), _p(self.vw[li]),
                                                     c_void_p(0), self.w[li].numel(), float(lr), self.t, _s()),
                          "jtfs_adam_update")
            _native.check(self._lib.jtfs_adam_update(_p(self.b[li]), _p(self.gb[li]), _p(self.mb[li]), _p(self.vb[li]),
                                                     c_void_p(0), self.b[li].numel(), float(lr), self.t, _s()),
                          "jtfs_adam_update")
        self._pack()

    def check_errors(self) -> None:
        """Raise if a tensor-core kernel gave up waiting since the last check (synchronises)."""
        torch.cuda.synchronize()
        if self._lib.jtfs_decoder_error():
            raise RuntimeError("a decoder tensor-core kernel timed out on a barrier; its outputs are invalid")

    def state_dict(self) -> dict:
        d = {"dims": np.array(self.dims), "frames": np.array(self.frames), "row_scale": self.row_scale.cpu().numpy()}
        for li in range(self.layers):
            d[f"w{li}"] = self.w[li].cpu().numpy()
            d[f"b{li}"] = self.b[li].cpu().numpy()
        return d

    def save(self, path: str) -> None:
        np.savez(path, **self.state_dict())

    @classmethod
    def load(cls, path: str, device: str = "cuda") -> "Decoder":
        d = np.load(path)
        dims = [int(v) for v in d["dims"]]
        dec = cls(dims[0], int(d["frames"]), channels=dims[1], layers=len(dims) - 1, row_scale=d["row_scale"],
                  device=device)
        for li in range(dec.layers):
            dec.w[li] = torch.tensor(d[f"w{li}"], device=dec.device)
            dec.b[li] = torch.tensor(d[f"b{li}"], device=dec.device)
        dec._alloc_state()
        return dec


def phi_shape(plan) -> Tuple[int, int]:
    """(rows, frames) of one clip's Phi: every block of the layout is rows of N/T frames."""
    frames = plan.info["n_frames"]
    return plan.phi_size // frames, frames


def channel_scale(phi: torch.Tensor, floor: float = 1e-6) -> np.ndarray:
    """1 / RMS of each Phi row over a sample of clips ([B][rows][frames]); rows with
    RMS below ``floor`` times the largest are clamped there."""
    rms = phi.double().pow(2).mean(dim=(0, 2)).sqrt().cpu().numpy()
    return 1.0 / np.maximum(rms, floor * rms.max())


def train(dec: Decoder, plan, clips: torch.Tensor, steps: int, lr: float = 1e-3, lr_min: float = 1e-5,
          seed: int = 0, log_every: int = 50, log=print) -> List[Tuple[int, float]]:
    """Fit the decoder with the JTFS loss: for a batch of clips x, minimise
    sum ||Phi(dec(Phi x)) - Phi x||^2 (Eq. 5) over the decoder's parameters.

    ``clips`` [n][N] float32 on the device; ``plan`` a JTFSPlan whose batch is the
    training batch.  Cosine learning-rate decay from ``lr`` to ``lr_min``.
    Returns (step, mean loss per clip) every ``log_every`` steps.
    """
    B = plan.batch
    rows, frames = phi_shape(plan)
    g = torch.Generator(device="cpu").manual_seed(seed)
    order = torch.randperm(clips.shape[0], generator=g)
    pos, history, acc, cnt = 0, [], torch.zeros((), device=clips.device), 0
    ws = plan.workspace(clips.device)
    for it in range(steps):
        if pos + B > order.numel():
            order, pos = torch.randperm(clips.shape[0], generator=g), 0
        idx = order[pos:pos + B].to(clips.device)
        pos += B
        x = clips.index_select(0, idx)
        phi_t = plan.forward(x, workspace=ws)
        y = dec.forward(phi_t.view(B, rows, frames))
        loss, grad = plan.loss_grad(y, phi_t, workspace=ws)
        dec.backward(grad)
        dec.step(lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * it / max(steps - 1, 1))))
        acc += loss.sum()
        cnt += B
        if (it + 1) % log_every == 0 or it + 1 == steps:
            plan.check_status("decoder training")
            dec.check_errors()
            history.append((it + 1, float(acc) / cnt))
            log(f"step {it + 1}/{steps}  mean JTFS loss per clip {history[-1][1]:.5g}")
            acc.zero_()
            cnt = 0
    return history


def propose(dec: Decoder, plan, phi_target: torch.Tensor) -> torch.Tensor:
    """Initial waveforms [B][N] for the targets' Phi [B][phi_size]."""
    rows, frames = phi_shape(plan)
    return dec.forward(phi_target.view(-1, rows, frames), keep=False)


def descend(plan, y: torch.Tensor, phi_target: torch.Tensor, steps: int, lr: float) -> Tuple[torch.Tensor, float]:
    """``steps`` Adam metamer steps from y (modified in place); returns the loss of
    every step [steps][B] (loss of the iterate before each update) and the device
    time in ms."""
    m = torch.zeros_like(y)
    v = torch.zeros_like(y)
    losses = torch.empty(steps, plan.batch, device=y.device)
    ws = plan.workspace(y.device)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(steps):
        plan.metamer_step(y, phi_target, m, v, s + 1, lr, loss_out=losses[s], workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.check_status("Adam descent")
    return losses, e0.elapsed_time(e1)


def compare_initialisations(dec: Decoder, plan, phi_target: torch.Tensor, noise: torch.Tensor, steps: int = 200,
                            lr: float = 0.1) -> dict:
    """Metamers of one batch of targets from white noise and from the decoder's
    proposal, each refined by ``steps`` Adam steps.  Reports, for the proposal,
    the first step whose batch loss is at or below the noise run's final loss
    and the wall time to get there (decoder forward included)."""
    y_plain = noise.clone()
    loss_plain, ms_plain = descend(plan, y_plain, phi_target, steps, lr)
    final_plain = float(plan.loss_grad(y_plain, phi_target, need_grad=False)[0].sum())
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    y = propose(dec, plan, phi_target)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_decoder = e0.elapsed_time(e1)
    loss_learned, ms_learned = descend(plan, y, phi_target, steps, lr)
    final_learned = float(plan.loss_grad(y, phi_target, need_grad=False)[0].sum())
    curve = loss_learned.sum(dim=1).cpu().numpy()
    hit = np.nonzero(curve <= final_plain)[0]
    reached = int(hit[0]) if hit.size else None
    ms_step = ms_learned / steps
    return {
        "steps": steps, "lr": lr, "batch": plan.batch,
        "plain_initial_loss": float(loss_plain[0].sum()), "plain_final_loss": final_plain,
        "plain_ms": ms_plain,
        "learned_initial_loss": float(curve[0]), "learned_final_loss": final_learned,
        "decoder_ms": ms_decoder,
        "learned_steps_to_plain_final": reached,
        "learned_ms_to_plain_final": None if reached is None else ms_decoder + reached * ms_step,
        "plain_curve": loss_plain.sum(dim=1).cpu().tolist(), "learned_curve": curve.tolist(),
    }
