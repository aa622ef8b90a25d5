"""Learned initialiser: a transposed-convolution decoder from Phi to a waveform.

Six transposed 1-D convolutions (stride 2, kernel 9; 128 channels; GELU
between layers) map the Phi of a clip, read as (rows of Phi) channels x
(frames) time steps, to N = frames * 2^6 samples.  With T = 2^6 this is
exactly the clip length.  Operands are BF16 and products accumulate in FP32
on the tensor cores (library kernels ``jtfs_convt_*``); parameters are kept
in FP32 and updated with the library's Adam kernel.  It is trained with the
JTFS loss itself: the gradient reaching the waveform comes from
``jtfs_loss_grad`` (the hand-written adjoint).  Its proposal replaces the
noise initialisation of metamer descent; plain noise initialisation stays the
fallback.
"""

from __future__ import annotations

import ctypes
import math
from ctypes import c_void_p
from typing import List, Optional

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
    has frames * 2^layers samples.
    """

    def __init__(self, in_channels: int, frames: int, channels: int = 128, layers: int = 6, seed: int = 0,
                 in_scale: Optional[np.ndarray] = None, device: str = "cuda"):
        self._lib = _native.load()
        self.dims = [in_channels] + [channels] * (layers - 1) + [1]
        self.frames = frames
        self.layers = layers
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        self.w: List[torch.Tensor] = []
        self.b: List[torch.Tensor] = []
        for li in range(layers):
            ci, co = self.dims[li], self.dims[li + 1]
            std = math.sqrt(2.0 / (ci * KERNEL / 2.0))
            w = rng.standard_normal((ci, co, KERNEL)) * std
            if li == 0 and in_scale is not None:
                w = w / np.asarray(in_scale, dtype=np.float64)[:, None, None]
            self.w.append(torch.tensor(w, dtype=torch.float32, device=self.device))
            self.b.append(torch.zeros(co, dtype=torch.float32, device=self.device))
        self._alloc_state()

    def _alloc_state(self):
        self.wb = [torch.empty(w.shape, dtype=torch.int16, device=self.device) for w in self.w]
        self.mw = [torch.zeros_like(w) for w in self.w]
        self.vw = [torch.zeros_like(w) for w in self.w]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.gw = [torch.zeros_like(w) for w in self.w]
        self.gb = [torch.zeros_like(b) for b in self.b]
        self.t = 0
        self._sync_bf16()

    def _sync_bf16(self):
        for w, wb in zip(self.w, self.wb):
            _native.check(self._lib.jtfs_cast_bf16(_p(w), _p(wb), w.numel(), _s()), "jtfs_cast_bf16")

    @property
    def n_params(self) -> int:
        return sum(w.numel() for w in self.w) + sum(b.numel() for b in self.b)

    def forward(self, phi: torch.Tensor, keep: bool = True) -> torch.Tensor:
        """phi [B][in_channels][frames] float32 (CUDA) -> waveform [B][frames * 2^layers] float32."""
        if phi.dtype != torch.float32 or not phi.is_cuda or phi.dim() != 3 or phi.shape[1] != self.dims[0]:
            raise ValueError("phi must be a float32 CUDA tensor [B][in_channels][frames]")
        phi = phi.contiguous()
        B, _, T = phi.shape
        h = torch.empty(phi.shape, dtype=torch.int16, device=self.device)
        _native.check(self._lib.jtfs_cast_bf16(_p(phi), _p(h), phi.numel(), _s()), "jtfs_cast_bf16")
        self._h, self._z = [h], []
        for li in range(self.layers):
            ci, co = self.dims[li], self.dims[li + 1]
            z = torch.empty(B, co, 2 * T, dtype=torch.float32, device=self.device)
            _native.check(self._lib.jtfs_convt_forward(_p(h), _p(self.wb[li]), _p(self.b[li]), _p(z), B, ci, co, T,
                                                       _s()), "jtfs_convt_forward")
            T *= 2
            if li + 1 < self.layers:
                h = torch.empty(z.shape, dtype=torch.int16, device=self.device)
                _native.check(self._lib.jtfs_gelu_forward(_p(z), _p(h), z.numel(), _s()), "jtfs_gelu_forward")
                if keep:
                    self._z.append(z)
                    self._h.append(h)
            else:
                out = z
        if not keep:
            self._h, self._z = [], []
        return out.reshape(B, T)

    def backward(self, dy: torch.Tensor) -> None:
        """Accumulate parameter gradients (into gw, gb) from dL/dy [B][N] of the last forward."""
        if not self._h:
            raise RuntimeError("backward needs a forward with keep=True")
        B = dy.shape[0]
        dz = dy.reshape(B, 1, -1).contiguous().float()
        for li in reversed(range(self.layers)):
            ci, co = self.dims[li], self.dims[li + 1]
            T = dz.shape[-1] // 2
            dzb = torch.empty(dz.shape, dtype=torch.int16, device=self.device)
            _native.check(self._lib.jtfs_cast_bf16(_p(dz), _p(dzb), dz.numel(), _s()), "jtfs_cast_bf16")
            ws_bytes = self._lib.jtfs_convt_weight_workspace_bytes(B, ci, co, T)
            ws = torch.empty(max(int(ws_bytes), 4), dtype=torch.uint8, device=self.device)
            _native.check(self._lib.jtfs_convt_backward_weight(_p(self._h[li]), _p(dzb), _p(dz), _p(self.gw[li]),
                                                               _p(self.gb[li]), B, ci, co, T, _p(ws), _s()),
                          "jtfs_convt_backward_weight")
            if li > 0:
                dh = torch.empty(B, ci, T, dtype=torch.float32, device=self.device)
                _native.check(self._lib.jtfs_convt_backward_data(_p(dzb), _p(self.wb[li]), _p(dh), B, ci, co, T, _s()),
                              "jtfs_convt_backward_data")
                z = self._z[li - 1]
                dz = torch.empty_like(dh)
                _native.check(self._lib.jtfs_gelu_backward(_p(dh), _p(z), _p(dz), dh.numel(), _s()),
                              "jtfs_gelu_backward")

    def step(self, lr: float) -> None:
        """One Adam update of every parameter from the gradients of the last backward."""
        self.t += 1
        for li in range(self.layers):
            _native.check(self._lib.jtfs_adam_update(_p(self.w[li]), _p(self.gw[li]), _p(self.mw[li]), _p(self.vw[li]),
                                                     _p(self.wb[li]), self.w[li].numel(), float(lr), self.t, _s()),
                          "jtfs_adam_update")
            _native.check(self._lib.jtfs_adam_update(_p(self.b[li]), _p(self.gb[li]), _p(self.mb[li]), _p(self.vb[li]),
                                                     c_void_p(0), self.b[li].numel(), float(lr), self.t, _s()),
                          "jtfs_adam_update")

    def state_dict(self) -> dict:
        d = {"dims": np.array(self.dims), "frames": np.array(self.frames)}
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
        dec = cls(dims[0], int(d["frames"]), channels=dims[1], layers=len(dims) - 1, device=device)
        for li in range(dec.layers):
            dec.w[li] = torch.tensor(d[f"w{li}"], device=dec.device)
            dec.b[li] = torch.tensor(d[f"b{li}"], device=dec.device)
        dec._alloc_state()
        return dec
