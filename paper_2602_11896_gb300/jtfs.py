"""PyTorch-facing API over the C ABI: plans, forward, adjoint, loss and Adam step.

PyTorch supplies device memory and the current CUDA stream; every step of the
transform runs in the library's CUDA kernels.  Inputs must be contiguous
float32 CUDA tensors of shape [batch, N]; anything else raises.
"""

from __future__ import annotations

import ctypes
from ctypes import c_double, c_float, c_int32, c_int64, c_void_p
from typing import Dict, Optional, Tuple

import numpy as np
import torch

from . import _native

INFO_KEYS = ("N", "J", "Q", "Q2", "J_fr", "Q_fr", "T", "F", "batch", "N1", "N2", "K", "N_fr",
             "log2_T", "log2_F", "R_out", "n_frames", "n_active", "phi_size")


def _ptr(t: torch.Tensor) -> c_void_p:
    return c_void_p(t.data_ptr())


def _stream() -> c_void_p:
    return c_void_p(torch.cuda.current_stream().cuda_stream)


class JTFSPlan:
    """A JTFS configuration (filterbanks, schedule, device tables) for one batch size.

    Parameters follow ``jtfs_plan`` in include/jtfs.h: N samples (power of
    two), J octaves, Q and Q2 filters per octave of the first- and
    second-order time filterbanks, J_fr and Q_fr of the frequential
    filterbank, time averaging T (power of two) and frequency averaging F.
    ``average_local`` / ``average_local_fr`` False give the unpooled outputs
    (JTFS_PLAN_UNPOOLED_T / _F in include/jtfs.h).
    """

    def __init__(self, N: int, J: int, Q: int, Q2: int, J_fr: int, Q_fr: int, T: int, F: int,
                 batch: int = 1, host_only: bool = False, average_local: bool = True,
                 average_local_fr: bool = True):
        lib = _native.load()
        h = c_void_p()
        flags = ((_native.PLAN_HOST_ONLY if host_only else 0) | (0 if average_local else _native.PLAN_UNPOOLED_T)
                 | (0 if average_local_fr else _native.PLAN_UNPOOLED_F))
        if not host_only and not torch.cuda.is_available():
            raise RuntimeError("JTFSPlan needs a CUDA device (or host_only=True for inspection)")
        _native.check(lib.jtfs_plan(ctypes.byref(h), N, J, Q, Q2, J_fr, Q_fr, T, F, batch, flags),
                      "jtfs_plan")
        self._h = h
        self._lib = lib
        self.host_only = host_only
        self.average_local = average_local
        self.average_local_fr = average_local_fr
        buf = (c_int64 * len(INFO_KEYS))()
        n = lib.jtfs_plan_info(h, buf, len(INFO_KEYS))
        if n < len(INFO_KEYS):
            raise RuntimeError("jtfs_plan_info returned too few values")
        self.info: Dict[str, int] = {k: int(buf[i]) for i, k in enumerate(INFO_KEYS)}
        self.N = self.info["N"]
        self.batch = self.info["batch"]
        self.phi_size = int(lib.jtfs_phi_size(h))
        self.workspace_bytes = int(lib.jtfs_workspace_bytes(h))
        self._ws: Optional[torch.Tensor] = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.jtfs_plan_destroy(h)
            self._h = None

    # -- inspection -------------------------------------------------------
    def filters(self, which: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(xi, sigma, j) of filterbank `which` (0 psi1, 1 psi2, 2 psi_fr, 3 phi_T/phi_F)."""
        n = self._lib.jtfs_plan_filters(self._h, which, None, None, None, 0)
        _native.check(0 if n >= 0 else n, "jtfs_plan_filters")
        xi = (c_double * n)()
        sg = (c_double * n)()
        jj = (c_int32 * n)()
        self._lib.jtfs_plan_filters(self._h, which, xi, sg, jj, n)
        return np.array(xi[:]), np.array(sg[:]), np.array(jj[:], dtype=np.int64)

    def path_meta(self) -> Dict[str, np.ndarray]:
        """Per path of Phi, in order: order (0, 1, 2), n2, beta_idx, spin and offset (see jtfs_path_meta)."""
        n = int(self._lib.jtfs_path_meta(self._h, None, None, None, None, None))
        _native.check(0 if n >= 0 else n, "jtfs_path_meta")
        arrs = [(c_int32 * n)() for _ in range(4)]
        off = (c_int64 * n)()
        self._lib.jtfs_path_meta(self._h, *arrs, off)
        keys = ("order", "n2", "beta_idx", "spin")
        out = {k: np.array(a[:], dtype=np.int64) for k, a in zip(keys, arrs)}
        out["offset"] = np.array(off[:], dtype=np.int64)
        return out

    def schedule(self, which: int) -> np.ndarray:
        """One of the plan's work tables (see jtfs_plan_schedule): which = 0 U1-row gradient blocks
        [n][row, block, log2 length]; 1 banded phi_T adjoint CTAs [n][clip, group, first row, first sample];
        2 per active group [n_active][s2, rows, n1max, W, band samples per CTA, forward KA, adjoint KA]."""
        n = int(self._lib.jtfs_plan_schedule(self._h, which, None, 0))
        _native.check(0 if n >= 0 else n, "jtfs_plan_schedule")
        buf = (c_int64 * max(n, 1))()
        self._lib.jtfs_plan_schedule(self._h, which, buf, n)
        return np.array(buf[:n], dtype=np.int64).reshape(-1, (3, 4, 7)[which])

    # -- tuning -----------------------------------------------------------
    def tuning(self) -> Tuple[int, int, int, int, int, int]:
        """(wide forward tiles, pooling split, small-FFT points per CTA, tensor-core frequential path,
        tensor-core time pooling, radix-16 / cluster time-axis FFT engine) in use."""
        buf = (c_int64 * 6)()
        self._lib.jtfs_get_tuning(self._h, buf, 6)
        return tuple(int(buf[i]) for i in range(6))

    def set_tuning(self, choice) -> None:
        """Apply 3 to 6 choices (see ``tuning``); choices not given are unchanged."""
        vals = [int(c) for c in choice]
        buf = (c_int64 * len(vals))(*vals)
        n = self._lib.jtfs_set_tuning(self._h, buf, len(vals))
        _native.check(0 if n >= 0 else n, "jtfs_set_tuning")

    def tc_table(self, which: int) -> np.ndarray:
        """Operand table of the tensor-core frequential kernels (float, hi + lo of the BF16 split).

        which = 0: H [rows][128] (row 2 (off_beta + r) + x, column 2 n + y); which = 1: P [lF + 1][R_out][N_fr].
        """
        n = int(self._lib.jtfs_tc_table(self._h, which, None, 0))
        _native.check(0 if n >= 0 else n, "jtfs_tc_table")
        buf = (c_float * n)()
        self._lib.jtfs_tc_table(self._h, which, buf, n)
        a = np.frombuffer(buf, dtype=np.float32).copy()
        if which == 0:
            return a.reshape(-1, 128)
        return a.reshape(self.info["log2_F"] + 1, self.info["R_out"], self.info["N_fr"])

    def _tune_key(self) -> str:
        name = torch.cuda.get_device_name() if torch.cuda.is_available() else "host"
        return f"{name}|" + ",".join(f"{k}={self.info[k]}" for k in INFO_KEYS[:9])

    def autotune(self, y: torch.Tensor, phi_target: torch.Tensor,
                 cache: Optional[str] = None) -> Tuple[int, ...]:
        """Pick the fastest execution choices for this plan by timing jtfs_loss_grad on (y, phi_target).

        With ``cache`` (default: the JTFS_TUNE_CACHE environment variable) the choices are read
        from / written to that JSON file, keyed by device name and plan parameters.
        """
        import json
        import os
        path = cache if cache is not None else os.environ.get("JTFS_TUNE_CACHE")
        key = self._tune_key()
        if path and os.path.exists(path):
            try:
                table = json.load(open(path))
            except (OSError, ValueError):
                table = {}
            if key in table:
                self.set_tuning(table[key])
                return self.tuning()
        self._check(y, self.N, "y")
        self._check(phi_target, self.phi_size, "phi_target")
        loss = torch.empty(self.batch, device=y.device)
        dy = torch.empty_like(y)
        ws = self.workspace(y.device)
        buf = (c_int64 * 6)()
        n = self._lib.jtfs_autotune(self._h, _ptr(y), _ptr(phi_target), _ptr(loss), _ptr(dy), _ptr(ws), _stream(),
                                    buf, 6)
        _native.check(0 if n >= 0 else n, "jtfs_autotune")
        choice = [int(buf[i]) for i in range(6)]
        if path:
            table = {}
            if os.path.exists(path):
                try:
                    table = json.load(open(path))
                except (OSError, ValueError):
                    table = {}
            table[key] = choice
            with open(path, "w") as f:
                json.dump(table, f, indent=1)
        return tuple(choice)

    # -- compute ----------------------------------------------------------
    def workspace(self, device: Optional[torch.device] = None) -> torch.Tensor:
        """Device scratch of jtfs_workspace_bytes(), cached (calls on one stream serialise)."""
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self._ws is None or self._ws.device != dev:
            self._ws = torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=dev)
        return self._ws

    def _check(self, t: torch.Tensor, cols: int, name: str) -> None:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor (the library has no CPU path)")
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError(f"{name} must be contiguous float32")
        if tuple(t.shape) != (self.batch, cols):
            raise ValueError(f"{name} must have shape {(self.batch, cols)}, got {tuple(t.shape)}")

    def forward(self, x: torch.Tensor, out: Optional[torch.Tensor] = None,
                workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        self._check(x, self.N, "x")
        phi = out if out is not None else torch.empty(self.batch, self.phi_size, device=x.device)
        ws = workspace if workspace is not None else self.workspace(x.device)
        _native.check(self._lib.jtfs_forward(self._h, _ptr(x), _ptr(phi), _ptr(ws), _stream()), "jtfs_forward")
        return phi

    def forward_noalloc(self, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Forward transform without a workspace (fixed 32 MiB library scratch).

        For callers that cannot allocate device memory; see
        jtfs_forward_noalloc in include/jtfs.h for the limits and the
        sharing rule (calls overlapping on the GPU race on the scratch).
        """
        self._check(x, self.N, "x")
        phi = out if out is not None else torch.empty(self.batch, self.phi_size, device=x.device)
        _native.check(self._lib.jtfs_forward_noalloc(self._h, _ptr(x), _ptr(phi), _stream()),
                      "jtfs_forward_noalloc")
        return phi

    def backward(self, x: torch.Tensor, dphi: torch.Tensor, out: Optional[torch.Tensor] = None,
                 workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        self._check(x, self.N, "x")
        self._check(dphi, self.phi_size, "dphi")
        dx = out if out is not None else torch.empty_like(x)
        ws = workspace if workspace is not None else self.workspace(x.device)
        _native.check(self._lib.jtfs_backward(self._h, _ptr(x), _ptr(dphi), _ptr(dx), _ptr(ws), _stream()),
                      "jtfs_backward")
        return dx

    def loss_grad(self, y: torch.Tensor, phi_target: torch.Tensor, need_grad: bool = True,
                  loss_out: Optional[torch.Tensor] = None, grad_out: Optional[torch.Tensor] = None,
                  workspace: Optional[torch.Tensor] = None) -> Tuple[torch.Tensor, Optional[torch.Tensor]]:
        self._check(y, self.N, "y")
        self._check(phi_target, self.phi_size, "phi_target")
        loss = loss_out if loss_out is not None else torch.empty(self.batch, device=y.device)
        dy = (grad_out if grad_out is not None else torch.empty_like(y)) if need_grad else None
        ws = workspace if workspace is not None else self.workspace(y.device)
        _native.check(self._lib.jtfs_loss_grad(self._h, _ptr(y), _ptr(phi_target), _ptr(loss),
                                               _ptr(dy) if dy is not None else c_void_p(0), _ptr(ws),
                                               _stream()), "jtfs_loss_grad")
        return loss, dy

    def metamer_step(self, y: torch.Tensor, phi_target: torch.Tensor, adam_m: torch.Tensor,
                     adam_v: torch.Tensor, step: int, lr: float, loss_out: Optional[torch.Tensor] = None,
                     workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        for t, n in ((y, "y"), (adam_m, "adam_m"), (adam_v, "adam_v")):
            self._check(t, self.N, n)
        self._check(phi_target, self.phi_size, "phi_target")
        loss = loss_out if loss_out is not None else torch.empty(self.batch, device=y.device)
        ws = workspace if workspace is not None else self.workspace(y.device)
        _native.check(self._lib.metamer_step(self._h, _ptr(y), _ptr(phi_target), _ptr(adam_m), _ptr(adam_v),
                                             int(step), float(lr), _ptr(loss), _ptr(ws), _stream()),
                      "metamer_step")
        return loss

    def metamer_step_counted(self, y: torch.Tensor, phi_target: torch.Tensor, adam_m: torch.Tensor,
                             adam_v: torch.Tensor, step: torch.Tensor, lr: float,
                             loss_out: Optional[torch.Tensor] = None,
                             workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        """metamer_step with the Adam step index in a 1-element int32 CUDA tensor (1-based,
        incremented on the device), so that the call can be captured in a CUDA graph."""
        for t, n in ((y, "y"), (adam_m, "adam_m"), (adam_v, "adam_v")):
            self._check(t, self.N, n)
        self._check(phi_target, self.phi_size, "phi_target")
        if (not isinstance(step, torch.Tensor) or not step.is_cuda or step.dtype != torch.int32
                or step.numel() != 1):
            raise TypeError("step must be a 1-element int32 CUDA tensor")
        loss = loss_out if loss_out is not None else torch.empty(self.batch, device=y.device)
        ws = workspace if workspace is not None else self.workspace(y.device)
        _native.check(self._lib.metamer_step_counted(self._h, _ptr(y), _ptr(phi_target), _ptr(adam_m),
                                                     _ptr(adam_v), _ptr(step), float(lr), _ptr(loss), _ptr(ws),
                                                     _stream()), "metamer_step_counted")
        return loss

    @staticmethod
    def check_status(what: str = "JTFS", allow_nonfinite: bool = False) -> None:
        """Synchronise the current stream and raise DeviceStatusError if, since the last check, a
        tensor-core kernel gave up on a barrier (its outputs are invalid) or, unless
        ``allow_nonfinite``, a loss was NaN / Inf."""
        code = _native.status(torch.cuda.current_stream().cuda_stream)
        if code == _native.ERR_NONFINITE and allow_nonfinite:
            return
        if code in (_native.ERR_TIMEOUT, _native.ERR_NONFINITE):
            raise _native.DeviceStatusError(code, what)
        _native.check(code, what)

    # -- reconstruction variant of §2.3 --------------------------------------
    def init_gains(self) -> np.ndarray:
        """Per first-order filter, the band gain of the coloured initialisation times 2^(lT-k1)."""
        n = int(self._lib.jtfs_init_gains(self._h, None, 0))
        _native.check(0 if n >= 0 else n, "jtfs_init_gains")
        buf = (c_float * n)()
        self._lib.jtfs_init_gains(self._h, buf, n)
        return np.frombuffer(buf, dtype=np.float32).copy()

    def coloured_init(self, x: torch.Tensor, w_noise: torch.Tensor, out: Optional[torch.Tensor] = None,
                      workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Coloured Gaussian noise following the target's S1 (jtfs_coloured_init), energy of x."""
        self._check(x, self.N, "x")
        self._check(w_noise, self.N, "w_noise")
        y0 = out if out is not None else torch.empty_like(x)
        ws = workspace if workspace is not None else self.workspace(x.device)
        _native.check(self._lib.jtfs_coloured_init(self._h, _ptr(x), _ptr(w_noise), _ptr(y0), _ptr(ws), _stream()),
                      "jtfs_coloured_init")
        return y0

    def momentum_state(self, mu0: float = 0.1, device=None) -> Dict[str, torch.Tensor]:
        """Zero momentum, zero stored gradient and per-clip (mu0, +inf, 0, 0) bold-driver state."""
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        st = torch.zeros(self.batch, 4, device=dev)
        st[:, 0] = float(mu0)
        st[:, 1] = float("inf")
        return {"u": torch.zeros(self.batch, self.N, device=dev), "g_acc": torch.zeros(self.batch, self.N, device=dev),
                "state": st}

    def metamer_step_momentum(self, y: torch.Tensor, phi_target: torch.Tensor, opt: Dict[str, torch.Tensor],
                              m: float = 0.9, loss_out: Optional[torch.Tensor] = None,
                              workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        """One momentum / bold-driver evaluation (metamer_step_momentum); ``opt`` from ``momentum_state``."""
        self._check(y, self.N, "y")
        self._check(opt["u"], self.N, "u")
        self._check(opt["g_acc"], self.N, "g_acc")
        self._check(opt["state"], 4, "state")
        self._check(phi_target, self.phi_size, "phi_target")
        loss = loss_out if loss_out is not None else torch.empty(self.batch, device=y.device)
        ws = workspace if workspace is not None else self.workspace(y.device)
        _native.check(self._lib.metamer_step_momentum(self._h, _ptr(y), _ptr(phi_target), _ptr(opt["u"]),
                                                      _ptr(opt["g_acc"]), _ptr(opt["state"]), float(m), _ptr(loss),
                                                      _ptr(ws), _stream()), "metamer_step_momentum")
        return loss


def momentum_update(y: torch.Tensor, opt: Dict[str, torch.Tensor], grad: torch.Tensor, loss: torch.Tensor,
                    m: float = 0.9) -> None:
    """The update of metamer_step_momentum alone (jtfs_momentum_update), from a given loss and gradient."""
    B, n = y.shape
    for t, name in ((y, "y"), (opt["u"], "u"), (opt["g_acc"], "g_acc"), (grad, "grad")):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != (B, n):
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor of shape {(B, n)}")
    st = opt["state"]
    if not st.is_cuda or st.dtype != torch.float32 or tuple(st.shape) != (B, 4) or not st.is_contiguous():
        raise TypeError("state must be a contiguous float32 CUDA tensor of shape (batch, 4)")
    if not loss.is_cuda or loss.dtype != torch.float32 or loss.numel() != B:
        raise TypeError("loss must be a float32 CUDA tensor of batch elements")
    lib = _native.load()
    _native.check(lib.jtfs_momentum_update(_ptr(y), _ptr(opt["u"]), _ptr(opt["g_acc"]), _ptr(grad), _ptr(st),
                                           _ptr(loss), B, n, float(m), _stream()), "jtfs_momentum_update")


class JTFSBatch:
    """Clips of uneven lengths solved together (jtfs_batch_* in include/jtfs.h).

    Each clip is zero-padded to the next power of two >= max(L, T) and its Phi
    cropped to ceil(L/T) frames per row; with ``boundary="reflect"`` it is
    mirrored on both sides instead and the frames over the clip are kept (see
    jtfs_batch_create).  Samples and Phi are packed: ``sample_offsets`` /
    ``phi_offsets`` give each clip's slice.
    """

    def __init__(self, lengths, J: int, Q: int, Q2: int, J_fr: int, Q_fr: int, T: int, F: int,
                 host_only: bool = False, boundary: str = "zero"):
        if boundary not in ("zero", "reflect"):
            raise ValueError("boundary must be 'zero' or 'reflect'")
        lib = _native.load()
        if not host_only and not torch.cuda.is_available():
            raise RuntimeError("JTFSBatch needs a CUDA device (or host_only=True for inspection)")
        lens = [int(v) for v in lengths]
        arr = (c_int64 * len(lens))(*lens)
        h = c_void_p()
        flags = (_native.PLAN_HOST_ONLY if host_only else 0) | (_native.BATCH_REFLECT if boundary == "reflect" else 0)
        _native.check(lib.jtfs_batch_create(ctypes.byref(h), arr, len(lens), J, Q, Q2, J_fr, Q_fr, T, F, flags),
                      "jtfs_batch_create")
        self.boundary = boundary
        self._h, self._lib = h, lib
        so = (c_int64 * (len(lens) + 1))()
        po = (c_int64 * (len(lens) + 1))()
        lib.jtfs_batch_layout(h, so, po)
        self.lengths = lens
        self.sample_offsets = [int(v) for v in so]
        self.phi_offsets = [int(v) for v in po]
        self.n_samples = self.sample_offsets[-1]
        self.phi_size = self.phi_offsets[-1]
        self.workspace_bytes = int(lib.jtfs_batch_workspace_bytes(h))
        self._ws: Optional[torch.Tensor] = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.jtfs_batch_destroy(h)
            self._h = None

    def workspace(self, device=None) -> torch.Tensor:
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self._ws is None or self._ws.device != dev:
            self._ws = torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=dev)
        return self._ws

    @staticmethod
    def _need(t: torch.Tensor, n: int, name: str, dtype=torch.float32) -> None:
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
        if t.numel() != n:
            raise ValueError(f"{name} must have {n} elements, got {t.numel()}")

    def pack(self, clips) -> torch.Tensor:
        """Concatenate per-clip 1-D tensors (lengths must match) into packed samples."""
        for c, L in zip(clips, self.lengths):
            if c.numel() != L:
                raise ValueError("clip length does not match the batch")
        return torch.cat([c.reshape(-1) for c in clips]).contiguous()

    def forward(self, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        self._need(x, self.n_samples, "x")
        phi = out if out is not None else torch.empty(self.phi_size, device=x.device)
        ws = self.workspace(x.device)
        _native.check(self._lib.jtfs_batch_forward(self._h, _ptr(x), _ptr(phi), _ptr(ws), _stream()),
                      "jtfs_batch_forward")
        return phi

    def metamer_step(self, y: torch.Tensor, phi_target: torch.Tensor, adam_m: torch.Tensor,
                     adam_v: torch.Tensor, step: torch.Tensor, lr: float,
                     loss_out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """One Adam step on every clip; `step` is a 1-element int32 CUDA tensor (1-based,
        incremented on the device), so the call can be captured in a CUDA graph."""
        for t, n in ((y, "y"), (adam_m, "adam_m"), (adam_v, "adam_v")):
            self._need(t, self.n_samples, n)
        self._need(phi_target, self.phi_size, "phi_target")
        self._need(step, 1, "step", torch.int32)
        loss = loss_out if loss_out is not None else torch.empty(len(self.lengths), device=y.device)
        ws = self.workspace(y.device)
        _native.check(self._lib.jtfs_batch_metamer_step(self._h, _ptr(y), _ptr(phi_target), _ptr(adam_m),
                                                        _ptr(adam_v), _ptr(step), float(lr), _ptr(loss),
                                                        _ptr(ws), _stream()), "jtfs_batch_metamer_step")
        return loss


class _JTFSFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, plan: JTFSPlan) -> torch.Tensor:  # type: ignore[override]
        ctx.plan = plan
        ctx.save_for_backward(x)
        return plan.forward(x.contiguous())

    @staticmethod
    def backward(ctx, dphi: torch.Tensor):  # type: ignore[override]
        (x,) = ctx.saved_tensors
        return ctx.plan.backward(x.contiguous(), dphi.contiguous()), None


def jtfs(x: torch.Tensor, plan: JTFSPlan) -> torch.Tensor:
    """Phi(x) with a hand-written adjoint as its autograd backward (recomputes U1)."""
    return _JTFSFunction.apply(x, plan)
