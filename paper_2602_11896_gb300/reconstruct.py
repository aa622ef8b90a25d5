"""The reconstruction variant of §2.3 against the Adam descent, on one batch of targets.

§2.3 starts from coloured Gaussian noise following the target's S1 and
refines it by momentum updates (m = 0.9) whose step size starts at 0.1 and
follows the bold-driver rule; the library's other workloads start from white
noise and use Adam (lr 0.1).  ``compare_reconstruction`` runs every pairing of
the two starts and the two optimisers for the same number of gradient
evaluations and reports loss against device time.  Every step runs in the
library's kernels (jtfs_coloured_init, metamer_step_momentum, metamer_step).

Loss curves are per-clip running minima (the iterate one would keep) summed
over the batch: for the bold driver this is the loss at the last accepted
point, since rejected evaluations are never kept.
"""

from __future__ import annotations

from typing import Dict, Tuple

import numpy as np
import torch


def _timed(fn) -> float:
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def descend_adam(plan, y: torch.Tensor, phi_target: torch.Tensor, steps: int, lr: float = 0.1
                 ) -> Tuple[torch.Tensor, float]:
    """``steps`` Adam metamer steps from y (in place): per-step losses [steps][B] and device ms."""
    m = torch.zeros_like(y)
    v = torch.zeros_like(y)
    losses = torch.empty(steps, plan.batch, device=y.device)
    ws = plan.workspace(y.device)

    def run():
        for s in range(steps):
            plan.metamer_step(y, phi_target, m, v, s + 1, lr, loss_out=losses[s], workspace=ws)
    ms = _timed(run)
    plan.check_status("Adam descent")
    return losses, ms


def descend_momentum(plan, y: torch.Tensor, phi_target: torch.Tensor, steps: int, mu0: float = 0.1,
                     m: float = 0.9) -> Tuple[torch.Tensor, float, torch.Tensor]:
    """``steps`` momentum / bold-driver evaluations from y (in place): per-evaluation losses
    [steps][B], device ms, and the final per-clip state (mu, E_acc, accepted, evaluations)."""
    opt = plan.momentum_state(mu0=mu0, device=y.device)
    losses = torch.empty(steps, plan.batch, device=y.device)
    ws = plan.workspace(y.device)

    def run():
        for s in range(steps):
            plan.metamer_step_momentum(y, phi_target, opt, m=m, loss_out=losses[s], workspace=ws)
    ms = _timed(run)
    # A NaN loss is one the bold driver rejects (the step halves), not an error.
    plan.check_status("momentum descent", allow_nonfinite=True)
    return losses, ms, opt["state"]


def _curve(losses: torch.Tensor) -> np.ndarray:
    """Batch sum of the per-clip running minimum."""
    return torch.cummin(losses, dim=0).values.sum(dim=1).cpu().numpy().astype(np.float64)


def compare_reconstruction(plan, x: torch.Tensor, phi_target: torch.Tensor, noise: torch.Tensor,
                           steps: int = 200, lr: float = 0.1, mu0: float = 0.1, m: float = 0.9) -> Dict:
    """Four arms of ``steps`` gradient evaluations each: {white noise, coloured noise} x {Adam, momentum}.

    For every arm: the loss curve, device time of the descent (and of the
    coloured initialisation, counted in the wall time of its arms), and the
    first evaluation at which the arm reaches the white-noise Adam run's
    final loss, with the wall time to get there.
    """
    out: Dict = {"steps": steps, "lr": lr, "mu0": mu0, "m": m, "batch": plan.batch, "arms": {}}
    y_col = torch.empty_like(noise)
    init_ms = _timed(lambda: plan.coloured_init(x, noise, out=y_col))
    for name, start, opt in (("white_adam", noise, "adam"), ("coloured_momentum", y_col, "momentum"),
                             ("coloured_adam", y_col, "adam"), ("white_momentum", noise, "momentum")):
        y = start.clone()
        extra = {}
        if opt == "adam":
            losses, ms = descend_adam(plan, y, phi_target, steps, lr)
        else:
            losses, ms, st = descend_momentum(plan, y, phi_target, steps, mu0, m)
            st = st.cpu().numpy()
            extra = {"final_mu": st[:, 0].tolist(), "accepted_last": st[:, 2].tolist()}
            extra["rejected"] = int((losses > torch.cummin(losses, dim=0).values).sum().item())
        curve = _curve(losses)
        ms0 = init_ms if start is y_col else 0.0
        out["arms"][name] = {"curve": curve, "ms": ms, "init_ms": ms0, "ms_per_step": ms / steps,
                             "initial_loss": float(curve[0]), "final_loss": float(curve[-1]), **extra}
    target = out["arms"]["white_adam"]["final_loss"]
    out["target_loss"] = target
    for arm in out["arms"].values():
        hit = np.nonzero(arm["curve"] <= target)[0]
        arm["steps_to_target"] = int(hit[0]) + 1 if hit.size else None
        arm["ms_to_target"] = (None if not hit.size
                               else arm["init_ms"] + (int(hit[0]) + 1) * arm["ms_per_step"])
        arm["curve"] = arm["curve"].tolist()
    return out
