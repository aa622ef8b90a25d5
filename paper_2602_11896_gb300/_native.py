"""ctypes binding of the C ABI declared in include/jtfs.h (argument marshalling only).

The library is the in-tree ``libjtfs.so`` built by ``paper_2602_11896_gb300.build``.
There is no fallback: if it is missing, importing the compute API raises.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_size_t, c_uint32, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libjtfs.so")

# Every symbol include/jtfs.h declares, with (restype, argtypes).
SIGNATURES = {
    "jtfs_plan": (c_int, [POINTER(c_void_p), c_int64, c_int, c_int, c_int, c_int, c_int,
                          c_int64, c_int, c_int, c_uint32]),
    "jtfs_plan_destroy": (c_int, [c_void_p]),
    "jtfs_phi_size": (c_int64, [c_void_p]),
    "jtfs_workspace_bytes": (c_size_t, [c_void_p]),
    "jtfs_path_meta": (c_int, [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32), POINTER(c_int32),
                               POINTER(c_int64)]),
    "jtfs_plan_ragged": (c_int, [POINTER(c_void_p), POINTER(c_int64), c_int, c_int, c_int, c_int, c_int,
                                 c_int, c_int64, c_int, c_uint32]),
    "jtfs_plan_info": (c_int, [c_void_p, POINTER(c_int64), c_int]),
    "jtfs_plan_filters": (c_int, [c_void_p, c_int, POINTER(c_double), POINTER(c_double),
                                  POINTER(c_int32), c_int]),
    "jtfs_plan_schedule": (c_int64, [c_void_p, c_int, POINTER(c_int64), c_int64]),
    "jtfs_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "jtfs_coloured_init": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "jtfs_init_gains": (c_int64, [c_void_p, POINTER(c_float), c_int64]),
    "metamer_step_momentum": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float,
                                      c_void_p, c_void_p, c_void_p]),
    "jtfs_momentum_update": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int64,
                                     c_float, c_void_p]),
    "jtfs_forward_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "jtfs_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "jtfs_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p]),
    "metamer_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_float,
                             c_void_p, c_void_p, c_void_p]),
    "jtfs_batch_create": (c_int, [POINTER(c_void_p), POINTER(c_int64), c_int, c_int, c_int, c_int, c_int,
                                  c_int, c_int64, c_int, c_uint32]),
    "jtfs_batch_destroy": (c_int, [c_void_p]),
    "jtfs_batch_layout": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64)]),
    "jtfs_batch_workspace_bytes": (c_size_t, [c_void_p]),
    "jtfs_batch_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "jtfs_batch_metamer_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float,
                                        c_void_p, c_void_p, c_void_p]),
    "jtfs_autotune": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              POINTER(c_int64), c_int]),
    "jtfs_set_tuning": (c_int, [c_void_p, POINTER(c_int64), c_int]),
    "jtfs_get_tuning": (c_int, [c_void_p, POINTER(c_int64), c_int]),
    "jtfs_convt_padded_channels": (c_int, [c_int]),
    "jtfs_convt_pack_input": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "jtfs_convt_pack_weights": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "jtfs_convt_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int,
                                   c_void_p]),
    "jtfs_convt_backward_data": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int,
                                         c_int, c_void_p]),
    "jtfs_convt_weight_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int]),
    "jtfs_convt_backward_weight": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int,
                                           c_void_p, c_void_p]),
    "jtfs_convt_bias_workspace_bytes": (c_size_t, [c_int64]),
    "jtfs_convt_bias_grad": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_void_p, c_void_p]),
    "jtfs_convt_out_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "jtfs_convt_out_backward_data": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int,
                                             c_void_p]),
    "jtfs_convt_out_workspace_bytes": (c_size_t, [c_int, c_int]),
    "jtfs_convt_out_backward_weight": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int,
                                               c_void_p, c_void_p]),
    "jtfs_decoder_error": (c_int, []),
    "jtfs_cast_bf16": (c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    "jtfs_adam_update": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_float, c_int,
                                 c_void_p]),
    "jtfs_tc_error": (c_int, []),
    "jtfs_tc_error_info": (c_int, [POINTER(c_int64), c_int]),
    "jtfs_tc_table": (c_int64, [c_void_p, c_int, POINTER(c_float), c_int64]),
    "jtfs_profile_stage": (c_int, [c_void_p, c_int, POINTER(c_void_p), c_int]),
    "jtfs_launch_count": (c_int64, [c_void_p, c_int]),
    "jtfs_error_string": (c_char_p, [c_int]),
    "metamer_step_counted": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float,
                                     c_void_p, c_void_p, c_void_p]),
    "jtfs_status": (c_int, [c_void_p]),
    "jtfs_set_wait_limit": (c_int, [c_int64]),
}

ERR_NONFINITE = -8
ERR_TIMEOUT = -9

PLAN_HOST_ONLY = 1
BATCH_REFLECT = 2
PLAN_UNPOOLED_T = 4
PLAN_UNPOOLED_F = 8

_lib = None


def load() -> ctypes.CDLL:
    """Load libjtfs.so once; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing; build it with "
                "`python -m paper_2602_11896_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def error_string(code: int) -> str:
    return load().jtfs_error_string(code).decode()


class DeviceStatusError(RuntimeError):
    """A failure only a running kernel could see (jtfs_status): ``code`` is JTFS_ERR_TIMEOUT or
    JTFS_ERR_NONFINITE."""

    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {error_string(code)} ({code})")
        self.code = code


def check(code: int, what: str) -> None:
    if code != 0:
        raise RuntimeError(f"{what} failed: {error_string(code)} ({code})")


def status(stream: int = 0) -> int:
    """jtfs_status on a raw cudaStream_t handle (synchronises it): 0, ERR_TIMEOUT or ERR_NONFINITE."""
    return int(load().jtfs_status(c_void_p(stream)))


def check_status(what: str, stream: int = 0) -> None:
    """Raise DeviceStatusError if a kernel gave up on a barrier or a loss was non-finite since the
    last check (synchronises the stream)."""
    code = status(stream)
    if code in (ERR_TIMEOUT, ERR_NONFINITE):
        raise DeviceStatusError(code, what)
    check(code, what)
