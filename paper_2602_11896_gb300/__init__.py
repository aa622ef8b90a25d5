"""GB300-native joint time-frequency scattering (JTFS) for metamer synthesis.

Lostanlen & Han, "Musical Metamerism with Time-Frequency Scattering": the
transform Phi(x), its adjoint, the loss ||Phi(y) - Phi(x)||^2 and its
gradient, computed by hand-written sm_103a CUDA kernels behind the C ABI of
include/jtfs.h.  This package is the thin PyTorch-side binding.
"""

from .jtfs import JTFSPlan, JTFSBatch, jtfs, momentum_update, INFO_KEYS  # noqa: F401
from . import _native  # noqa: F401

__all__ = ["JTFSPlan", "JTFSBatch", "jtfs", "momentum_update", "INFO_KEYS"]
