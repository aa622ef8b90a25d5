"""Seeded synthetic workloads for the JTFS hot path.

This package holds the *inputs* only: signal generators and the named
parameter sets of the benchmark workloads.  It contains none of the
scattering arithmetic, so both the FP64 oracle (``oracle/``) and the CUDA
path (``paper_2602_11896_gb300``) can draw identical bytes from it without
sharing any method code.
"""

from .signals import (  # noqa: F401
    white_noise,
    harmonic_tones,
    chirp_am_mix,
    polyphonic_notes,
    pink_noise,
    uneven_lengths,
)
from .configs import WORKLOADS, Workload, get_workload  # noqa: F401
