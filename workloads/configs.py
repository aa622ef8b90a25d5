"""Named JTFS workloads: filterbank parameters, batch shape and input recipe.

Names state what each workload is.  ``params`` are the arguments of a JTFS
plan: N (samples), J, Q (first-order filters per octave), Q2 (second-order
time filters per octave), J_fr, Q_fr (frequential filterbank), T (time
averaging scale, a power of two) and F (frequency averaging scale).
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List

import numpy as np

from . import signals


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    J: int
    Q: int
    Q2: int
    J_fr: int
    Q_fr: int
    T: int
    F: int
    batch: int
    sr: float
    target_seeds: List[int] = field(default_factory=list)
    init_seeds: List[int] = field(default_factory=list)
    target_kind: str = "tones"

    @property
    def params(self) -> Dict[str, int]:
        return dict(N=self.N, J=self.J, Q=self.Q, Q2=self.Q2, J_fr=self.J_fr,
                    Q_fr=self.Q_fr, T=self.T, F=self.F)

    def targets(self) -> np.ndarray:
        """[batch, N] float32 target clips."""
        gen: Callable[[int, float, int], np.ndarray] = {
            "tones": signals.harmonic_tones,
            "chirps": signals.chirp_am_mix,
            "notes": signals.polyphonic_notes,
        }[self.target_kind]
        return np.stack([gen(self.N, self.sr, s) for s in self.target_seeds])

    def inits(self) -> np.ndarray:
        """[batch, N] float32 white-noise initial iterates."""
        return np.stack([signals.white_noise(self.N, s) for s in self.init_seeds])


WORKLOADS: Dict[str, Workload] = {
    # Single clip, 8 kHz: white noise x (seed 0) against harmonic tones y (seed 1).
    "tones8k_n8192": Workload(
        name="tones8k_n8192", N=2 ** 13, J=6, Q=8, Q2=1, J_fr=3, Q_fr=1,
        T=2 ** 6, F=2 ** 2, batch=1, sr=8000.0, target_seeds=[1], init_seeds=[0],
        target_kind="tones"),
    # Batch of 8 clips of 2^16 samples at 22.05 kHz: chirp/AM/pink-noise targets.
    "chirps22k_b8_n65536": Workload(
        name="chirps22k_b8_n65536", N=2 ** 16, J=12, Q=12, Q2=1, J_fr=5, Q_fr=2,
        T=2 ** 11, F=12, batch=8, sr=22050.0,
        target_seeds=list(range(100, 108)), init_seeds=list(range(200, 208)),
        target_kind="chirps"),
    # Long signals: 4 clips of 2^20 samples, polyphonic notes + pink noise.
    "notes22k_b4_n1048576": Workload(
        name="notes22k_b4_n1048576", N=2 ** 20, J=14, Q=16, Q2=2, J_fr=6, Q_fr=2,
        T=2 ** 13, F=16, batch=4, sr=22050.0,
        target_seeds=list(range(400, 404)), init_seeds=list(range(500, 504)),
        target_kind="notes"),
    # Held-out batch for the learned initialiser: 32 clips of 2^16 samples at 8 kHz,
    # the single-clip tone parameters; training clips use seeds TRAIN_SEED0 + i.
    "tones8k_b32_n65536": Workload(
        name="tones8k_b32_n65536", N=2 ** 16, J=6, Q=8, Q2=1, J_fr=3, Q_fr=1,
        T=2 ** 6, F=2 ** 2, batch=32, sr=8000.0,
        target_seeds=[2_000_000 + i for i in range(32)], init_seeds=[3_000_000 + i for i in range(32)],
        target_kind="tones"),
}

# Seeds of the decoder's training clips: TRAIN_SEED0 + i, i < 20000 (disjoint from
# every target and initialisation seed above).
TRAIN_SEED0 = 1_000_000
TRAIN_CLIPS = 20_000


def get_workload(name: str) -> Workload:
    return WORKLOADS[name]
