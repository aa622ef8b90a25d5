"""Seeded synthetic audio generators.

Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64),
computes in float64, RMS-normalises targets to 1 (so they sit at the same
level as N(0,1) white-noise initialisations) and returns float32.  The paper
evaluates on "any audio recording" (Abstract, Conclusion); these signals stand
in for recordings with the structures its workloads name: harmonic tones with
decaying envelopes, chirps, amplitude-modulated tones, pink noise and
polyphonic note sequences.
"""

from __future__ import annotations

import math

import numpy as np


def _rms_normalise(y: np.ndarray) -> np.ndarray:
    r = math.sqrt(float(np.mean(y * y)))
    return y / r if r > 0 else y


def white_noise(n: int, seed: int) -> np.ndarray:
    """N(0,1) white noise of length ``n``."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n).astype(np.float32)


def pink_noise(n: int, rng: np.random.Generator) -> np.ndarray:
    """1/f-power noise, shaped in the Fourier domain, unit RMS (float64)."""
    w = rng.standard_normal(n)
    W = np.fft.rfft(w)
    f = np.arange(W.shape[0], dtype=np.float64)
    f[0] = 1.0
    W = W / np.sqrt(f)
    W[0] = 0.0
    p = np.fft.irfft(W, n)
    return _rms_normalise(p)


def harmonic_tones(n: int, sr: float, seed: int, n_tones: int = 3,
                   n_partials: int = 5, noise: float = 0.05) -> np.ndarray:
    """Sum of ``n_tones`` harmonic tones plus a little white noise.

    Each tone: f0 ~ U(100, 800) Hz, ``n_partials`` partials with amplitude
    1/k and uniform random phase (partials at or above Nyquist dropped),
    exponential decay envelope exp(-t/tau), tau ~ U(0.1, 0.5) s.
    """
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=np.float64) / sr
    y = np.zeros(n, dtype=np.float64)
    for _ in range(n_tones):
        f0 = rng.uniform(100.0, 800.0)
        tau = rng.uniform(0.1, 0.5)
        env = np.exp(-t / tau)
        for k in range(1, n_partials + 1):
            phase = rng.uniform(0.0, 2.0 * math.pi)
            if k * f0 >= sr / 2:
                continue
            y += (1.0 / k) * np.sin(2.0 * math.pi * k * f0 * t + phase) * env
    y += noise * rng.standard_normal(n)
    return _rms_normalise(y).astype(np.float32)


def chirp_am_mix(n: int, sr: float, seed: int, pink_db: float = -20.0) -> np.ndarray:
    """Mix of 1-3 components (linear chirp, exponential chirp, AM tone) + pink noise.

    Linear/exponential chirps sweep f_start ~ U(50, 500) Hz to
    f_end ~ U(1000, 8000) Hz over the clip.  AM tones have carrier
    ~ U(200, 4000) Hz, modulation rate ~ U(2, 16) Hz and depth ~ U(0.5, 1).
    Pink noise is added at ``pink_db`` dB relative to the mix RMS.
    """
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=np.float64) / sr
    dur = n / sr
    y = np.zeros(n, dtype=np.float64)
    n_comp = int(rng.integers(1, 4))
    for _ in range(n_comp):
        kind = int(rng.integers(0, 3))
        amp = rng.uniform(0.5, 1.0)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        if kind == 0:
            f0 = rng.uniform(50.0, 500.0)
            f1 = rng.uniform(1000.0, 8000.0)
            inst_phase = 2 * math.pi * (f0 * t + 0.5 * (f1 - f0) / dur * t * t)
            y += amp * np.sin(inst_phase + phase)
        elif kind == 1:
            f0 = rng.uniform(50.0, 500.0)
            f1 = rng.uniform(1000.0, 8000.0)
            k = math.log(f1 / f0) / dur
            inst_phase = 2 * math.pi * f0 * (np.exp(k * t) - 1.0) / k
            y += amp * np.sin(inst_phase + phase)
        else:
            fc = rng.uniform(200.0, 4000.0)
            fm = rng.uniform(2.0, 16.0)
            depth = rng.uniform(0.5, 1.0)
            mod = 1.0 + depth * np.sin(2 * math.pi * fm * t + rng.uniform(0, 2 * math.pi))
            y += amp * mod * np.sin(2 * math.pi * fc * t + phase)
    y = _rms_normalise(y)
    y += 10.0 ** (pink_db / 20.0) * pink_noise(n, rng)
    return _rms_normalise(y).astype(np.float32)


def polyphonic_notes(n: int, sr: float, seed: int, rate_hz: float = 4.0,
                     pink_db: float = -20.0) -> np.ndarray:
    """Poisson-onset harmonic notes (rate ``rate_hz``), durations U(1,3) s.

    f0 = MIDI pitch ~ U{36..96}; 10 partials with amplitude 1/k (below
    Nyquist); exponential decay over the note.  With mean duration 2 s and
    4 onsets per second, about 8 notes overlap at any time.
    """
    rng = np.random.default_rng(seed)
    dur = n / sr
    y = np.zeros(n, dtype=np.float64)
    onset = rng.exponential(1.0 / rate_hz)
    while onset < dur:
        length = rng.uniform(1.0, 3.0)
        midi = int(rng.integers(36, 97))
        f0 = 440.0 * 2.0 ** ((midi - 69) / 12.0)
        i0 = int(onset * sr)
        i1 = min(n, i0 + int(length * sr))
        tt = np.arange(i1 - i0, dtype=np.float64) / sr
        env = np.exp(-3.0 * tt / length)
        note = np.zeros(i1 - i0)
        for k in range(1, 11):
            if k * f0 >= sr / 2:
                break
            note += (1.0 / k) * np.sin(2 * math.pi * k * f0 * tt + rng.uniform(0, 2 * math.pi))
        y[i0:i1] += note * env
        onset += rng.exponential(1.0 / rate_hz)
    y = _rms_normalise(y)
    y += 10.0 ** (pink_db / 20.0) * pink_noise(n, rng)
    return _rms_normalise(y).astype(np.float32)


def uneven_lengths(count: int, seed: int, lo_log2: float = 14.0,
                   hi_log2: float = 18.0) -> np.ndarray:
    """Clip lengths drawn log-uniformly from 2^lo_log2 .. 2^hi_log2 samples."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(lo_log2, hi_log2, size=count)
    return np.round(2.0 ** e).astype(np.int64)
