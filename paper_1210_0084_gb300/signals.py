"""Seeded synthetic audio shaped like the paper's workloads (NumPy, float32).

The paper times its transforms on random signals at 44.1 kHz (Sec. 5.2) and
measures approximation quality on random complex signals and on music
(Sec. 5.3); the music set is not available, so these generators stand in for
it.  This module holds no arithmetic of the transform itself: it only draws
inputs, and both the CUDA path and the FP64 oracle consume its arrays.

Every generator takes an explicit integer seed (NumPy PCG64 via
``default_rng``) and returns C-contiguous float32 arrays.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

__all__ = [
    "noise_plus_sines", "pink_noise_harmonic_tones", "noise_plus_chirps",
    "RaggedClip", "ragged_clips", "noisy_clean_tone_mixtures", "seed_for",
]


def seed_for(config_index: int, clip_index: int = 0) -> int:
    """seed = config index * 1000 + clip index."""
    return int(config_index) * 1000 + int(clip_index)


def noise_plus_sines(n: int, fs: float, seed: int, sigma: float = 0.1,
                     n_sines: int = 3, fband=(100.0, 8000.0),
                     amp=(0.1, 0.5)) -> np.ndarray:
    """White Gaussian noise N(0, sigma^2) plus sinusoids with uniform random
    frequency, amplitude and phase."""
    rng = np.random.default_rng(seed)
    t = np.arange(n) / fs
    x = sigma * rng.standard_normal(n)
    for _ in range(n_sines):
        f = rng.uniform(*fband)
        a = rng.uniform(*amp)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        x += a * np.sin(2.0 * np.pi * f * t + ph)
    return x.astype(np.float32)


def _pink(n: int, rng: np.random.Generator, rms: float) -> np.ndarray:
    """1/f power spectrum by shaping white Gaussian noise in frequency."""
    w = rng.standard_normal(n)
    W = np.fft.rfft(w)
    k = np.arange(W.shape[0], dtype=np.float64)
    k[0] = 1.0
    W /= np.sqrt(k)
    W[0] = 0.0
    x = np.fft.irfft(W, n)
    return x * (rms / max(np.sqrt(np.mean(x * x)), 1e-30))


def pink_noise_harmonic_tones(n: int, fs: float, channels: int, seed: int,
                              rms: float = 0.1, n_tones: int = 20,
                              f0_range=(55.0, 880.0), partials: int = 8,
                              tau_range=(0.2, 2.0)) -> np.ndarray:
    """Pink noise (RMS ``rms``) plus decaying harmonic tones per channel:
    f0 log-uniform, partials k f0 with 1/k amplitude, exponential decay with
    time constant tau, random onset.  Returns [channels, n] float32."""
    rng = np.random.default_rng(seed)
    out = np.empty((channels, n), dtype=np.float32)
    t = np.arange(n) / fs
    for c in range(channels):
        x = _pink(n, rng, rms)
        for _ in range(n_tones):
            f0 = float(np.exp(rng.uniform(np.log(f0_range[0]), np.log(f0_range[1]))))
            tau = rng.uniform(*tau_range)
            onset = rng.uniform(0.0, n / fs)
            amp = rng.uniform(0.05, 0.2)
            ph = rng.uniform(0.0, 2.0 * np.pi, partials)
            # the envelope is below 1e-7 after 16 tau: evaluate the active span only
            i0 = int(np.ceil(onset * fs))
            i1 = min(n, i0 + int(16.0 * tau * fs) + 1)
            if i0 >= n:
                continue
            ts = t[i0:i1]
            env = np.exp(-(ts - onset) / tau)
            for kk in range(1, partials + 1):
                if kk * f0 >= fs / 2:
                    break
                x[i0:i1] += amp / kk * env * np.sin(2.0 * np.pi * kk * f0 * ts + ph[kk - 1])
        out[c] = x
    return out


def noise_plus_chirps(n: int, fs: float, seed: int, sigma: float = 0.05,
                      n_chirps: int = 4, f_lo: float = 40.0,
                      f_hi: float = 20000.0) -> np.ndarray:
    """Gaussian noise plus exponential (log-frequency) chirps sweeping f_lo to
    f_hi over a random duration, each starting at a random time."""
    rng = np.random.default_rng(seed)
    x = sigma * rng.standard_normal(n)
    for _ in range(n_chirps):
        dur = int(rng.uniform(0.2, 0.6) * n)
        start = int(rng.uniform(0, n - dur))
        tt = np.arange(dur) / fs
        T = dur / fs
        r = np.log(f_hi / f_lo)
        phase = 2.0 * np.pi * f_lo * T / r * (np.exp(r * tt / T) - 1.0)
        x[start:start + dur] += rng.uniform(0.1, 0.3) * np.sin(phase)
    return x.astype(np.float32)


@dataclass
class RaggedClip:
    fs: float
    bins_per_octave: int
    signal: np.ndarray


def ragged_clips(n_clips: int, seed: int, len_s=(1.0, 30.0),
                 rates=(16000, 22050, 44100, 48000),
                 bpos=(12, 24, 48, 96)) -> List[RaggedClip]:
    """Clips of uniform random length, sample rate and bins per octave, each
    noise plus sinusoids (seeded per clip)."""
    rng = np.random.default_rng(seed)
    clips = []
    for i in range(n_clips):
        fs = float(rates[rng.integers(len(rates))])
        B = int(bpos[rng.integers(len(bpos))])
        n = int(rng.uniform(*len_s) * fs)
        clips.append(RaggedClip(fs, B, noise_plus_sines(
            n, fs, seed * 7919 + i, fband=(60.0, min(8000.0, fs / 2 - 100)))))
    return clips


def noisy_clean_tone_mixtures(batch: int, n: int, fs: float, seed: int,
                              sigma: float = 0.05, n_tones: int = 5):
    """(noisy, clean) pairs [batch, n]: clean is a tone mixture, noisy adds
    N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    t = np.arange(n) / fs
    clean = np.zeros((batch, n))
    for b in range(batch):
        for _ in range(n_tones):
            f = float(np.exp(rng.uniform(np.log(80.0), np.log(8000.0))))
            clean[b] += rng.uniform(0.05, 0.3) * np.sin(2 * np.pi * f * t + rng.uniform(0, 2 * np.pi))
    noisy = clean + sigma * rng.standard_normal((batch, n))
    return noisy.astype(np.float32), clean.astype(np.float32)
