"""The seeded synthetic inputs (no method arithmetic): deterministic per
seed, float32, and shaped as the workloads they stand in for describe."""

import numpy as np

from paper_1210_0084_gb300 import signals


def test_seed_scheme():
    assert signals.seed_for(2, 5) == 2005
    assert signals.seed_for(0) == 0


def test_deterministic_and_float32():
    a = signals.noise_plus_sines(5000, 44100.0, seed=7)
    b = signals.noise_plus_sines(5000, 44100.0, seed=7)
    c = signals.noise_plus_sines(5000, 44100.0, seed=8)
    assert a.dtype == np.float32 and a.shape == (5000,)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_pink_noise_tones_stereo_shape_and_level():
    fs, n = 44100.0, 2 * 44100
    x = signals.pink_noise_harmonic_tones(n, fs, 2, seed=signals.seed_for(1))
    assert x.shape == (2, n) and x.dtype == np.float32
    rms = np.sqrt(np.mean(x.astype(np.float64) ** 2, axis=1))
    assert np.all(rms > 0.1) and np.all(rms < 1.0)  # pink floor of RMS 0.1 plus tones


def test_pink_noise_spectrum_falls_as_one_over_f():
    """The noise floor alone (no tones) has power density ~ 1/f: the power
    per octave band is about constant."""
    rng = np.random.default_rng(0)
    x = signals._pink(1 << 18, rng, 0.1)
    p = np.abs(np.fft.rfft(x)) ** 2
    f = np.arange(p.shape[0])
    bands = [np.sum(p[(f >= lo) & (f < 2 * lo)]) for lo in (64, 256, 1024, 4096, 16384)]
    bands = np.array(bands) / np.mean(bands)
    assert np.all(bands > 0.7) and np.all(bands < 1.3), bands
    assert abs(np.sqrt(np.mean(x.astype(np.float64) ** 2)) - 0.1) < 1e-6


def test_ragged_clips_recipe():
    clips = signals.ragged_clips(256, seed=signals.seed_for(3))
    assert len(clips) == 256
    assert {c.fs for c in clips} <= {16000.0, 22050.0, 44100.0, 48000.0}
    assert {c.bins_per_octave for c in clips} <= {12, 24, 48, 96}
    secs = np.array([c.signal.shape[0] / c.fs for c in clips])
    assert secs.min() >= 1.0 - 1e-9 and secs.max() <= 30.0 + 1e-9
    assert 10.0 < secs.mean() < 20.0  # uniform on [1, 30] s


def test_noisy_clean_pairs():
    noisy, clean = signals.noisy_clean_tone_mixtures(4, 8000, 44100.0, seed=9)
    assert noisy.shape == clean.shape == (4, 8000)
    d = (noisy - clean).astype(np.float64)
    assert abs(np.std(d) - 0.05) < 0.005  # N(0, 0.05^2) noise on top of the tones
