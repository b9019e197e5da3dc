"""Approximation quality of the sliCQ against the full-length CQ-NSGT
(Sec. 5.3, the experiment behind Fig. 4) with the FP64 oracle -- TEST AND
DOCUMENTATION INFRASTRUCTURE ONLY.

For complex Gaussian signals (the paper's Set 1 kind, shorter: L = 4 x the
slice length) it prints the mean SNR 20 log10(||c|| / ||c - (s^0 + s^1)||)
for Blackman-Harris windows, B = 48, fmin = 50 Hz at 44.1 kHz, slice lengths
4096 and 16384, transitions of 1/4 and 1/128 of the slice, and minimal
filter lengths 4, 8, 16, 32.  The paper prints no values for this figure;
only its trend (SNR rising with the minimal filter length) compares.

    python -m oracle.prop4_experiment [--signals 3]
"""

from __future__ import annotations

import argparse

import numpy as np

from .slicq_oracle import SliCQParams, approximation_snr_db, make_plan


def table(signals: int = 3, seed: int = 1210):
    rng = np.random.default_rng(seed)
    rows = []
    for L2 in (4096, 16384):
        L = 4 * L2
        fs = [rng.standard_normal(L) + 1j * rng.standard_normal(L) for _ in range(signals)]
        for frac in (4, 128):
            M = L2 // frac
            snr = []
            for ml in (4, 8, 16, 32):
                plan = make_plan(SliCQParams(44100.0, 50.0, 22050.0, 48, L2, M, min_filter_len=ml,
                                             window="blackman_harris"))
                snr.append(float(np.mean([approximation_snr_db(f, plan) for f in fs])))
            rows.append((L2, M, snr))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--signals", type=int, default=3)
    a = ap.parse_args()
    print("| slice 2N | transition M | SNR (dB) at min filter length 4 | 8 | 16 | 32 |")
    print("|---|---|---|---|---|---|")
    for L2, M, snr in table(a.signals):
        print(f"| {L2} | {M} | " + " | ".join(f"{v:.1f}" for v in snr) + " |")


if __name__ == "__main__":
    main()
