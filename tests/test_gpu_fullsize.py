"""Parity at the full sizes of the ragged-batch and differentiation
workloads, on sampled outputs the oracle computes (FP64), through the C ABI
in the launch configuration the benchmark times.

* Ragged batch: 256 mono clips, 1-30 s, fs in {16, 22.05, 44.1, 48} kHz,
  B in {12, 24, 48, 96}, fmin 50 Hz, fmax min(22 kHz, fs/2), 2N = 16384,
  M = 4096, one batch forward + inverse: every clip reconstructs to 1e-5;
  the coefficients of three sampled clips (the shortest, a median and the
  longest of one plan) match the oracle's to 1e-5 (relative L2) and 2e-5
  of each slice's largest value per element.
* Differentiation: batch 32 x 6 s at 44.1 kHz, B = 12, 24, 48 (fmin 40 Hz,
  2N = 8192, M = 2048): the forward of two sampled clips and the adjoint of
  random coefficients for them match the oracle at every resolution.
Tolerances as in test_gpu_parity.py (float32 FFT stages, twiddles from FP64).
"""

import numpy as np
import pytest

import oracle as O
from paper_1210_0084_gb300 import signals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL, ELEM = 1e-5, 2e-5


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_0084_gb300 import slicq
    return slicq


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _check(got, ref):
    assert got.shape == ref.shape
    assert _rel(got, ref) <= REL, _rel(got, ref)
    for m in range(ref.shape[0]):
        assert np.abs(got[m] - ref[m]).max() <= ELEM * np.abs(ref[m]).max() + 1e-30, m


def test_ragged_batch_full_size(S):
    clips = signals.ragged_clips(256, seed=signals.seed_for(3, 0))
    keys = sorted({(c.fs, c.bins_per_octave) for c in clips})
    prm = {k: (k[0], 50.0, min(22000.0, k[0] / 2), k[1], 16384, 4096) for k in keys}
    plans = [S.SliCQPlan(S.SliCQParams(*prm[k])) for k in keys]
    clip_plan = [keys.index((c.fs, c.bins_per_octave)) for c in clips]
    lens = [c.signal.shape[0] for c in clips]
    batch = S.SliCQBatch(plans, clip_plan, lens)
    sig = batch.pack([c.signal for c in clips])
    coef = batch.forward(sig)
    rec = batch.inverse(coef)
    torch.cuda.synchronize()
    assert sum(lens) > 10 ** 8
    for c in range(len(clips)):
        y = batch.clip_signal(rec, c).cpu().numpy()
        assert _rel(y, clips[c].signal) <= REL, c
    # three sampled clips of the most used plan
    p = max(set(clip_plan), key=clip_plan.count)
    mine = sorted((lens[c], c) for c in range(len(clips)) if clip_plan[c] == p)
    op = O.make_plan(O.SliCQParams(*prm[keys[p]]))
    for _, c in (mine[0], mine[len(mine) // 2], mine[-1]):
        got = batch.clip_coefs(coef, c).cpu().numpy().astype(np.complex128)
        _check(got, O.slicq_forward(clips[c].signal.astype(np.float64), op))


def test_differentiation_batch_full_size(S):
    fs, n, nb = 44100.0, 6 * 44100, 32
    noisy, _ = signals.noisy_clean_tone_mixtures(nb, n, fs, seed=signals.seed_for(4))
    xd = torch.from_numpy(noisy).cuda()
    rng = np.random.default_rng(12)
    for B in (12, 24, 48):
        prm = (fs, 40.0, fs / 2, B, 8192, 2048)
        plan = S.SliCQPlan(S.SliCQParams(*prm))
        op = O.make_plan(O.SliCQParams(*prm))
        c = plan.forward(xd).cpu().numpy().astype(np.complex128)
        cr = (rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).astype(np.complex64)
        g = plan.adjoint(torch.from_numpy(cr).cuda(), n).cpu().numpy()
        for b in (0, nb - 1):
            _check(c[b], O.slicq_forward(noisy[b].astype(np.float64), op))
            assert _rel(g[b], O.slicq_adjoint(cr[b].astype(np.complex128), op, n)) <= REL
