"""Pins of the full-length CQ-NSGT and of the sliCQ approximation
(Proposition 4, Sec. 5.3), CPU only.

* The full-length system on C^L with L = 2N is the slice system itself.
* The full-length system is a painless frame: Algorithm 2 with its canonical
  dual inverts Algorithm 1 (Proposition 1).
* Proposition 4: |s^0 + s^1 - c| <= ||f|| (inner + outer) at every
  time-frequency index, for complex random signals (the paper's Set 1 kind)
  and for real signals; shifting the two-layer sum by one time index breaks
  the bound, so it pins the slice time origin and the layer offsets.
* Sec. 5.3: the approximation SNR grows with the minimal filter length.
"""

import numpy as np
import pytest

import oracle as O

FS = 44100.0


def _plan(L2, M, B=12, fmin=100.0, min_len=16):
    return O.make_plan(O.SliCQParams(FS, fmin, FS / 2, B, L2, M, min_filter_len=min_len))


def _complex_signal(L, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(L) + 1j * rng.standard_normal(L)


def _violations(f, plan, shift=0):
    L = f.shape[0]
    c = O.cqnsgt_forward(f, plan)
    s = O.two_layer_sum(O.slicq_forward_complex(f, plan), plan)
    b = O.prop4_bound(plan, L)
    nf = np.linalg.norm(f)
    worst = 0.0
    for ck, sk, bk in zip(c, s, b):
        reps = ck.shape[0] // bk.shape[0]
        err = np.abs(np.roll(sk, shift) - ck)
        worst = max(worst, float(np.max(err / (nf * np.tile(bk, reps) + 1e-12 * nf))))
    return worst


def test_full_length_system_at_slice_length_is_slice_system():
    plan = _plan(2048, 512)
    sysL = O.full_length_system(plan, 2048)
    for a, b in zip(sysL.channels, plan.sys.channels):
        assert a.j0 == b.j0 and a.M == b.M
        np.testing.assert_array_equal(a.g, b.g)


def test_full_length_system_samples_the_slice_windows():
    """g_k[j] = sqrt(L/2N) g^L_k[j L/2N] on the whole circle (Proposition 4
    with the unitary DFT, reading R15)."""
    plan = _plan(2048, 512)
    L = 8192
    sysL = O.full_length_system(plan, L)
    for a, b in zip(sysL.channels, plan.sys.channels):
        gL = a.full(L)
        g = b.full(2048)
        np.testing.assert_allclose(g, np.sqrt(L / 2048) * gL[:: L // 2048], rtol=0, atol=1e-15)
        assert a.M == (L // 2048) * b.M


def test_full_length_cqnsgt_reconstructs():
    """The full-length CQ-NSGT with its own band lengths (M_k >= |J_k| at
    length L, painless): Algorithm 2 with the canonical dual inverts
    Algorithm 1 on C^L (Proposition 1).  (The system of Proposition 4 keeps
    the slice hops a_k instead; where M_k = |J_k| at 2N its L-length band is
    one sample shorter than the support, which the analysis allows.)"""
    plan = _plan(2048, 512)
    L = 8192
    sysL = O.nsg_system(plan.params, L)
    assert all(ch.M >= ch.length for ch in sysL.channels)  # painless (Prop. 2)
    f = _complex_signal(L, 3)
    c = O.nsgt_analysis(f, sysL)
    fr = O.nsgt_synthesis(c, O.dual_system(sysL))
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) < 1e-12


@pytest.mark.parametrize("L2,M", [(2048, 512), (2048, 16), (4096, 1024)])
def test_prop4_bound_complex(L2, M):
    plan = _plan(L2, M)
    f = _complex_signal(4 * L2, 10 + M)
    assert _violations(f, plan) <= 1.0


def test_prop4_bound_real_signal_and_shift_breaks_it():
    plan = _plan(2048, 512, B=24, fmin=60.0)
    L = 4 * 2048
    t = np.arange(L) / FS
    f = (np.sin(2 * np.pi * 440.0 * t) + 0.5 * np.sin(2 * np.pi * 3100.0 * t)
         + 0.05 * np.random.default_rng(5).standard_normal(L)).astype(np.complex128)
    assert _violations(f, plan) <= 1.0
    assert _violations(f, plan, shift=1) > 1.0


def test_snr_grows_with_min_filter_length():
    """Sec. 5.3: longer minimal filters approximate the full-length
    transform better (complex random signal, 2N = 2048, M = 512)."""
    f = _complex_signal(4 * 2048, 21)
    snr = [O.approximation_snr_db(f, _plan(2048, 512, min_len=ml)) for ml in (4, 8, 16, 32)]
    assert all(b > a for a, b in zip(snr, snr[1:])), snr
    assert snr[2] > 30.0, snr
