"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these re-derives a value with the oracle's own formula: each checks a
property that an independent route (brute-force atoms, an explicit frame
operator, a closed-form identity, an invariant) fixes, chosen so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails one
of them.  Citations: arXiv:1210.0084, by section / equation / algorithm.
"""

import math

import numpy as np
import pytest

import oracle as O

# tiny systems for brute force (2N <= 256), and mid-size ones for invariants
TINY = [
    O.SliCQParams(1000.0, 40.0, 500.0, 4, 128, 16, min_filter_len=4),
    O.SliCQParams(8000.0, 150.0, 3000.0, 6, 256, 32, min_filter_len=6),
    O.SliCQParams(2000.0, 35.0, 1000.0, 3, 64, 8, min_filter_len=4),
]
MID = [
    O.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048),          # Hann, B=12
    O.SliCQParams(44100.0, 32.7, 22050.0, 48, 4096, 1024),
    O.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512),
    O.SliCQParams(48000.0, 27.5, 20000.0, 24, 4096, 256),           # fmax < Nyquist
]


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- Table 1 ---

@pytest.mark.parametrize("B", [3, 12, 24, 48, 96])
def test_constant_q_bandwidth_identity(B):
    """Sec. 3: Omega_k = xi_{k+1} - xi_{k-1} for interior k gives the constant Q,
    and xi_{k+B} = 2 xi_k (B bins per octave)."""
    p = O.SliCQParams(44100.0, 30.0, 22050.0, B, 1 << 22, 1 << 16, min_filter_len=1)
    K, xi, Om = O.cq_table(p)
    k = np.arange(2, K)
    np.testing.assert_allclose(Om[k], xi[k + 1] - xi[k - 1], rtol=1e-12)
    kk = np.arange(1, K + 1 - B)
    np.testing.assert_allclose(xi[kk + B], 2.0 * xi[kk], rtol=1e-13)
    # Q = xi_k / Omega_k is the same for every channel 1..K
    q = xi[1:K + 1] / Om[1:K + 1]
    np.testing.assert_allclose(q, q[0], rtol=1e-12)


def test_two_semitones_is_eight_bins_at_48():
    """Sec. 6: a transposition by 2 semitones corresponds to 8 bins at B = 48."""
    p = O.SliCQParams(44100.0, 50.0, 20000.0, 48, 1 << 16, 1 << 14)
    K, xi, _ = O.cq_table(p)
    np.testing.assert_allclose(xi[9:K + 1] / xi[1:K - 7], 2.0 ** (2.0 / 12.0), rtol=1e-13)


@pytest.mark.parametrize("p", MID + TINY)
def test_table1_structure(p):
    """Table 1: xi_max <= xi_K < xi_s/2 (reading R2), plateau widths, mirrors."""
    K, xi, Om = O.cq_table(p)
    assert xi[K] < p.fs / 2
    assert xi[K] >= p.fmax - 1e-9 or xi[K] * 2 ** (1 / p.bins_per_octave) >= p.fs / 2
    assert xi[0] == 0 and Om[0] == 2 * p.fmin
    assert xi[K + 1] == p.fs / 2 and math.isclose(Om[K + 1], p.fs - 2 * xi[K])
    for k in range(1, K + 1):
        assert math.isclose(xi[2 * K + 2 - k], p.fs - xi[k])
        assert Om[2 * K + 2 - k] == Om[k]


# ---------------------------------------------------------------- windows ---

@pytest.mark.parametrize("p", MID)
def test_hann_window_moments(p):
    """Sec. 3 window sampling with a Hann H: the mean of H over its support is
    1/2 and the mean of H^2 is 3/8 (so a cos instead of cos^2, or a wrong
    dilation, fails).  Also |J_k| is L_k = Omega_k L / xi_s up to one sample."""
    sys_ = O.nsg_system(p)
    L = sys_.L
    for k in range(1, sys_.K + 1):
        ch = sys_.channels[k]
        Lk = sys_.Omega[k] * L / p.fs
        assert abs(ch.length - Lk) <= 1.0 + 1e-9
        if Lk >= 200:
            assert abs(ch.g.sum() / Lk - 0.5) < 2.0 / Lk
            assert abs((ch.g ** 2).sum() / Lk - 0.375) < 2.0 / Lk
        # window peaks next to the centre bin omega_k = xi_k L / xi_s
        jpk = ch.j0 + int(np.argmax(ch.g))
        assert abs(((jpk - sys_.xi[k] * L / p.fs + L / 2) % L) - L / 2) <= 1.0


@pytest.mark.parametrize("p", MID + TINY)
def test_mirror_windows(p):
    """Table 1 rows K+2..2K+1: g_{2K+2-k}[j] = g_k[-j] on the circle."""
    sys_ = O.nsg_system(p)
    L, K = sys_.L, sys_.K
    j = np.arange(L)
    for k in range(1, K + 1):
        gk = sys_.channels[k].full(L)
        gm = sys_.channels[2 * K + 2 - k].full(L)
        np.testing.assert_array_equal(gm, gk[(-j) % L])


@pytest.mark.parametrize("p", MID + TINY)
def test_painless_admissibility(p):
    """eq. framecond1: every support fits in M_k = L/a_k samples, and the
    supports cover the whole frequency circle (eq. painlessframe1 > 0)."""
    sys_ = O.nsg_system(p)
    for ch in sys_.channels:
        assert ch.length <= ch.M and p.slice_len % ch.M == 0
    d = O.frame_diagonal(sys_)
    assert d.min() > 0


# -------------------------------------------------------------- DFT paths ---

@pytest.mark.parametrize("n", [7, 64, 256, 300, 512])
def test_dft_against_definition(n):
    """Sec. 2.1: the oracle's DFT equals the defining double sum (both paths)."""
    x = _rng(n).standard_normal(n) + 1j * _rng(n + 1).standard_normal(n)
    l = np.arange(n)
    for sign in (-1, +1):
        ref = np.array([np.sum(x * np.exp(sign * 2j * np.pi * l * jj / n)) for jj in range(n)])
        np.testing.assert_allclose(O.dft(x, sign), ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    np.testing.assert_allclose(O.unitary_idft(O.unitary_dft(x)), x, atol=1e-12)


# ------------------------------------------------ brute force: atoms / S ---

@pytest.mark.parametrize("p", TINY)
def test_coefficients_equal_inner_products_with_atoms(p):
    """eq. CQ_coeff / Algorithm 1: c_{n,k} = <f, phi_{n,k}>, phi_{n,k} = F^{-1}(M_{-n a_k} g_k),
    with the atoms built from the definition (explicit modulation and inverse DFT)."""
    sys_ = O.nsg_system(p)
    L = sys_.L
    rng = _rng(7)
    f = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    c = O.nsgt_analysis(f, sys_)
    for k in range(sys_.n_channels):
        A = O.atoms(sys_, k)                       # rows phi_{n,k}
        ref = A.conj() @ f                         # <f, phi> = sum f conj(phi)
        np.testing.assert_allclose(c[k], ref, atol=1e-12 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("p", TINY)
def test_frame_operator_is_diagonal_in_frequency(p):
    """Prop. 2 / eq. painlessframe1: S = sum phi phi^H equals F^H diag(d) F with
    d = sum_k (L/a_k) |g_k|^2, hence frame bounds A = min d, B = max d."""
    sys_ = O.nsg_system(p)
    L = sys_.L
    S = O.frame_operator_matrix(sys_)
    F = np.exp(-2j * np.pi * np.outer(np.arange(L), np.arange(L)) / L) / math.sqrt(L)
    D = F @ S @ F.conj().T
    d = O.frame_diagonal(sys_)
    np.testing.assert_allclose(np.diag(D).real, d, rtol=1e-11)
    off = D - np.diag(np.diag(D))
    assert np.abs(off).max() < 1e-10 * d.max()
    ev = np.linalg.eigvalsh((S + S.conj().T) / 2)
    assert ev.min() >= d.min() * (1 - 1e-10) and ev.max() <= d.max() * (1 + 1e-10)


@pytest.mark.parametrize("p", TINY)
def test_canonical_dual_is_inverse_frame_operator(p):
    """eq. candual: the dual atoms are S^{-1} phi_{n,k}, checked against the
    explicit matrix inverse of S."""
    sys_ = O.nsg_system(p)
    dual = O.dual_system(sys_)
    S = O.frame_operator_matrix(sys_)
    Sinv = np.linalg.inv(S)
    for k in range(sys_.n_channels):
        A = O.atoms(sys_, k)
        Ad = O.atoms(dual, k)
        np.testing.assert_allclose(Ad, (Sinv @ A.T).T, atol=1e-11 * np.abs(Ad).max())


# ------------------------------------------------- perfect reconstruction ---

@pytest.mark.parametrize("p", TINY + MID)
def test_nsgt_perfect_reconstruction(p):
    """Prop. 1 with the canonical dual: iCQ-NSGT(CQ-NSGT(f)) = f on C^{2N}."""
    sys_ = O.nsg_system(p)
    dual = O.dual_system(sys_)
    rng = _rng(11)
    f = rng.standard_normal(sys_.L) + 1j * rng.standard_normal(sys_.L)
    fr = O.nsgt_synthesis(O.nsgt_analysis(f, sys_), dual)
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) < 1e-13


@pytest.mark.parametrize("p", TINY + MID[:3])
def test_tight_frame_energy(p):
    """Windows g_k / sqrt(d) make S the identity (eq. painlessframe1 = 1), so
    ||c||^2 = ||f||^2 (eq. frameop with S = I)."""
    sys_ = O.nsg_system(p)
    d = O.frame_diagonal(sys_)
    for ch in sys_.channels:
        idx = (ch.j0 + np.arange(ch.length)) % sys_.L
        ch.g = ch.g / np.sqrt(d[idx])
    np.testing.assert_allclose(O.frame_diagonal(sys_), 1.0, rtol=1e-13)
    rng = _rng(3)
    f = rng.standard_normal(sys_.L) + 1j * rng.standard_normal(sys_.L)
    c = O.nsgt_analysis(f, sys_)
    e = sum(np.vdot(ck, ck).real for ck in c)
    assert abs(e / np.vdot(f, f).real - 1) < 1e-13


@pytest.mark.parametrize("N,M", [(64, 16), (4096, 1024), (32768, 16384), (100, 2)])
def test_partition_of_unity(N, M):
    """eq. BUPU and eq. dualwincond: sum_m T_{mN} h_0 = 1 and
    sum_m T_{mN}(h_0 conj(h~_0)) = 1 on Z_L."""
    h0, h0d = O.tukey_slicing_window(N, M)
    L = 8 * N
    acc = np.zeros(L)
    acc2 = np.zeros(L)
    j = np.arange(2 * N)
    for m in range(L // N):
        np.add.at(acc, (j + (m - 1) * N) % L, h0)
        np.add.at(acc2, (j + (m - 1) * N) % L, h0 * h0d)
    np.testing.assert_allclose(acc, 1.0, atol=1e-15)
    np.testing.assert_allclose(acc2, 1.0, atol=1e-15)
    # essential length N, transitions M (Sec. 4.2): N - M + 1 ones, N + M - 1 support
    assert int((h0 == 1.0).sum()) == N - M + 1
    assert int((h0 > 0).sum()) == N + M - 1


def _slicq_params_cases():
    return [
        (O.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048), 65536),   # exact multiple
        (O.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048), 30001),   # ragged tail
        (O.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512), 2048),      # S = 2
        (O.SliCQParams(1000.0, 40.0, 500.0, 4, 128, 16, min_filter_len=4), 1000),
        # rectangular representation: one M for every channel (Sec. 4.1)
        (O.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512, mk_policy="const"), 5000),
    ]


@pytest.mark.parametrize("p,n", _slicq_params_cases())
def test_slicq_perfect_reconstruction_real(p, n):
    """Prop. 3: isliCQ(sliCQ(f)) = f for real f (kept channels 0..K+1)."""
    plan = O.make_plan(p)
    f = _rng(n).standard_normal(n)
    c = O.slicq_forward(f, plan)
    assert c.shape == (O.num_slices(n, p.slice_len), plan.coefs_per_slice)
    fr = O.slicq_inverse(c, plan, n)
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) < 1e-12


@pytest.mark.parametrize("p,n", _slicq_params_cases()[1:])
def test_slicq_perfect_reconstruction_complex(p, n):
    """Prop. 3 for complex f with all 2K+2 channels."""
    plan = O.make_plan(p)
    rng = _rng(n + 5)
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    fr = O.slicq_inverse_complex(O.slicq_forward_complex(f, plan), plan, n)
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) < 1e-12


def test_slices_follow_algorithm3_indices():
    """Algorithm 3 lines 3-4: f^m[j] = f[j + (m-1)N] h_0[j - N], circular in L."""
    p = O.SliCQParams(1000.0, 40.0, 500.0, 4, 128, 16, min_filter_len=4)
    plan = O.make_plan(p)
    n = 200
    f = np.arange(1, n + 1, dtype=np.float64)
    xs = O.slicq_slices(f, plan)
    L = 256
    N = 64
    assert xs.shape == (L // N, 2 * N)
    fp = np.concatenate([f, np.zeros(L - n)])
    for m in range(L // N):
        for j in (0, 17, 64, 100, 127):
            assert xs[m, j] == fp[(j + (m - 1) * N) % L] * plan.h0[j]
    # slice 0 wraps to the end of the padded signal; h_0 is centred at j = N
    assert plan.h0[N] == 1.0 and plan.h0[0] == 0.0


# ---------------------------------------------------- real-signal symmetry ---

@pytest.mark.parametrize("p", TINY + MID[:2])
def test_real_signal_conjugate_channels(p):
    """Table 1 / reading R12: for real f, c_{n,2K+2-k} = conj(c_{n,k}) and the
    DC and Nyquist channels are real."""
    sys_ = O.nsg_system(p)
    K = sys_.K
    f = _rng(5).standard_normal(sys_.L)
    c = O.nsgt_analysis(f, sys_)
    scale = max(np.abs(ck).max() for ck in c)
    for k in range(1, K + 1):
        np.testing.assert_allclose(c[2 * K + 2 - k], np.conj(c[k]), atol=1e-13 * scale)
    assert np.abs(c[0].imag).max() < 1e-13 * scale
    assert np.abs(c[K + 1].imag).max() < 1e-13 * scale


def test_real_inverse_is_real_part_of_complex_inverse():
    """The real-signal inverse equals Re of Algorithm 4 run on the full channel
    set with conjugate mirrors, also for coefficients that are not from a real
    signal (modified coefficients, Sec. 6)."""
    p = MID[2]
    plan = O.make_plan(p)
    rng = _rng(9)
    S = 4
    c = rng.standard_normal((S, plan.coefs_per_slice)) + 1j * rng.standard_normal((S, plan.coefs_per_slice))
    n = S * p.N
    K = plan.K
    full = []
    for row in c:
        parts = [row[o:o + M] for o, M in zip(plan.offsets, plan.M)]
        full.append(parts + [np.conj(parts[2 * K + 2 - k]) for k in range(K + 2, 2 * K + 2)])
    ref = np.real(O.slicq_inverse_complex(full, plan, n))
    np.testing.assert_allclose(O.slicq_inverse(c, plan, n), ref, atol=1e-13)


# --------------------------------------------------------------- pure tone ---

@pytest.mark.parametrize("k0", [30, 60, 90])
def test_pure_tone_peaks_in_its_channel(k0):
    """A sinusoid at xi_{k0} has its largest mean coefficient magnitude in
    channel k0 (Sec. 3: g_k is centred at xi_k and decays away from it)."""
    p = O.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048)
    plan = O.make_plan(p)
    n = 32768
    t = np.arange(n) / p.fs
    f = np.sin(2 * np.pi * plan.sys.xi[k0] * t + 0.3)
    c = O.slicq_forward(f, plan)
    mean_mag = [np.abs(c[2:-2, o:o + M]).mean() for o, M in zip(plan.offsets, plan.M)]
    assert int(np.argmax(mean_mag)) == k0


# ----------------------------------------------------------------- adjoint ---

@pytest.mark.parametrize("p,n", [(TINY[0], 300), (MID[2], 5000)])
def test_adjoint_identity(p, n):
    """<A f, c> = <f, A^H c> for the real-input analysis map A (real inner
    product on the real side, Re of the complex one on the coefficient side)."""
    plan = O.make_plan(p)
    rng = _rng(n)
    f = rng.standard_normal(n)
    S = O.num_slices(n, p.slice_len)
    c = rng.standard_normal((S, plan.coefs_per_slice)) + 1j * rng.standard_normal((S, plan.coefs_per_slice))
    lhs = np.real(np.vdot(O.slicq_forward(f, plan), c))
    rhs = float(np.dot(f, O.slicq_adjoint(c, plan, n)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(f) * np.linalg.norm(c))


def test_adjoint_equals_explicit_matrix_transpose():
    """A^H c from the explicit Jacobian of the forward map (built column by
    column from unit impulses), on a tiny case."""
    p = TINY[2]
    plan = O.make_plan(p)
    n = 96
    cols = [O.slicq_forward(np.eye(n)[i], plan).ravel() for i in range(n)]
    A = np.array(cols).T                      # complex [P, n]
    rng = _rng(1)
    c = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    ref = np.real(A.conj().T @ c)
    got = O.slicq_adjoint(c.reshape(-1, plan.coefs_per_slice), plan, n)
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())


# ------------------------------------------------------------ 2-layer view ---

def test_two_layer_view_places_every_coefficient_once():
    """Sec. 4.1 / Algorithm 3 lines 9-11: slice m goes to layer m mod 2 at
    offset (m-1) M_k / 2; each layer position is written by exactly one slice."""
    p = MID[2]
    plan = O.make_plan(p)
    S = 6
    rng = _rng(2)
    c = rng.standard_normal((S, plan.coefs_per_slice)) + 0j
    k = 5
    s = O.two_layer_view(c, plan, k)
    M = int(plan.M[k])
    o = int(plan.offsets[k])
    assert s.shape == (2, S * M // 2)
    assert np.isclose(np.abs(s).sum(), np.abs(c[:, o:o + M]).sum())
    assert s[1, 0] == c[1, o]        # slice 1 starts at n = 0 of layer 1
    assert s[0, 0] == c[0, o + M // 2]   # slice 0 starts at -M/2 (circular)


def test_rectangular_representation_has_one_band_length():
    """Sec. 4.1: with L/a_k constant the coefficients of a slice form a
    (K+2) x M array; M is a power of two >= every |J_k|, so it divides 2N."""
    p = O.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512, mk_policy="const")
    plan = O.make_plan(p)
    M = set(int(m) for m in plan.M)
    assert len(M) == 1
    (m,) = M
    assert m & (m - 1) == 0 and p.slice_len % m == 0
    assert m >= max(len(ch.g) for ch in plan.sys.channels)
    assert plan.coefs_per_slice == m * plan.real_channels


# ------------------------------------------------------- sliCQ spectrogram ---

def _channel_blocks(spec, plan, S):
    blocks, o = [], 0
    for k in range(plan.real_channels):
        n = S * int(plan.M[k]) // 2
        blocks.append(spec[o:o + n])
        o += n
    assert o == spec.shape[0]
    return blocks


def test_spectrogram_localises_an_impulse_in_time():
    """An impulse at sample t0 peaks, in channel k, at time index t0 / a_k
    (a_k = 2N / M_k): slice m's coefficient n sits at time (m-1)N + n a_k
    (Algorithm 3 with the slice's first sample as time origin), which the
    2-layer array places at n + (m-1) M_k / 2 (Sec. 4.1)."""
    p = O.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512)
    plan = O.make_plan(p)
    n = 16384
    S = O.num_slices(n, p.slice_len)
    for t0 in (5000, 9100):
        f = np.zeros(n)
        f[t0] = 1.0
        blocks = _channel_blocks(O.slicq_spectrogram(O.slicq_forward(f, plan), plan), plan, S)
        for k in range(plan.real_channels - 12, plan.real_channels - 1):  # short atoms
            a = p.slice_len // int(plan.M[k])
            peak = int(np.argmax(blocks[k]))
            assert abs(peak * a - t0) <= a, (k, peak, t0)


def test_spectrogram_localises_a_tone_in_frequency():
    """A sinusoid at xi_{k0} has the largest mean spectrogram value in
    channel k0 (Sec. 3: g_k is centred at xi_k)."""
    p = O.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048)
    plan = O.make_plan(p)
    n = 32768
    S = O.num_slices(n, p.slice_len)
    t = np.arange(n) / p.fs
    for k0 in (40, 75):
        f = np.sin(2 * np.pi * plan.sys.xi[k0] * t + 0.7)
        blocks = _channel_blocks(O.slicq_spectrogram(O.slicq_forward(f, plan), plan), plan, S)
        assert int(np.argmax([b.mean() for b in blocks])) == k0


# ---------------------------------------------------- Blackman-Harris window ---

BH = O.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048, window="blackman_harris")


def test_blackman_harris_window_moments():
    """4-term Blackman-Harris (Harris 1978) sampled as H((j xi_s/L - xi_k)/Omega_k):
    mean over the support a0 = 0.35875, mean square a0^2 + (a1^2 + a2^2 + a3^2)/2
    (the cosines integrate to 0 over whole periods), peak 1 at the centre."""
    a = (0.35875, 0.48829, 0.14128, 0.01168)
    sys_ = O.nsg_system(BH)
    L = sys_.L
    checked = 0
    for k in range(1, sys_.K + 1):
        ch = sys_.channels[k]
        Lk = sys_.Omega[k] * L / BH.fs
        if Lk >= 200:
            assert abs(ch.g.sum() / Lk - a[0]) < 2.0 / Lk
            assert abs((ch.g ** 2).sum() / Lk - (a[0] ** 2 + (a[1] ** 2 + a[2] ** 2 + a[3] ** 2) / 2)) < 2.0 / Lk
            assert abs(ch.g.max() - 1.0) < 1e-3
            checked += 1
    assert checked > 5


@pytest.mark.parametrize("n", [30001, 8192])
def test_blackman_harris_perfect_reconstruction(n):
    """Prop. 3 holds for any admissible window: the canonical dual of the
    Blackman-Harris system reconstructs (painless frame, eq. painlessframe1)."""
    plan = O.make_plan(BH)
    assert plan.dual is not None
    f = _rng(n + 11).standard_normal(n)
    fr = O.slicq_inverse(O.slicq_forward(f, plan), plan, n)
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) < 1e-12


def test_blackman_harris_changes_only_the_window_values():
    """Same supports J_k and band lengths as Hann (the support is |t| < 1/2 for
    both), different values."""
    h = O.make_plan(O.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048))
    b = O.make_plan(BH)
    for ch, cb in zip(h.sys.channels, b.sys.channels):
        assert (ch.j0, ch.length, ch.M) == (cb.j0, cb.length, cb.M)
    k = h.K // 2
    assert not np.allclose(h.sys.channels[k].g, b.sys.channels[k].g)


# ------------------------------------------- transposition and masking ---

RECT = O.SliCQParams(44100.0, 50.0, 22050.0, 48, 8192, 2048, mk_policy="const")


def _channel_energy(c, plan):
    M = int(plan.M[0])
    return np.array([np.sum(np.abs(c[2:-2, k * M:(k + 1) * M]) ** 2) for k in range(plan.real_channels)])


@pytest.mark.parametrize("shift", [8, -8, 4])
def test_transposition_moves_a_tone_by_the_shift(shift):
    """Sec. 6: in the rectangular representation a shift by s channels
    transposes by s/B octaves (8 channels = 2 semitones at B = 48): a tone
    at xi_k0, shifted, resynthesised and analysed again, peaks in k0 + s."""
    plan = O.make_plan(RECT)
    n = 65536
    t = np.arange(n) / RECT.fs
    k0 = 200
    f = np.sin(2 * np.pi * plan.sys.xi[k0] * t + 0.4)
    g = O.slicq_inverse(O.slicq_modify(O.slicq_forward(f, plan), plan, shift=shift), plan, n)
    assert int(np.argmax(_channel_energy(O.slicq_forward(g, plan), plan))) == k0 + shift


def test_mask_selects_channels():
    """A 0/1 mask over channels is a band-pass: the resynthesised signal has
    no energy in the masked-out channels beyond the frame's overlap, and a
    mask of ones is the identity (Prop. 3)."""
    plan = O.make_plan(RECT)
    n = 32768
    f = _rng(3).standard_normal(n)
    c = O.slicq_forward(f, plan)
    ones = np.ones(c.shape)
    assert np.linalg.norm(O.slicq_inverse(O.slicq_modify(c, plan, mask=ones), plan, n) - f) <= 1e-12 * np.linalg.norm(f)
    M = int(plan.M[0])
    mask = np.zeros(c.shape)
    mask[:, 150 * M:200 * M] = 1.0
    e = _channel_energy(O.slicq_forward(O.slicq_inverse(O.slicq_modify(c, plan, mask=mask), plan, n), plan), plan)
    assert e[160:190].min() > 1e3 * e[:100].max()
    assert e[160:190].min() > 1e3 * e[260:].max()


# --- mixed-radix band lengths (M_k the smallest multiple of 4 >= |J_k|) ---

MULT4 = O.SliCQParams(44100.0, 50.0, 22050.0, 12, 2048, 512, mk_policy="mult4")


def test_mult4_real_signal_plans_are_refused():
    """A band length that does not divide 2N breaks the conjugate symmetry
    of a real signal's dropped channels (reading R12)."""
    with pytest.raises(ValueError):
        O.make_plan(MULT4)


def test_mult4_complex_perfect_reconstruction_and_redundancy():
    """Algorithm 4 inverts Algorithm 3 with M_k multiples of 4 (Props. 1-3
    need only M_k >= |J_k|), with fewer coefficients than powers of two."""
    plan = O.make_plan(MULT4, real_signal=False)
    Ms = [ch.M for ch in plan.sys.channels]
    assert all(m % 4 == 0 and m >= ch.length for m, ch in zip(Ms, plan.sys.channels))
    assert any(2048 % m for m in Ms)
    pow2 = O.make_plan(O.SliCQParams(44100.0, 50.0, 22050.0, 12, 2048, 512))
    assert sum(Ms) < sum(ch.M for ch in pow2.sys.channels)
    rng = _rng(31)
    f = rng.standard_normal(8192) + 1j * rng.standard_normal(8192)
    fr = O.slicq_inverse_complex(O.slicq_forward_complex(f, plan), plan, f.shape[0])
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) < 1e-12


def test_mult4_coefficients_equal_inner_products_with_atoms():
    """With a_k = 2N / M_k fractional, c_{n,k} is still <f, F^{-1}(M_{-n a_k} g_k)>."""
    p = O.SliCQParams(8000.0, 200.0, 4000.0, 3, 128, 32, min_filter_len=4, mk_policy="mult4")
    sys_ = O.nsg_system(p, 128)
    assert any(128 % ch.M for ch in sys_.channels)
    rng = _rng(32)
    f = rng.standard_normal(128) + 1j * rng.standard_normal(128)
    c = O.nsgt_analysis(f, sys_)
    for k in range(sys_.n_channels):
        A = O.atoms(sys_, k)
        np.testing.assert_allclose(c[k], A.conj() @ f, rtol=0, atol=1e-12 * np.linalg.norm(f) * 16)
