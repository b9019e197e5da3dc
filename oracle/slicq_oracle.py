"""FP64 CPU oracle of the sliCQ transform — TEST INFRASTRUCTURE ONLY.

Plain NumPy, double precision, no blocking, fusion or reordering beyond what
the paper's definitions and algorithms state.  Citations are to
Holighaus, Doerfler, Velasco, Grill, "A framework for invertible, real-time
constant-Q transforms" (arXiv:1210.0084):

* Sec. 2.1   frames, frame operator (eq. frameop), canonical dual (eq. candual),
             unitary DFT normalisation, translation / modulation operators.
* Sec. 2.2   painless nonstationary Gabor systems, eq. framecond1, eq. CQ_coeff,
             Algorithm 1 (NSG analysis), Algorithm 2 (NSG synthesis),
             Proposition 1 (perfect reconstruction), Proposition 2 (diagonal
             frame operator and canonical dual, eq. painlessframe1/2).
* Sec. 3     Table 1 (centre frequencies and bandwidths), constant Q, window
             sampling g_k[j] = H((j xi_s/L - xi_k)/Omega_k), plateau windows.
* Sec. 4     sliCQ steps, Algorithm 3 (analysis), Algorithm 4 (synthesis),
             Proposition 3, eq. BUPU and the Tukey partition of unity.

Readings taken where the paper is silent, ambiguous or inconsistent (each is
listed with its reason in the design notes of the repository):

R1  Coefficients are the frame coefficients c_{n,k} = <f, phi_{n,k}> with the
    unitary DFT of Sec. 2.1 (eq. CQ_coeff); the band transform of Algorithm 1
    is therefore the *unnormalised* backward DFT of the folded band, and the
    band transform of Algorithm 2 is the unnormalised forward DFT, so that the
    canonical dual of Proposition 2 (weights L/a_k = M_k) inverts exactly.
R2  K is the smallest integer with xi_K >= xi_max, decreased while
    xi_K >= xi_s/2 (Table 1 requires xi_K < xi_s/2).
R3  g_0 and g_{K+1} are flat (value 1) on their open supports of width
    Omega_0 and Omega_{K+1} from Table 1.
R4  H is zero on the closed complement of ]-1/2, 1/2[ (strict support).
R5  The lower bound on the filter length (Sec. 5.2) widens Omega_k to
    min_filter_len * xi_s / L for k = 1..K, keeping the centre.
R6  M_k = L/a_k = max(16, next power of two >= |J_k|) (pow2 policy); the
    const policy (the rectangular representation, Sec. 4.1) gives every
    channel the largest of these.
R7  The configured "slice length" is 2N and the "transition" is M (< N).
R8  Tukey slicing window h_0(d), d = j - N, with u = clip((|d|-(N-M)/2)/M, 0, 1)
    and h_0 = cos^2(pi u / 2) for |d| < (N+M)/2, 0 otherwise.
R9  Dual slicing window: the indicator of the support of h_0.
R10 The signal is zero-padded to L = 2N * ceil(n / 2N); indices are circular.
R11 Windows live on the frequency circle: the sample j (any integer) has
    frequency j xi_s / L, and channel 2K+2-k is the mirror image of
    channel k (g_{2K+2-k}[j] = g_k[-j]), as in the rows K+2..2K+1 of Table 1.
R12 Real signals keep channels 0..K+1; the dropped channels are the complex
    conjugates of the kept ones, and synthesis restores them before
    inverting (real part of the full synthesis).
R13 Typos read as meant: the slicing line of Algorithm 3 is
    f[j + (m-1)N] h_0[j - N], and the CQ-NSGT there acts on f^m.
R14 Transposition (Sec. 6) translates baseband coefficients along the
    channels; ours keep the channel's absolute frequency (R1 folds by the
    absolute bin), so a shift by s channels also modulates by the centre-bin
    difference (slicq_modify).
R15 Proposition 4 relates the slice windows to full-length ones by
    sampling, g_k[j] = g^L_k[j L/2N]; its proof periodises inverse DFTs,
    which holds for the 1/n-normalised inverse DFT.  With the unitary DFT
    (R1) the full-length system the sliCQ approximates has the continuous
    windows times sqrt(2N/L) (full_length_system).

Parity status: every public function is pinned by a test under ``tests/``
(brute-force atoms, explicit frame operator, perfect reconstruction, tight
frame energy, adjoint identity, closed forms of Table 1, partition of unity,
time and frequency localisation of the sliCQ spectrogram, FP64 gradcheck of
the adjoint under a log-magnitude loss, and Proposition 4's bound between the
sliCQ and the full-length CQ-NSGT at every time-frequency index).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "SliCQParams", "Channel", "NSGSystem", "SliCQPlan",
    "constant_q", "cq_table", "nsg_system", "frame_diagonal", "dual_system",
    "tukey_slicing_window", "make_plan", "dft", "unitary_dft", "unitary_idft",
    "nsgt_analysis", "nsgt_synthesis", "slicq_slices", "slicq_forward",
    "slicq_inverse", "slicq_adjoint", "slicq_forward_complex",
    "slicq_inverse_complex", "atoms", "frame_operator_matrix",
    "num_slices", "padded_length", "two_layer_view", "slicq_spectrogram", "slicq_modify",
    "full_length_system", "cqnsgt_forward", "two_layer_sum", "prop4_bound", "approximation_snr_db",
]

# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class SliCQParams:
    """sliCQ problem statement (Sec. 3 parameters and Sec. 4.1 slicing).

    fs              sampling rate xi_s in Hz
    fmin, fmax      xi_min and xi_max in Hz
    bins_per_octave B
    slice_len       2N (FFT length of one slice), even
    trans_len       M, the Tukey transition length (Sec. 4.2), 0 < M < N
    min_filter_len  lower bound on the support length of g_k (Sec. 5.2)
    mk_policy       'pow2' (reading R6), 'mult4' (smallest multiple of 4 that
                    is >= |J_k|) or 'const' (one M for all channels: the
                    rectangular representation of Sec. 6)
    window          'hann' (Sec. 3) or 'blackman_harris' (4-term, Harris 1978;
                    the alternative the paper's experiments mention)
    """

    fs: float
    fmin: float
    fmax: float
    bins_per_octave: int
    slice_len: int
    trans_len: int
    min_filter_len: int = 16
    mk_policy: str = "pow2"
    window: str = "hann"

    @property
    def N(self) -> int:
        return self.slice_len // 2


def constant_q(B: int) -> float:
    """Q = (2^{1/B} - 2^{-1/B})^{-1} (Sec. 3)."""
    return 1.0 / (2.0 ** (1.0 / B) - 2.0 ** (-1.0 / B))


def cq_table(p: SliCQParams):
    """Centre frequencies xi_k and bandwidths Omega_k, k = 0..2K+1 (Table 1).

    Returns (K, xi, Omega) with xi, Omega float64 arrays of length 2K+2.
    Bandwidths of channels 1..K are widened to the minimal filter length
    (reading R5); their mirrors K+2..2K+1 inherit the widened values.
    """
    if not (p.fmin > 0 and p.fmax > p.fmin and p.fs > 0):
        raise ValueError("need 0 < fmin < fmax and fs > 0")
    B = p.bins_per_octave
    Q = constant_q(B)
    # reading R2: smallest K with xi_K >= xi_max, then below Nyquist
    K = int(math.ceil(B * math.log2(p.fmax / p.fmin) - 1e-9)) + 1
    while K >= 1 and p.fmin * 2.0 ** ((K - 1) / B) >= p.fs / 2:
        K -= 1
    if K < 1:
        raise ValueError("fmin at or above Nyquist: no constant-Q channel")
    xi = np.zeros(2 * K + 2)
    Om = np.zeros(2 * K + 2)
    ks = np.arange(1, K + 1)
    xi[1:K + 1] = p.fmin * 2.0 ** ((ks - 1) / B)
    Om[1:K + 1] = xi[1:K + 1] / Q
    floor_bw = p.min_filter_len * p.fs / p.slice_len
    Om[1:K + 1] = np.maximum(Om[1:K + 1], floor_bw)
    xi[0], Om[0] = 0.0, 2.0 * p.fmin
    xi[K + 1], Om[K + 1] = p.fs / 2.0, p.fs - 2.0 * xi[K]
    for k in range(K + 2, 2 * K + 2):
        xi[k] = p.fs - xi[2 * K + 2 - k]
        Om[k] = Om[2 * K + 2 - k]
    return K, xi, Om


# ---------------------------------------------------------------------------
# Painless NSG system on C^L (Sec. 2.2, Sec. 3)
# ---------------------------------------------------------------------------


@dataclass
class Channel:
    """One frequency channel: window g_k on the circle Z_L.

    j0      first support sample (circular index in [0, L))
    g       window values on J_k = {j0, j0+1, ..., j0+len-1} (mod L)
    M       number of coefficients L/a_k (M_k)
    """

    j0: int
    g: np.ndarray
    M: int

    @property
    def length(self) -> int:
        return int(self.g.shape[0])

    def full(self, L: int) -> np.ndarray:
        """The window as a length-L vector."""
        out = np.zeros(L)
        idx = (self.j0 + np.arange(self.length)) % L
        np.add.at(out, idx, self.g)
        return out


@dataclass
class NSGSystem:
    L: int
    K: int
    channels: List[Channel]          # k = 0..2K+1
    xi: np.ndarray
    Omega: np.ndarray

    @property
    def n_channels(self) -> int:
        return len(self.channels)


def _hann(t: np.ndarray) -> np.ndarray:
    """H(t) = cos^2(pi t) on ]-1/2, 1/2[, zero outside (Sec. 3, reading R4)."""
    return np.where(np.abs(t) < 0.5, np.cos(np.pi * t) ** 2, 0.0)


# 4-term Blackman-Harris window (F. J. Harris, "On the use of windows for
# harmonic analysis with the discrete Fourier transform", Proc. IEEE 66(1),
# 1978): a0 - a1 cos(2 pi x) + a2 cos(4 pi x) - a3 cos(6 pi x) on x in [0, 1],
# here centred (x = t + 1/2), which flips the signs of the odd terms.
_BH = (0.35875, 0.48829, 0.14128, 0.01168)


def _blackman_harris(t: np.ndarray) -> np.ndarray:
    """H(t) = sum_i a_i cos(2 pi i t) on ]-1/2, 1/2[, zero outside (the
    alternative window of Sec. 5.3; strict support as reading R4)."""
    w = sum(a * np.cos(2 * np.pi * i * t) for i, a in enumerate(_BH))
    return np.where(np.abs(t) < 0.5, w, 0.0)


def _window(t: np.ndarray, shape: str) -> np.ndarray:
    if shape == "hann":
        return _hann(t)
    if shape == "blackman_harris":
        return _blackman_harris(t)
    raise ValueError(shape)


def _next_pow2(n: int) -> int:
    return 1 << max(0, int(n - 1).bit_length())


def _band_length(support: int, policy: str, L: int, const_M: int) -> int:
    """M_k >= |J_k| (eq. framecond1); policy per reading R6."""
    if policy == "pow2":
        M = max(16, _next_pow2(support))
    elif policy == "mult4":
        M = max(16, 4 * ((support + 3) // 4))
    elif policy == "const":
        M = const_M
    else:
        raise ValueError(policy)
    if M < support or M > L:
        raise ValueError("band length outside [|J_k|, L]")
    return M


def nsg_system(p: SliCQParams, L: Optional[int] = None) -> NSGSystem:
    """Sample the constant-Q windows on C^L (Sec. 3).

    g_k[j] = H((j xi_s / L - xi_k) / Omega_k) for the Hann channels and a flat
    plateau for k = 0, K+1 (reading R3).  j runs over the integers around the
    centre (reading R11) and is stored modulo L.  Mirror channels are the
    reflections of channels 1..K (Table 1, rows K+2..2K+1).
    """
    L = p.slice_len if L is None else L
    K, xi, Om = cq_table(p)
    const_M = 0
    raw = []
    for k in range(0, K + 2):
        centre = xi[k] * L / p.fs
        half = Om[k] * L / (2.0 * p.fs)
        lo = int(math.floor(centre - half)) - 1
        hi = int(math.ceil(centre + half)) + 1
        j = np.arange(lo, hi + 1)
        t = (j * p.fs / L - xi[k]) / Om[k]
        inside = np.abs(t) < 0.5
        j, t = j[inside], t[inside]
        if k in (0, K + 1):
            vals = np.ones(j.shape[0])
        else:
            vals = _window(t, p.window)
        raw.append((int(j[0]) if j.size else int(round(centre)), vals))
        const_M = max(const_M, vals.shape[0])
    if p.mk_policy == "const":
        const_M = max(16, _next_pow2(const_M))
    chans: List[Channel] = []
    for k in range(0, K + 2):
        jlo, vals = raw[k]
        M = _band_length(vals.shape[0], p.mk_policy, L, const_M)
        chans.append(Channel(jlo % L, vals, M))
    for k in range(K + 2, 2 * K + 2):
        src = chans[2 * K + 2 - k]
        # g_{2K+2-k}[j] = g_k[-j]: reversed values on the negated interval
        j_last = src.j0 + src.length - 1
        chans.append(Channel((-j_last) % L, src.g[::-1].copy(), src.M))
    return NSGSystem(L, K, chans, xi, Om)


def frame_diagonal(sys_: NSGSystem) -> np.ndarray:
    """d[j] = sum_k (L/a_k) |g_k[j]|^2 = sum_k M_k g_k[j]^2 (eq. painlessframe1)."""
    d = np.zeros(sys_.L)
    for ch in sys_.channels:
        d += ch.M * ch.full(sys_.L) ** 2
    return d


def dual_system(sys_: NSGSystem) -> NSGSystem:
    """Canonical dual windows g~_k = g_k / d (eq. painlessframe2)."""
    d = frame_diagonal(sys_)
    if not np.all(d > 0):
        raise ValueError("painless condition violated: frame diagonal has zeros")
    chans = []
    for ch in sys_.channels:
        idx = (ch.j0 + np.arange(ch.length)) % sys_.L
        chans.append(Channel(ch.j0, ch.g / d[idx], ch.M))
    return NSGSystem(sys_.L, sys_.K, chans, sys_.xi, sys_.Omega)


# ---------------------------------------------------------------------------
# Slicing windows (Sec. 4.2, eq. BUPU, Proposition 3)
# ---------------------------------------------------------------------------


def tukey_slicing_window(N: int, M: int):
    """h_0 and its dual on [0, 2N), centred at j = N (readings R8, R9)."""
    if N % 2 or M % 2 or not (0 < M < N):
        raise ValueError("need N, M even and 0 < M < N")
    j = np.arange(2 * N)
    d = np.abs(j - N).astype(np.float64)
    u = np.clip((d - (N - M) / 2.0) / M, 0.0, 1.0)
    support = d < (N + M) / 2.0
    h0 = np.where(support, np.cos(np.pi * u / 2.0) ** 2, 0.0)
    h0_dual = support.astype(np.float64)
    return h0, h0_dual


# ---------------------------------------------------------------------------
# DFTs (Sec. 2.1 normalisation)
# ---------------------------------------------------------------------------


def dft(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised DFT sum_l x[l] exp(sign 2 pi i l j / n) along the last axis.

    Explicit DFT matrix for n <= 256, numpy.fft otherwise.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n <= 256:
        return x @ _dft_matrix(n, sign).T
    if sign < 0:
        return np.fft.fft(x, axis=-1)
    return np.fft.ifft(x, axis=-1) * n


@lru_cache(maxsize=64)
def _dft_matrix(n: int, sign: int) -> np.ndarray:
    """W[j, l] = exp(sign 2 pi i j l / n) (cached; read-only)."""
    jl = np.outer(np.arange(n), np.arange(n)) % n
    W = np.exp(sign * 2j * np.pi * jl / n)
    W.setflags(write=False)
    return W


def unitary_dft(x):
    """F f[j] = L^{-1/2} sum_l f[l] e^{-2 pi i l j / L} (Sec. 2.1)."""
    return dft(x, -1) / math.sqrt(np.asarray(x).shape[-1])


def unitary_idft(X):
    """F^{-1} (Sec. 2.1)."""
    return dft(X, +1) / math.sqrt(np.asarray(X).shape[-1])


# ---------------------------------------------------------------------------
# NSG analysis / synthesis on C^L (Algorithms 1 and 2, reading R1)
# ---------------------------------------------------------------------------


def nsgt_analysis(f: np.ndarray, sys_: NSGSystem,
                  channels: Optional[Sequence[int]] = None) -> List[np.ndarray]:
    """c = CQ-NSGT_L(f, g, a) (Algorithm 1).

    f_hat = F f; for each channel the product f_hat * conj(g_k) is periodised
    to length M_k = L/a_k and transformed with the unnormalised backward DFT,
    which gives c_{n,k} = <f_hat, M_{-n a_k} g_k> (eq. CQ_coeff).
    """
    L = sys_.L
    fh = unitary_dft(np.asarray(f, dtype=np.complex128))
    ks = range(sys_.n_channels) if channels is None else channels
    out = []
    for k in ks:
        ch = sys_.channels[k]
        idx = (ch.j0 + np.arange(ch.length)) % L
        y = np.zeros(ch.M, dtype=np.complex128)
        # periodisation: sample j lands at residue j mod M_k
        np.add.at(y, idx % ch.M, fh[idx] * np.conj(ch.g))
        out.append(dft(y, +1))
    return out


def nsgt_synthesis(c: Sequence[np.ndarray], dual: NSGSystem,
                   channels: Optional[Sequence[int]] = None) -> np.ndarray:
    """f~ = iCQ-NSGT_L(c, g~, a) (Algorithm 2).

    Per channel the unnormalised forward DFT of c_k is read back at the
    residues j mod M_k of the support J_k, multiplied by g~_k and summed over
    channels; the result is the Fourier transform of f~ (Sec. 2.1 unitary).
    """
    L = dual.L
    ks = range(dual.n_channels) if channels is None else channels
    acc = np.zeros(L, dtype=np.complex128)
    for ck, k in zip(c, ks):
        ch = dual.channels[k]
        Y = dft(np.asarray(ck, dtype=np.complex128), -1)
        idx = (ch.j0 + np.arange(ch.length)) % L
        np.add.at(acc, idx, Y[idx % ch.M] * ch.g)
    return unitary_idft(acc)


# ---------------------------------------------------------------------------
# Brute-force atoms and frame operator (Sec. 2.1/2.2 definitions)
# ---------------------------------------------------------------------------


def atoms(sys_: NSGSystem, k: int) -> np.ndarray:
    """phi_{n,k} = F^{-1}(M_{-n a_k} g_k), n = 0..M_k-1, as rows (Sec. 2.2).

    Built from the definition with explicit modulation and an explicit
    inverse DFT matrix — independent of the periodisation used in
    :func:`nsgt_analysis`.
    """
    L = sys_.L
    ch = sys_.channels[k]
    g = ch.full(L)
    j = np.arange(L)
    l = np.arange(L)
    Finv = np.exp(2j * np.pi * np.outer(l, j) / L) / math.sqrt(L)   # [l, j]
    a = L / ch.M
    rows = []
    for n in range(ch.M):
        mod = np.exp(-2j * np.pi * j * n * a / L) * g   # (M_{-n a_k} g_k)[j]
        rows.append(Finv @ mod)
    return np.array(rows)


def frame_operator_matrix(sys_: NSGSystem) -> np.ndarray:
    """S = sum_{n,k} phi_{n,k} phi_{n,k}^H as an explicit L x L matrix (eq. frameop)."""
    L = sys_.L
    S = np.zeros((L, L), dtype=np.complex128)
    for k in range(sys_.n_channels):
        A = atoms(sys_, k)
        S += A.T @ A.conj()
    return S


# ---------------------------------------------------------------------------
# sliCQ (Sec. 4, Algorithms 3 and 4)
# ---------------------------------------------------------------------------


@dataclass
class SliCQPlan:
    params: SliCQParams
    sys: NSGSystem          # analysis system on C^{2N}
    dual: NSGSystem         # canonical dual on C^{2N}
    h0: np.ndarray          # slicing window on [0, 2N)
    h0_dual: np.ndarray
    offsets: np.ndarray = field(default=None)  # coefficient offsets of channels 0..K+1

    @property
    def K(self) -> int:
        return self.sys.K

    @property
    def N(self) -> int:
        return self.params.N

    @property
    def real_channels(self) -> int:
        return self.sys.K + 2

    @property
    def M(self) -> np.ndarray:
        return np.array([ch.M for ch in self.sys.channels[: self.real_channels]])

    @property
    def coefs_per_slice(self) -> int:
        return int(self.M.sum())


def make_plan(p: SliCQParams, real_signal: bool = True) -> SliCQPlan:
    """Analysis system, canonical dual and slicing windows for one parameter set.

    With real_signal=False the plan serves the complex-input functions
    (slicq_forward_complex / slicq_inverse_complex, all 2K+2 channels) and
    accepts band lengths that do not divide 2N (the mult4 policy); the
    real-signal functions need every M_k to divide 2N (reading R12)."""
    sys_ = nsg_system(p, p.slice_len)
    if real_signal and any(p.slice_len % ch.M for ch in sys_.channels):
        # channel 2K+2-k equals conj(channel k) only when M_k divides 2N
        raise ValueError("real-signal sliCQ needs every M_k to divide 2N")
    dual = dual_system(sys_)
    h0, h0d = tukey_slicing_window(p.N, p.trans_len)
    plan = SliCQPlan(p, sys_, dual, h0, h0d)
    M = plan.M
    plan.offsets = np.concatenate([[0], np.cumsum(M)[:-1]]).astype(np.int64)
    return plan


def padded_length(n: int, slice_len: int) -> int:
    """L = 2N ceil(n / 2N) (Sec. 4.1: L must be a multiple of 2N)."""
    return slice_len * max(1, -(-n // slice_len))


def num_slices(n: int, slice_len: int) -> int:
    """L / N slices (Algorithm 3, m = 0..L/N-1)."""
    return 2 * padded_length(n, slice_len) // slice_len


def slicq_slices(f: np.ndarray, plan: SliCQPlan) -> np.ndarray:
    """f^m[j] = f[j + (m-1)N] h_0[j - N], j < 2N (Algorithm 3, reading R10)."""
    N = plan.N
    n = f.shape[-1]
    L = padded_length(n, 2 * N)
    fp = np.zeros(L, dtype=np.asarray(f).dtype)
    fp[:n] = f
    S = L // N
    j = np.arange(2 * N)
    out = np.empty((S, 2 * N), dtype=np.result_type(fp, np.float64))
    for m in range(S):
        out[m] = fp[(j + (m - 1) * N) % L] * plan.h0
    return out


def slicq_forward_complex(f: np.ndarray, plan: SliCQPlan) -> List[List[np.ndarray]]:
    """sliCQ_{L,N}(f, h_0, g, a) for complex f: all 2K+2 channels per slice (Algorithm 3)."""
    xs = slicq_slices(np.asarray(f, dtype=np.complex128), plan)
    return [nsgt_analysis(x, plan.sys) for x in xs]


def slicq_forward(f: np.ndarray, plan: SliCQPlan) -> np.ndarray:
    """Real-signal sliCQ coefficients, packed [slice][off_k + n] for k = 0..K+1.

    Algorithm 3 per slice, keeping the channels 0..K+1 (reading R12).
    """
    f = np.asarray(f, dtype=np.float64)
    xs = slicq_slices(f, plan)
    keep = range(plan.real_channels)
    out = np.empty((xs.shape[0], plan.coefs_per_slice), dtype=np.complex128)
    for m, x in enumerate(xs):
        out[m] = np.concatenate(nsgt_analysis(x, plan.sys, keep))
    return out


def _unpack(row: np.ndarray, plan: SliCQPlan) -> List[np.ndarray]:
    return [row[o:o + M] for o, M in zip(plan.offsets, plan.M)]


def _overlap_add(slices: np.ndarray, plan: SliCQPlan, n: int, window: np.ndarray):
    """f~[j + (m-1)N] += f~^m[j] h~_0[j - N] (Algorithm 4), trimmed to n samples."""
    N = plan.N
    S = slices.shape[0]
    L = S * N
    acc = np.zeros(L, dtype=slices.dtype)
    j = np.arange(2 * N)
    for m in range(S):
        np.add.at(acc, (j + (m - 1) * N) % L, slices[m] * window)
    return acc[:n]


def slicq_inverse_complex(coefs: List[List[np.ndarray]], plan: SliCQPlan, n: int):
    """isliCQ_{L,N}(s, h~_0, g~, a) from all 2K+2 channels (Algorithm 4)."""
    xs = np.array([nsgt_synthesis(c, plan.dual) for c in coefs])
    return _overlap_add(xs, plan, n, plan.h0_dual)


def slicq_inverse(coef: np.ndarray, plan: SliCQPlan, n: int) -> np.ndarray:
    """Real-signal inverse: restore channels K+2..2K+1 as conjugates (reading R12),
    run Algorithm 2 per slice with the canonical dual, overlap-add with h~_0
    (Algorithm 4) and keep the real part."""
    K = plan.K
    xs = []
    for row in coef:
        c = _unpack(row, plan)
        full = c + [np.conj(c[2 * K + 2 - k]) for k in range(K + 2, 2 * K + 2)]
        xs.append(nsgt_synthesis(full, plan.dual))
    return np.real(_overlap_add(np.array(xs), plan, n, plan.h0_dual))


def slicq_adjoint(coef: np.ndarray, plan: SliCQPlan, n: int) -> np.ndarray:
    """Adjoint of the real-signal analysis map f -> slicq_forward(f).

    A^H c = sum_{m,n,k} c^m_{n,k} phi_{n,k} (shifted to slice m) times h_0,
    i.e. Algorithm 2 with the analysis windows g_k over the kept channels only,
    overlap-added with h_0; the real part gives the gradient for real input.
    """
    xs = []
    keep = list(range(plan.real_channels))
    for row in coef:
        xs.append(nsgt_synthesis(_unpack(row, plan), plan.sys, keep))
    return np.real(_overlap_add(np.array(xs), plan, n, plan.h0))


def two_layer_view(coef: np.ndarray, plan: SliCQPlan, k: int) -> np.ndarray:
    """The 2-layer array s^l_{n,k} of Sec. 4.1 for one channel (Algorithm 3 scatter).

    Slice m's coefficients c^m_{n^s,k} land in layer l = m mod 2 at
    n = n^s + (m-1) M_k / 2 (circular in L M_k / 2N).
    """
    S = coef.shape[0]
    M = int(plan.M[k])
    o = int(plan.offsets[k])
    total = S * M // 2
    s = np.zeros((2, total), dtype=coef.dtype)
    for m in range(S):
        idx = (np.arange(M) + (m - 1) * M // 2) % total
        s[m % 2, idx] = coef[m, o:o + M]
    return s


def slicq_spectrogram(coef: np.ndarray, plan: SliCQPlan) -> np.ndarray:
    """sliCQ spectrogram |s^0 + s^1|^2 (Sec. 4.1): the two layers of the
    2-layer array summed, squared magnitude, for the kept channels
    k = 0..K+1 concatenated (channel k's S M_k / 2 time indices start at
    S off_k / 2)."""
    return np.concatenate([np.abs(two_layer_view(coef, plan, k).sum(axis=0)) ** 2
                           for k in range(plan.real_channels)])


def slicq_modify(coef: np.ndarray, plan: SliCQPlan, shift: int = 0,
                 mask: Optional[np.ndarray] = None) -> np.ndarray:
    """Coefficients for transposition and masking in the rectangular
    representation (Sec. 6: a translation of the spectrum along the channels,
    8 channels = 2 semitones at B = 48).  The paper's coefficients of a
    channel are at baseband; ours keep the channel's absolute frequency
    (readings R1, R14), so channel k = 1..K takes channel k - shift modulated by
    the centre-bin difference: at global time t = (m-1)N + n a of slice m,
    c'_k = c_{k-shift} exp(2 pi i (jc_k - jc_{k-shift}) t / 2N) with
    jc_k = round(xi_k 2N / xi_s); zero when k - shift is outside 1..K.  The
    plateaus k = 0, K+1 keep their own.  Then every coefficient is
    multiplied by mask (same shape).  A shift needs one band length for all
    channels (one time grid)."""
    c = np.array(coef, dtype=np.complex128, copy=True)
    if shift:
        M = set(int(m) for m in plan.M[: plan.real_channels])
        if len(M) != 1:
            raise ValueError("a channel shift needs the rectangular representation")
        (Mc,) = M
        K, N = plan.K, plan.N
        S = c.shape[0]
        jc = np.rint(plan.sys.xi[: K + 2] * 2 * N / plan.params.fs).astype(np.int64)
        t = (np.arange(S)[:, None] - 1) * N + np.arange(Mc)[None, :] * (2 * N // Mc)
        out = c.copy()
        for k in range(1, K + 1):
            src = k - shift
            if 1 <= src <= K:
                dj = int(jc[k] - jc[src])
                out[:, k * Mc:(k + 1) * Mc] = c[:, src * Mc:(src + 1) * Mc] * np.exp(2j * np.pi * dj * t / (2 * N))
            else:
                out[:, k * Mc:(k + 1) * Mc] = 0.0
        c = out
    if mask is not None:
        c = c * mask
    return c


# ---------------------------------------------------------------------------
# Full-length CQ-NSGT and the sliCQ approximation (Sec. 4.2, Proposition 4)
# ---------------------------------------------------------------------------


def full_length_system(plan: SliCQPlan, L: int) -> NSGSystem:
    """The CQ-NSGT system G(g^L, a) on C^L that the slice windows sample
    (Proposition 4): the same continuous windows as the slice system (Table 1
    centres, bandwidths of cq_table) sampled on L bins, and the same time
    steps a_k = 2N / M_k, i.e. L / a_k = (L / 2N) M_k coefficients per
    channel.  L is a multiple of 2N.

    Reading R15: the proof of Proposition 4 uses that the inverse DFT of the
    sampled window is the periodisation of the inverse DFT of the full one,
    which holds for the 1/n-normalised inverse DFT.  With the unitary DFT of
    Sec. 2.1 (reading R1) it holds when g_k[j] = sqrt(L/2N) g^L_k[j L/2N], so
    the full-length windows here are the continuous windows times
    sqrt(2N/L).  (When M_k = |J_k| the L-length band may be shorter than its
    support; c_{n,k} = <f, T_{n a_k} g^L_k-check> is still what Algorithm 1
    computes, by periodisation.)"""
    L2 = plan.params.slice_len
    if L % L2:
        raise ValueError("L must be a multiple of the slice length 2N")
    r = L // L2
    sysL = nsg_system(plan.params, L)
    scale = 1.0 / math.sqrt(r)
    chans = [Channel(cl.j0, cl.g * scale, r * cs.M) for cl, cs in zip(sysL.channels, plan.sys.channels)]
    return NSGSystem(L, sysL.K, chans, sysL.xi, sysL.Omega)


def cqnsgt_forward(f: np.ndarray, plan: SliCQPlan) -> List[np.ndarray]:
    """Full-length CQ-NSGT coefficients c_{n,k} of f in C^L (Algorithm 1 on
    full_length_system), all 2K+2 channels, L = len(f)."""
    f = np.asarray(f, dtype=np.complex128)
    return nsgt_analysis(f, full_length_system(plan, f.shape[-1]))


def two_layer_sum(coefs: Sequence[Sequence[np.ndarray]], plan: SliCQPlan) -> List[np.ndarray]:
    """s^0 + s^1 for every channel from the slices' coefficients (the lists of
    slicq_forward_complex): slice m's c^m_{n^s,k} is added at
    n = n^s + (m-1) M_k / 2 (mod S M_k / 2), so time index n = m M_k/2 + n^s
    holds c^m_{n^s + M_k/2} + c^{m+1}_{n^s} (proof of Proposition 4)."""
    S = len(coefs)
    out = []
    for k, ch in enumerate(plan.sys.channels):
        M = ch.M
        total = S * M // 2
        acc = np.zeros(total, dtype=np.complex128)
        for m in range(S):
            idx = (np.arange(M) + (m - 1) * M // 2) % total
            np.add.at(acc, idx, coefs[m][k])
        out.append(acc)
    return out


def prop4_bound(plan: SliCQPlan, L: int) -> List[np.ndarray]:
    """Right-hand side of Proposition 4 divided by ||f||_2, per channel k and
    n^s < N/a_k = M_k/2:
        ||(1 - h_0 - h_1) T_{n^s a_k} g^L_k-check||
      + ||(h_0 + h_1) sum_{j=1}^{L/2N-1} T_{n^s a_k + 2jN} g^L_k-check||,
    with g^L_k-check = F^{-1} g^L_k and h_0, h_1 the slicing windows of slices
    0 and 1 on C^L (slice m covers t = (m-1)N + j, j < 2N).  The bound holds
    for every slice m (the proof's translation argument): entry n^s bounds
    |s^0 + s^1 - c| at every n = m M_k/2 + n^s."""
    N = plan.N
    L2 = 2 * N
    r = L // L2
    sysL = full_length_system(plan, L)
    j = np.arange(L2)
    h01 = np.zeros(L)
    np.add.at(h01, (j - N) % L, plan.h0)   # slice 0
    np.add.at(h01, j % L, plan.h0)         # slice 1
    out = []
    l = np.arange(L)
    for k, ch in enumerate(sysL.channels):
        gk = unitary_idft(ch.full(L))
        Mk = plan.sys.channels[k].M
        a = L2 // Mk
        ns = np.arange(Mk // 2)
        A = gk[(l[None, :] - ns[:, None] * a) % L]                    # rows T_{n^s a} g-check
        per = A.reshape(ns.size, r, L2).sum(axis=1)                    # sum over the 2N translates
        over = np.tile(per, (1, r)) - A                                # j = 1 .. L/2N - 1
        inner = np.linalg.norm((1.0 - h01)[None, :] * A, axis=1)
        outer = np.linalg.norm(h01[None, :] * over, axis=1)
        out.append(inner + outer)
    return out


def approximation_snr_db(f: np.ndarray, plan: SliCQPlan) -> float:
    """20 log10(||c|| / ||c - (s^0 + s^1)||) over all channels (Sec. 5.3):
    how closely the sliCQ of f approximates its full-length CQ-NSGT."""
    f = np.asarray(f, dtype=np.complex128)
    c = cqnsgt_forward(f, plan)
    s = two_layer_sum(slicq_forward_complex(f, plan), plan)
    num = math.sqrt(sum(float(np.sum(np.abs(ck) ** 2)) for ck in c))
    den = math.sqrt(sum(float(np.sum(np.abs(ck - sk) ** 2)) for ck, sk in zip(c, s)))
    return 20.0 * math.log10(num / den)
