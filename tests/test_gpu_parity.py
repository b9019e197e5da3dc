"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances follow from float32 arithmetic: each output is a sum over a
radix-2 FFT of length 2N (log2(2N) <= 17 stages) and a band FFT of length
M_k (<= 10 stages) with twiddles rounded once from FP64, so the relative L2
error is a small multiple of u * (log2(2N) + log2(M_k)) with
u = 2^-24 ~ 6e-8, i.e. about 2e-6.  The tests require
   coefficient, reconstruction and adjoint relative L2 error <= 1e-5
   (the reconstruction bound is the target accuracy of the method),
   per-element |error| <= 2e-5 * max|reference| per slice.
"""

import numpy as np
import pytest

import oracle as O
from paper_1210_0084_gb300 import signals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5
ELEM = 2e-5


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_0084_gb300 import slicq
    return slicq


def _oplan(p):
    return O.make_plan(O.SliCQParams(p.fs, p.fmin, p.fmax, p.bins_per_octave, p.slice_len,
                                     p.trans_len, p.min_filter_len, mk_policy=p.mk_policy,
                                     window=p.window))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _check_coefs(got, ref):
    assert got.shape == ref.shape
    assert _rel(got, ref) <= REL, _rel(got, ref)
    for m in range(ref.shape[0]):
        scale = np.abs(ref[m]).max()
        assert np.abs(got[m] - ref[m]).max() <= ELEM * scale + 1e-30, m


SMALL = [
    # (fs, fmin, fmax, B, 2N, M, n, batch)
    (16000.0, 50.0, 8000.0, 24, 2048, 512, 5000, 2),       # smallest slice, ragged
    (44100.0, 50.0, 22050.0, 12, 4096, 1024, 20000, 1),
    (44100.0, 50.0, 22050.0, 12, 8192, 2048, 65536, 1),    # exact multiple: circular wrap
    (16000.0, 50.0, 8000.0, 96, 16384, 4096, 40000, 1),    # many tiny bands
    (48000.0, 50.0, 22000.0, 12, 16384, 4096, 30001, 3),   # big Nyquist plateau, odd n
    (44100.0, 32.7, 22050.0, 48, 65536, 16384, 150000, 1), # bench plan, cluster of 4
    (16000.0, 50.0, 8000.0, 24, 2048, 512, 1500, 1),       # n < 2N: two slices
    (44100.0, 40.0, 22050.0, 48, 8192, 2048, 30000, 2),    # several channels cross DC
    (48000.0, 50.0, 22000.0, 96, 4096, 1024, 20000, 1),    # ~90 widened channels cross DC
    (48000.0, 50.0, 22000.0, 24, 16384, 4096, 60000, 1),   # Nyquist plateau of M = 2048
    (48000.0, 50.0, 20000.0, 24, 16384, 4096, 50000, 2),   # Nyquist plateau of M = 4096
    (44100.0, 50.0, 22050.0, 12, 4096, 1026, 20000, 2),    # transition = 2 mod 4, odd a0
    (16000.0, 50.0, 8000.0, 24, 2048, 512, 7000, 2, "const"),  # rectangular: one M_k
    (44100.0, 50.0, 22050.0, 12, 8192, 2048, 30000, 1, "const"),
    (44100.0, 50.0, 22050.0, 12, 8192, 2048, 30000, 2, "pow2", "blackman_harris"),
    (16000.0, 50.0, 8000.0, 24, 2048, 512, 7000, 1, "const", "blackman_harris"),
]


def _params(S, c):
    fs, fmin, fmax, B, L2, M, n, batch = c[:8]
    return S.SliCQParams(fs, fmin, fmax, B, L2, M, mk_policy=c[8] if len(c) > 8 else "pow2",
                         window=c[9] if len(c) > 9 else "hann"), n, batch


def _signal(n, fs, batch, seed):
    return np.stack([signals.noise_plus_sines(n, fs, seed + i) for i in range(batch)])


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"L{c[4]}_B{c[3]}_n{c[6]}x{c[7]}" + "".join("_" + x for x in c[8:]))
def test_forward_inverse_adjoint_parity(S, case):
    p, n, batch = _params(S, case)
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    x = _signal(n, p.fs, batch, 100)
    xd = torch.from_numpy(x).cuda()
    c = plan.forward(xd)
    y = plan.inverse(c, n)
    torch.cuda.synchronize()
    cg = c.cpu().numpy().astype(np.complex128)
    for b in range(batch):
        ref = O.slicq_forward(x[b].astype(np.float64), op)
        _check_coefs(cg[b], ref)
        # inverse from the GPU's own coefficients: perfect reconstruction
        assert _rel(y[b].cpu().numpy(), x[b]) <= REL
    # inverse and adjoint of coefficients that do not come from a real
    # signal (modified coefficients): compared with the oracle on the same input
    rng = np.random.default_rng(5)
    cr = (rng.standard_normal(cg.shape) + 1j * rng.standard_normal(cg.shape)).astype(np.complex64)
    crd = torch.from_numpy(cr).cuda()
    yi = plan.inverse(crd, n).cpu().numpy()
    ya = plan.adjoint(crd, n).cpu().numpy()
    for b in range(batch):
        ri = O.slicq_inverse(cr[b].astype(np.complex128), op, n)
        ra = O.slicq_adjoint(cr[b].astype(np.complex128), op, n)
        assert _rel(yi[b], ri) <= REL
        assert _rel(ya[b], ra) <= REL
        assert np.abs(yi[b] - ri).max() <= ELEM * np.abs(ri).max()
        assert np.abs(ya[b] - ra).max() <= ELEM * np.abs(ra).max()


@pytest.mark.parametrize("window", ["hann", "blackman_harris"])
def test_plan_tables_match_oracle(S, window):
    p = S.SliCQParams(44100.0, 32.7, 22050.0, 48, 65536, 16384, window=window)
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    K = op.K
    sc = 1.0 / np.sqrt(p.slice_len)
    ga = np.concatenate([ch.g for ch in op.sys.channels[:K + 2]]) * sc
    w = np.array([0.5 if k in (0, K + 1) else 1.0 for k in range(K + 2)])
    gs = np.concatenate([op.dual.channels[k].g * w[k] for k in range(K + 2)]) * sc
    np.testing.assert_allclose(plan.table(0), ga, rtol=2e-7, atol=1e-12)
    np.testing.assert_allclose(plan.table(1), gs, rtol=2e-7, atol=1e-16)
    np.testing.assert_allclose(plan.table(2), 0.5 * ga, rtol=2e-7, atol=1e-12)
    N, M = p.slice_len // 2, p.trans_len
    a0 = (N - M) // 2
    hw = op.h0[N + a0: N + a0 + M]
    np.testing.assert_allclose(plan.table(3)[:M], hw, rtol=2e-7, atol=1e-12)


def test_deterministic(S):
    p = S.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048)
    plan = S.SliCQPlan(p)
    x = torch.from_numpy(_signal(50000, p.fs, 2, 7)).cuda()
    c1 = plan.forward(x).clone()
    y1 = plan.inverse(c1, 50000).clone()
    c2 = plan.forward(x)
    y2 = plan.inverse(c2, 50000)
    assert torch.equal(c1, c2) and torch.equal(y1, y2)


def test_buffer_errors(S):
    p = S.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048)
    plan = S.SliCQPlan(p)
    n = 20000
    x = torch.zeros(n, device="cuda")
    Sn = plan.num_slices(n)
    small = torch.empty((Sn, plan.coefs_per_slice - 1), dtype=torch.complex64, device="cuda")
    w = plan.workspace(n, 1)
    lib = plan.lib
    st = lib.slicq_forward(plan.handle, x.data_ptr(), n, 1, small.data_ptr(), small.numel(),
                           w.data_ptr(), w.numel(), None)
    assert st == 4  # SLICQ_ESIZE
    c = torch.empty((Sn, plan.coefs_per_slice), dtype=torch.complex64, device="cuda")
    st = lib.slicq_forward(plan.handle, x.data_ptr(), n, 1, c.data_ptr(), c.numel(),
                           w.data_ptr(), 16, None)
    assert st == 4
    st = lib.slicq_forward(plan.handle, x.data_ptr(), 0, 1, c.data_ptr(), c.numel(),
                           w.data_ptr(), w.numel(), None)
    assert st == 1


def _sampled_full_size(S, p, x, slices_to_check):
    """Forward + inverse at full size on the GPU; oracle on sampled slices."""
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    batch, n = x.shape
    xd = torch.from_numpy(x).cuda()
    c = plan.forward(xd)
    y = plan.inverse(c, n)
    torch.cuda.synchronize()
    for b in range(batch):
        assert _rel(y[b].cpu().numpy(), x[b]) <= REL
    keep = list(range(op.real_channels))
    for b in range(batch):
        xs = O.slicq_slices(x[b].astype(np.float64), op)
        for m in slices_to_check:
            ref = np.concatenate(O.nsgt_analysis(xs[m], op.sys, keep))
            got = c[b, m].cpu().numpy().astype(np.complex128)
            assert _rel(got, ref) <= REL, (b, m, _rel(got, ref))
            assert np.abs(got - ref).max() <= ELEM * np.abs(ref).max()


def test_full_size_60s_stereo(S):
    """60 s stereo at 44.1 kHz, B = 48, 2N = 65536, M = 16384 (the bench workload)."""
    fs = 44100.0
    x = signals.pink_noise_harmonic_tones(60 * 44100, fs, 2, seed=signals.seed_for(1))
    p = S.SliCQParams(fs, 32.7, 22050.0, 48, 65536, 16384)
    _sampled_full_size(S, p, x, [0, 1, 40, 81])


def test_full_size_10min_48k(S):
    """10 min mono at 48 kHz, B = 96, 2N = 131072, M = 32768 (cluster of 8)."""
    fs = 48000.0
    x = signals.noise_plus_chirps(600 * 48000, fs, seed=signals.seed_for(3))[None]
    p = S.SliCQParams(fs, 27.5, 24000.0, 96, 131072, 32768)
    _sampled_full_size(S, p, x, [0, 217, 439])


def test_autograd_backward_is_adjoint(S):
    """loss = sum |c|^2: torch's gradient must equal 2 Re(A^H A x) from the
    oracle, and match an FP64 finite difference of the oracle's loss."""
    p = S.SliCQParams(44100.0, 50.0, 22050.0, 12, 4096, 1024)
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    n = 9000
    x = _signal(n, p.fs, 1, 3)[0]
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    c = S.slicq_transform(xt, plan)
    loss = (c.abs() ** 2).sum()
    loss.backward()
    g = xt.grad.cpu().numpy()
    x64 = x.astype(np.float64)
    gref = 2.0 * O.slicq_adjoint(O.slicq_forward(x64, op), op, n)
    assert _rel(g, gref) <= REL
    v = np.random.default_rng(1).standard_normal(n)
    h = 1e-4
    fp = np.sum(np.abs(O.slicq_forward(x64 + h * v, op)) ** 2)
    fm = np.sum(np.abs(O.slicq_forward(x64 - h * v, op)) ** 2)
    fd = (fp - fm) / (2 * h)
    assert abs(fd - float(np.dot(g, v))) <= 1e-4 * abs(fd)


@pytest.mark.parametrize("case", [SMALL[0], SMALL[3], SMALL[7], SMALL[-2]],
                         ids=["L2048", "L16384_B96", "L8192_DC", "L2048_const"])
def test_spectrogram_parity(S, case):
    """|s^0 + s^1|^2 (Sec. 4.1) of the GPU's coefficients against the oracle's
    spectrogram of the same coefficients, and the per-channel blocks."""
    p, n, batch = _params(S, case)
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    x = _signal(n, p.fs, batch, 300)
    c = plan.forward(torch.from_numpy(x).cuda())
    spec = plan.spectrogram(c, n)
    torch.cuda.synchronize()
    cg = c.cpu().numpy().astype(np.complex128)
    got = spec.cpu().numpy()
    for b in range(batch):
        ref = O.slicq_spectrogram(cg[b], op)
        assert got[b].shape == ref.shape
        assert _rel(got[b], ref) <= REL
        assert np.abs(got[b] - ref).max() <= ELEM * np.abs(ref).max()
    blocks = plan.spectrogram_blocks(spec, n)
    Sn = plan.num_slices(n)
    assert [int(bl.shape[-1]) for bl in blocks] == [Sn * int(m) // 2 for m in op.M[: op.real_channels]]


@pytest.mark.parametrize("shift,masked,case", [
    (8, False, (16000.0, 50.0, 8000.0, 24, 2048, 512, 7000, 2, "const")),
    (-3, True, (16000.0, 50.0, 8000.0, 24, 2048, 512, 7000, 2, "const")),
    (8, True, (44100.0, 50.0, 22050.0, 48, 8192, 2048, 30000, 1, "const")),
    (0, True, SMALL[1]),
])
def test_inverse_modified_parity(S, shift, masked, case):
    """Transposition and masking (Sec. 6) applied as the synthesis reads the
    coefficients, against the oracle's inverse of the oracle-modified
    coefficients (random gains; a shift only with one band length)."""
    p, n, batch = _params(S, case)
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    x = _signal(n, p.fs, batch, 77)
    c = plan.forward(torch.from_numpy(x).cuda())
    mask = None
    if masked:
        mask = torch.from_numpy(np.random.default_rng(9).uniform(0.0, 2.0, size=c.shape).astype(np.float32)).cuda()
    y = plan.inverse_modified(c, n, shift=shift, mask=mask).cpu().numpy()
    cg = c.cpu().numpy().astype(np.complex128)
    for b in range(batch):
        mb = None if mask is None else mask[b].cpu().numpy().astype(np.float64)
        ref = O.slicq_inverse(O.slicq_modify(cg[b], op, shift=shift, mask=mb), op, n)
        assert _rel(y[b], ref) <= REL, _rel(y[b], ref)
        assert np.abs(y[b] - ref).max() <= ELEM * np.abs(ref).max()


def test_inverse_modified_shift_needs_rectangular(S):
    p = S.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512)
    plan = S.SliCQPlan(p)
    c = plan.forward(torch.zeros(4096, device="cuda"))
    with pytest.raises(S.SliCQError):
        plan.inverse_modified(c, 4096, shift=2)


def test_multires_logmag_loss_backward(S):
    """Differentiation workload in small: L = sum_B mean |log(|c_B(x)| + eps) -
    log(|c_B(t)| + eps)| over B = 12, 24, 48 (fmin 40 Hz, 2N = 8192, M = 2048),
    batch 3 of noisy/clean tone mixtures.  The gradient torch computes through
    slicq_transform must equal, per resolution, the oracle's adjoint (FP64) of
    the same upstream gradient dL/dc, summed over resolutions; the loss must
    match the oracle's coefficients' loss.

    Scale of the bound: the upstream gradient of a log-magnitude loss weights
    each coefficient by 1/|c|.  The slices over the zero padding (n = 20000
    is padded to L = 24576) hold tiny coefficients, so their weights
    dominate, and their share of the adjoint lands in the padding, which the
    output drops: the adjoint over all L samples is 450-1100 times larger
    than the trimmed gradient.  A float32 linear map's error scales with the
    values it adds up, so the error is bounded by REL times the norm of the
    untrimmed adjoint (the oracle's adjoint with output length L).  An
    adjoint mistake is still ~1e-3 of that scale; the random-coefficient
    parity tests check the adjoint against its output's own norm."""
    fs, n, batch, eps = 44100.0, 20000, 3, 1e-6
    noisy, clean = signals.noisy_clean_tone_mixtures(batch, n, fs, seed=signals.seed_for(4, 1))
    plans = [S.SliCQPlan(S.SliCQParams(fs, 40.0, fs / 2, B, 8192, 2048)) for B in (12, 24, 48)]
    xt = torch.from_numpy(noisy).cuda().requires_grad_(True)
    tt = torch.from_numpy(clean).cuda()
    cs, cts, loss = [], [], 0.0
    for plan in plans:
        c = S.slicq_transform(xt, plan)
        c.retain_grad()
        ct = plan.forward(tt)
        loss = loss + (torch.log(c.abs() + eps) - torch.log(ct.abs() + eps)).abs().mean()
        cs.append(c)
        cts.append(ct)
    loss.backward()
    g = xt.grad.cpu().numpy().astype(np.float64)
    gref = np.zeros_like(g)
    lgpu, lref, scale2 = 0.0, 0.0, 0.0
    for plan, c, ct in zip(plans, cs, cts):
        op = _oplan(plan.params)
        up = c.grad.cpu().numpy().astype(np.complex128)
        L = O.padded_length(n, plan.params.slice_len)
        for b in range(batch):
            gref[b] += O.slicq_adjoint(up[b], op, n)
            scale2 += float(np.sum(O.slicq_adjoint(up[b], op, L) ** 2))
        cn = np.stack([O.slicq_forward(noisy[b].astype(np.float64), op) for b in range(batch)])
        cc = np.stack([O.slicq_forward(clean[b].astype(np.float64), op) for b in range(batch)])
        # the loss value over the coefficients float32 resolves: those of the
        # zero padding and far from the clean mixture's tones lie near its
        # rounding floor (~1e-7 max|c|), where log(|c| + eps) moves by O(1)
        keep = (np.abs(cn) > 1e-3 * np.abs(cn).max()) & (np.abs(cc) > 1e-3 * np.abs(cc).max())
        dn = c.detach().cpu().numpy().astype(np.complex128)
        dc = ct.cpu().numpy().astype(np.complex128)
        lgpu += np.mean(np.abs(np.log(np.abs(dn[keep]) + eps) - np.log(np.abs(dc[keep]) + eps)))
        lref += np.mean(np.abs(np.log(np.abs(cn[keep]) + eps) - np.log(np.abs(cc[keep]) + eps)))
    err = float(np.linalg.norm(g - gref))
    assert err <= REL * np.sqrt(scale2), (err, np.sqrt(scale2))
    assert abs(lgpu - lref) <= 1e-4 * lref, (lgpu, lref)


@pytest.mark.parametrize("case", [
    (16000.0, 50.0, 8000.0, 24, 2048, 512, 7000, 2, 1), (16000.0, 50.0, 8000.0, 24, 2048, 512, 7000, 2, 2),
    (16000.0, 50.0, 8000.0, 24, 2048, 512, 7000, 2, 4), (16000.0, 50.0, 8000.0, 24, 2048, 512, 7000, 2, 8),
    (48000.0, 50.0, 22000.0, 12, 16384, 4096, 30001, 2, 1), (48000.0, 50.0, 22000.0, 12, 16384, 4096, 30001, 2, 2),
    (48000.0, 50.0, 22000.0, 12, 16384, 4096, 30001, 2, 4), (48000.0, 50.0, 22000.0, 12, 16384, 4096, 30001, 2, 8),
    (44100.0, 32.7, 22050.0, 48, 65536, 16384, 150000, 1, 4), (44100.0, 32.7, 22050.0, 48, 65536, 16384, 150000, 1, 8),
], ids=lambda c: f"L{c[4]}_C{c[8]}")
def test_slice_cluster_sizes(S, case):
    """Every slice cluster size a plan may run (given, or picked by the
    plan's measurement): forward against the oracle, reconstruction, adjoint
    of random coefficients."""
    fs, fmin, fmax, B, L2, M, n, batch, C = case
    p = S.SliCQParams(fs, fmin, fmax, B, L2, M, slice_cluster=C)
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    x = _signal(n, fs, batch, 700)
    xd = torch.from_numpy(x).cuda()
    c = plan.forward(xd)
    y = plan.inverse(c, n)
    cg = c.cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(3)
    cr = (rng.standard_normal(cg.shape) + 1j * rng.standard_normal(cg.shape)).astype(np.complex64)
    ya = plan.adjoint(torch.from_numpy(cr).cuda(), n).cpu().numpy()
    for b in range(batch):
        _check_coefs(cg[b], O.slicq_forward(x[b].astype(np.float64), op))
        assert _rel(y[b].cpu().numpy(), x[b]) <= REL
        assert _rel(ya[b], O.slicq_adjoint(cr[b].astype(np.complex128), op, n)) <= REL


def test_slice_cluster_tuned_choice_is_valid(S):
    """With slice_cluster = 0 the plan measures the valid cluster sizes and
    keeps one of them; the transform it runs is the same transform."""
    p = S.SliCQParams(48000.0, 50.0, 22000.0, 12, 16384, 4096)
    plan = S.SliCQPlan(p)
    assert plan.slice_cluster in (1, 2, 4, 8)
    op = _oplan(p)
    x = _signal(30001, p.fs, 1, 77)
    c = plan.forward(torch.from_numpy(x).cuda())
    _check_coefs(c[0].cpu().numpy().astype(np.complex128), O.slicq_forward(x[0].astype(np.float64), op))


@pytest.mark.parametrize("L2,M", [(2048, 512), (4096, 1024)])
def test_slicq_spectrogram_approximates_full_length_cq(S, L2, M):
    """Proposition 4 on the library's output: the sliCQ spectrogram
    |s^0 + s^1|^2 of a real signal (GPU coefficients, GPU spectrogram kernel)
    against the full-length CQ-NSGT |c| of the same signal (oracle, FP64, with
    the windows of reading R15): ||s^0 + s^1| - |c|| <= ||f|| (inner + outer)
    at every kept (n, k), plus float32 rounding (2e-5 of the largest value)."""
    fs = 44100.0
    p = S.SliCQParams(fs, 100.0, fs / 2, 12, L2, M)
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    n = 4 * L2
    t = np.arange(n) / fs
    x = (np.sin(2 * np.pi * 440.0 * t) + 0.5 * np.sin(2 * np.pi * 3100.0 * t)
         + 0.05 * np.random.default_rng(8).standard_normal(n)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    spec = plan.spectrogram(plan.forward(xd), n)
    blocks = [np.sqrt(b.cpu().numpy().astype(np.float64)) for b in plan.spectrogram_blocks(spec, n)]
    x64 = x.astype(np.float64)
    c = O.cqnsgt_forward(x64, op)
    bound = O.prop4_bound(op, n)
    nf = float(np.linalg.norm(x64))
    top = max(float(np.abs(ck).max()) for ck in c[: op.real_channels])
    for k in range(op.real_channels):
        reps = c[k].shape[0] // bound[k].shape[0]
        assert blocks[k].shape == c[k].shape
        gap = np.abs(blocks[k] - np.abs(c[k]))
        assert np.all(gap <= nf * np.tile(bound[k], reps) + 2e-5 * top), k
