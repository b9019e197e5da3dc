"""Split-precision tensor-core band DFTs (SLICQ_PREC_SPLIT_FP16 / _BF16)
against the FP64 oracle, through the C ABI.

Each radix-8/16/32 stage of the band transforms (Algorithm 1's IFFT_{M_k},
Algorithm 2's FFT_{M_k}) runs as a tcgen05 product of (hi + lo) operands
with FP32 accumulation; the slice FFTs stay FP32.  Bounds from the split:

* FP16 pairs: |x - hi - lo| <= 2^-23 |x| (11-bit significands, rows scaled
  by powers of two so nothing is subnormal that matters), the dropped
  lo * lo term <= 2^-24: each stage is as accurate as FP32 arithmetic, so
  the FP32 bars hold: relative L2 error <= 1e-5 for coefficients,
  reconstruction and adjoint, and 2e-5 of each slice's largest value per
  element.
* BF16 pairs: 8-bit significands keep 2^-18 relative per operand, about
  1.1e-5 per stage (three partial products); a band transform has two such
  stages and a forward + inverse round trip four, about 5e-5.  Bound:
  relative L2 error <= 1e-4, per element 5e-4 of the slice maximum.
"""

import numpy as np
import pytest

import oracle as O
from paper_1210_0084_gb300 import signals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUNDS = {"split_fp16": (1e-5, 2e-5), "split_bf16": (1e-4, 5e-4)}

CASES = [
    # (fs, fmin, fmax, B, 2N, M, n, batch, mk_policy)
    (44100.0, 50.0, 22050.0, 12, 4096, 1024, 20000, 1, "pow2"),     # M_k 16..512
    (16000.0, 50.0, 8000.0, 96, 16384, 4096, 40000, 1, "pow2"),     # many tiny bands
    (48000.0, 50.0, 22000.0, 12, 16384, 4096, 30001, 3, "pow2"),    # Nyquist plateau, odd n
    (44100.0, 32.7, 22050.0, 48, 65536, 16384, 150000, 1, "pow2"),  # bench plan, M_k up to 1024
    (44100.0, 50.0, 22050.0, 12, 8192, 2048, 30000, 2, "const"),    # rectangular: one M
]


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


def _oplan(p):
    return O.make_plan(O.SliCQParams(p.fs, p.fmin, p.fmax, p.bins_per_octave, p.slice_len,
                                     p.trans_len, p.min_filter_len, mk_policy=p.mk_policy))


@pytest.mark.parametrize("precision", ["split_fp16", "split_bf16"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"L{c[4]}_B{c[3]}_n{c[6]}x{c[7]}_{c[8]}")
def test_split_precision_parity(S, case, precision):
    fs, fmin, fmax, B, L2, M, n, batch, mk = case
    rel, elem = BOUNDS[precision]
    p = S.SliCQParams(fs, fmin, fmax, B, L2, M, mk_policy=mk, precision=precision)
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    x = np.stack([signals.noise_plus_sines(n, fs, 300 + b) for b in range(batch)])
    xd = torch.from_numpy(x).cuda()
    c = plan.forward(xd)
    y = plan.inverse(c, n)
    rng = np.random.default_rng(9)
    shape = tuple(c.shape)
    cr = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    ya = plan.adjoint(torch.from_numpy(cr).cuda(), n)
    plan.check()  # no tensor-core wait gave up
    cg = c.cpu().numpy().astype(np.complex128)
    for b in range(batch):
        ref = O.slicq_forward(x[b].astype(np.float64), op)
        assert _rel(cg[b], ref) <= rel, _rel(cg[b], ref)
        for m in range(ref.shape[0]):
            assert np.abs(cg[b][m] - ref[m]).max() <= elem * np.abs(ref[m]).max() + 1e-30, m
        assert _rel(y[b].cpu().numpy(), x[b]) <= rel
        ra = O.slicq_adjoint(cr[b].astype(np.complex128), op, n)
        assert _rel(ya[b].cpu().numpy(), ra) <= rel


def test_split_precision_matches_fp32_path(S):
    """The split-FP16 and FP32 paths agree to the FP32 bar on the bench plan
    (same slice FFTs, only the band stages differ)."""
    fs, n = 44100.0, 200000
    x = signals.pink_noise_harmonic_tones(n, fs, 2, seed=signals.seed_for(1, 9))
    xd = torch.from_numpy(x).cuda()
    out = {}
    for prec in ("fp32", "split_fp16"):
        plan = S.SliCQPlan(S.SliCQParams(fs, 32.7, 22050.0, 48, 65536, 16384, precision=prec))
        out[prec] = plan.forward(xd).cpu().numpy()
        plan.check()
    assert _rel(out["split_fp16"], out["fp32"]) <= 1e-5


def test_precision_rejects_unknown(S):
    import ctypes
    lib = S.load_library()
    cp = S.SliCQParams(44100.0, 50.0, 22050.0, 12, 4096, 1024).to_c()
    cp.precision = 7
    h = ctypes.c_void_p()
    assert lib.slicq_plan_create(ctypes.byref(cp), 0, ctypes.byref(h)) == 1  # SLICQ_EINVAL


def _sig(n, fs, seed):
    return signals.noise_plus_sines(n, fs, seed)


def test_split_ragged_batch(S):
    """A ragged batch of split-FP16 plans: each clip's coefficients equal the
    single-clip path of its plan bit for bit, and reconstruct to the FP32 bar."""
    rates = [(16000.0, 24), (44100.0, 48), (48000.0, 96)]
    plans = [S.SliCQPlan(S.SliCQParams(fs, 50.0, min(22000.0, fs / 2), B, 4096, 1024,
                                       precision="split_fp16")) for fs, B in rates]
    rng = np.random.default_rng(4)
    clip_plan = [0, 1, 2, 1, 0, 2]
    lens = [int(rng.uniform(0.1, 1.0) * rates[p][0]) for p in clip_plan]
    xs = [_sig(n, rates[p][0], 40 + c) for c, (n, p) in enumerate(zip(lens, clip_plan))]
    batch = S.SliCQBatch(plans, clip_plan, lens)
    coef = batch.forward(batch.pack(xs))
    rec = batch.inverse(coef)
    torch.cuda.synchronize()
    for c, x in enumerate(xs):
        single = plans[clip_plan[c]].forward(torch.from_numpy(x).cuda()).cpu().numpy()
        assert np.array_equal(batch.clip_coefs(coef, c).cpu().numpy(), single), c
        assert _rel(batch.clip_signal(rec, c).cpu().numpy(), x) <= 1e-5, c
    for p in plans:
        p.check()


def test_split_stream_matches_forward(S):
    """Streaming one slice per call with a split-FP16 plan equals the plan's
    forward slice by slice (signal ending in N zeros, as the streaming
    tests require)."""
    fs, L2, M = 16000.0, 4096, 1024
    plan = S.SliCQPlan(S.SliCQParams(fs, 50.0, 8000.0, 24, L2, M, precision="split_fp16"))
    N = L2 // 2
    nblocks = 8
    x = _sig(nblocks * N, fs, 55)
    x[-N:] = 0.0
    xd = torch.from_numpy(x).cuda()
    c = plan.forward(xd)
    st = S.SliCQStream(plan)
    cs = torch.stack([st.forward(xd[m * N:(m + 1) * N]).clone() for m in range(nblocks)])
    torch.cuda.synchronize()
    assert torch.equal(cs, c)
    plan.check()


def test_split_masked_synthesis_and_backward(S):
    """Masked synthesis (Sec. 6) and the autograd backward with split-FP16
    band stages against the oracle, at the FP32 bars."""
    fs, n = 44100.0, 30000
    p = S.SliCQParams(fs, 50.0, 22050.0, 12, 8192, 2048, precision="split_fp16")
    plan = S.SliCQPlan(p)
    op = _oplan(p)
    x = _sig(n, fs, 66)
    xd = torch.from_numpy(x).cuda().requires_grad_(True)
    c = S.slicq_transform(xd, plan)
    mask = torch.from_numpy(np.random.default_rng(2).uniform(0.0, 2.0, size=c.shape).astype(np.float32)).cuda()
    y = plan.inverse_modified(c.detach(), n, mask=mask).cpu().numpy()
    cg = c.detach().cpu().numpy().astype(np.complex128)
    ref = O.slicq_inverse(O.slicq_modify(cg, op, mask=mask.cpu().numpy().astype(np.float64)), op, n)
    assert _rel(y, ref) <= 1e-5
    (c.abs() ** 2).sum().backward()
    g = xd.grad.cpu().numpy()
    gref = 2.0 * O.slicq_adjoint(O.slicq_forward(x.astype(np.float64), op), op, n)
    assert _rel(g, gref) <= 1e-5
    plan.check()


def test_bounded_wait_gives_up_and_context_survives(S):
    """The bounded wait of the tensor-core stages, on an mbarrier nothing
    completes, gives up after its limit (about 0.5 ms here) and reports
    SLICQ_ETIMEOUT; afterwards the device still runs a transform correctly."""
    lib = S.load_library()
    assert lib.slicq_selftest_wait(0, 1_000_000) == 5  # SLICQ_ETIMEOUT
    assert lib.slicq_selftest_wait(0, 0) == 1          # SLICQ_EINVAL
    p = S.SliCQParams(44100.0, 50.0, 22050.0, 12, 4096, 1024, precision="split_fp16")
    plan = S.SliCQPlan(p)
    x = signals.noise_plus_sines(20000, 44100.0, 91)
    c = plan.forward(torch.from_numpy(x).cuda())
    plan.check()
    ref = O.slicq_forward(x.astype(np.float64), _oplan(p))
    assert _rel(c.cpu().numpy().astype(np.complex128), ref) <= 1e-5
