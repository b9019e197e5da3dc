"""Ragged batches through the C ABI: clips of different lengths over several
plans (sample rate, bins per octave) of one slice geometry, in one call;
parity per clip with the single-clip path and with the FP64 oracle, perfect
reconstruction, and a CUDA-graph capture of the whole batch."""

import numpy as np
import pytest

import oracle as O
from paper_1210_0084_gb300 import signals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5


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


RATES_B = [(16000.0, 24), (22050.0, 12), (44100.0, 48), (48000.0, 96)]


def _make(S, L2=4096, M=1024, n_clips=10, seed=3):
    rng = np.random.default_rng(seed)
    plans = [S.SliCQPlan(S.SliCQParams(fs, 50.0, min(22000.0, fs / 2), B, L2, M)) for fs, B in RATES_B]
    clip_plan = rng.integers(0, len(plans), n_clips)
    lens = [int(rng.uniform(0.05, 1.2) * RATES_B[p][0]) for p in clip_plan]
    lens[0] = 1  # a one-sample clip
    xs = [signals.noise_plus_sines(n, RATES_B[p][0], seed * 100 + c) for c, (n, p) in enumerate(zip(lens, clip_plan))]
    return plans, clip_plan, lens, xs


def test_batch_matches_single_clip_path_and_oracle(S):
    plans, clip_plan, lens, xs = _make(S)
    batch = S.SliCQBatch(plans, clip_plan, lens)
    sig = batch.pack(xs)
    coef = batch.forward(sig)
    rec = batch.inverse(coef)
    torch.cuda.synchronize()
    for c in range(len(xs)):
        p = plans[clip_plan[c]]
        single = p.forward(torch.from_numpy(xs[c]).cuda()).cpu().numpy()
        got = batch.clip_coefs(coef, c).cpu().numpy()
        assert got.shape == single.shape
        assert np.array_equal(got, single), c          # same kernels, same arithmetic
        y = batch.clip_signal(rec, c).cpu().numpy()
        assert _rel(y, xs[c]) <= REL, c
    for c in (1, 2):
        fs, B = RATES_B[clip_plan[c]]
        op = O.make_plan(O.SliCQParams(fs, 50.0, min(22000.0, fs / 2), B, 4096, 1024))
        ref = O.slicq_forward(xs[c].astype(np.float64), op)
        assert _rel(batch.clip_coefs(coef, c).cpu().numpy().astype(np.complex128), ref) <= REL


def test_batch_rejects_mixed_slice_geometry(S):
    a = S.SliCQPlan(S.SliCQParams(44100.0, 50.0, 22050.0, 12, 4096, 1024))
    b = S.SliCQPlan(S.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 1024))
    with pytest.raises(S.SliCQError):
        S.SliCQBatch([a, b], [0, 1], [1000, 1000])


def test_batch_graph_replay(S):
    plans, clip_plan, lens, xs = _make(S, seed=5)
    batch = S.SliCQBatch(plans, clip_plan, lens)
    sig = batch.pack(xs)
    coef = torch.empty(batch.coef_total, dtype=torch.complex64, device="cuda")
    rec = torch.zeros(batch.sig_total, dtype=torch.float32, device="cuda")
    # warm up outside the capture (first launches set kernel attributes)
    batch.forward(sig, coef)
    batch.inverse(coef, rec)
    torch.cuda.synchronize()
    ref_coef = coef.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.forward(sig, coef)
            batch.inverse(coef, rec)
    coef.zero_()
    rec.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(coef, ref_coef)
    for c in range(len(xs)):
        assert _rel(batch.clip_signal(rec, c).cpu().numpy(), xs[c]) <= REL
