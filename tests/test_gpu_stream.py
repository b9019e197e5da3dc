"""Streaming sliCQ (one slice per call) against the batch transform, which is
checked against the FP64 oracle elsewhere.  With the signal followed by at
least N zeros, slice 0 of the batch transform (which wraps circularly to the
end) sees the same zeros as a stream with no history, so every slice must
agree; the stream runs the same kernels, so they agree bit for bit."""

import numpy as np
import pytest

from paper_1210_0084_gb300 import signals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_0084_gb300 import slicq
    return slicq


CASES = [
    (16000.0, 50.0, 8000.0, 24, 4096, 1024, 12),
    (44100.0, 32.7, 22050.0, 48, 65536, 16384, 6),    # the bench plan, cluster of 4
    (48000.0, 50.0, 22000.0, 12, 8192, 1026, 8),      # transition = 2 mod 4
]


def _signal(p, nblocks, seed):
    N = p.slice_len // 2
    x = signals.noise_plus_sines(nblocks * N, p.fs, seed).astype(np.float32)
    x[-N:] = 0.0   # the last block is silence: batch slice 0 wraps onto zeros
    return x


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"L{c[4]}_M{c[5]}")
def test_stream_matches_batch(S, case):
    fs, fmin, fmax, B, L2, Mtr, nblocks = case
    p = S.SliCQParams(fs, fmin, fmax, B, L2, Mtr)
    plan = S.SliCQPlan(p)
    N = L2 // 2
    a0 = (N - Mtr) // 2
    x = _signal(p, nblocks, 21)
    n = x.shape[0]
    xd = torch.from_numpy(x).cuda()
    c = plan.forward(xd)
    y = plan.inverse(c, n)
    st = S.SliCQStream(plan)
    assert st.hop == N
    cs = torch.stack([st.forward(xd[m * N:(m + 1) * N]).clone() for m in range(nblocks)])
    torch.cuda.synchronize()
    assert cs.shape == c.shape
    assert torch.equal(cs, c)                      # forward: slice m = batch slice m
    ys = [st.inverse(c[m]).clone() for m in range(nblocks)]
    torch.cuda.synchronize()
    # call m emits samples (m-1)N + a0 + 1 .. mN + a0
    for m in range(1, nblocks):
        ref = y[(m - 1) * N + a0 + 1: m * N + a0 + 1]
        torch.testing.assert_close(ys[m], ref, rtol=0, atol=1e-6 * float(y.abs().max()))
    torch.testing.assert_close(ys[0][N - a0 - 1:], y[: a0 + 1], rtol=0, atol=1e-6 * float(y.abs().max()))


def test_stream_round_trip_is_a_delay(S):
    """forward then inverse, block by block: the output is the input delayed
    by N - a0 - 1 samples (perfect reconstruction, Prop. 3)."""
    p = S.SliCQParams(16000.0, 50.0, 8000.0, 24, 4096, 1024)
    plan = S.SliCQPlan(p)
    N = p.slice_len // 2
    a0 = (N - p.trans_len) // 2
    x = torch.from_numpy(_signal(p, 10, 5)).cuda()
    fwd, inv = S.SliCQStream(plan), S.SliCQStream(plan)
    out = torch.cat([inv.inverse(fwd.forward(x[m * N:(m + 1) * N])).clone()
                     for m in range(10)])
    d = N - a0 - 1
    got = out[d:]
    ref = x[: got.shape[0]]
    assert float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)) <= 1e-5
    # reset: the same block sequence gives the same output again
    fwd.reset()
    inv.reset()
    again = torch.cat([inv.inverse(fwd.forward(x[m * N:(m + 1) * N])).clone() for m in range(10)])
    assert torch.equal(again, out)
