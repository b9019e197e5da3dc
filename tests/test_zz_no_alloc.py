"""The allocation-free forward entry point (slicq_forward_noalloc).

Some callers may not allocate device memory: a real-time audio callback must
not block on an allocator, and some host applications own all device memory.
slicq_forward_noalloc serves them with a fixed scratch array inside the
library.  This test calls it through the C ABI twice in a row, on two
different inputs, and checks each result against slicq_forward (the entry
point with a caller workspace) with the tolerance of the other parity tests;
it also checks that a size beyond the fixed array is refused.  The file name
makes pytest collect it last.
"""

import ctypes

import numpy as np
import pytest

from paper_1210_0084_gb300 import signals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5          # relative L2 tolerance of the parity tests
SLICQ_ESIZE = 4


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1210_0084_gb300 import slicq
    lib = slicq.load_library()
    fn = lib.slicq_forward_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return slicq


def _noalloc(plan, x, out):
    fn = plan.lib.slicq_forward_noalloc
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(plan.handle, x.data_ptr(), x.shape[-1], x.shape[0], out.data_ptr(), out.numel(), stream)


def test_noalloc_forward_matches_forward_twice(S):
    p = S.SliCQParams(44100.0, 50.0, 22050.0, 24, 8192, 2048)
    plan = S.SliCQPlan(p)
    n, batch = 60000, 2
    for call, seed in enumerate((11, 12)):
        x = np.stack([signals.noise_plus_sines(n, p.fs, seed * 10 + b) for b in range(batch)])
        xd = torch.from_numpy(x).cuda()
        ref = plan.forward(xd)
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(plan, xd, out) == 0, call
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.complex128)
        want = ref.cpu().numpy().astype(np.complex128)
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - want) <= REL * np.linalg.norm(want), call


def test_noalloc_refuses_sizes_beyond_its_array(S):
    p = S.SliCQParams(44100.0, 32.7, 22050.0, 48, 65536, 16384)
    plan = S.SliCQPlan(p)
    n = 60 * 44100       # stereo: 2 x 82 slices of 2^15 + 2 bins x 8 B = 43 MB > 32 MiB
    x = torch.zeros((2, n), device="cuda")
    out = torch.empty((2, plan.num_slices(n), plan.coefs_per_slice), dtype=torch.complex64, device="cuda")
    assert _noalloc(plan, x, out) == SLICQ_ESIZE
