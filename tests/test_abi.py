"""CPU tests of the C ABI: the library loads, exports every declared symbol,
and its host-only layout (Table 1 supports, M_k, offsets) equals the
oracle's, bit for bit.  No compute call touches a device here."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1210_0084_gb300 import build as B
from paper_1210_0084_gb300 import slicq as S


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load_library()


def _declared_symbols(repo_root):
    txt = open(os.path.join(repo_root, "include", "slicq.h")).read()
    return sorted(set(re.findall(r"SLICQ_API[^;(]*?\b(slicq_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib, repo_root):
    names = _declared_symbols(repo_root)
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert lib.slicq_abi_version() == 2


def test_status_strings(lib):
    for code, name in S.STATUS.items():
        assert lib.slicq_status_string(code).decode().startswith(name)


CASES = [
    S.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048),
    S.SliCQParams(44100.0, 32.7, 22050.0, 48, 65536, 16384),
    S.SliCQParams(48000.0, 27.5, 24000.0, 96, 131072, 32768),
    S.SliCQParams(16000.0, 50.0, 8000.0, 96, 16384, 4096),
    S.SliCQParams(48000.0, 50.0, 22000.0, 12, 16384, 4096),
    S.SliCQParams(22050.0, 50.0, 11025.0, 24, 16384, 4096),
    S.SliCQParams(44100.0, 40.0, 22050.0, 24, 8192, 2048),
    S.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512),
    S.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512, mk_policy="const"),
    S.SliCQParams(44100.0, 32.7, 22050.0, 48, 65536, 16384, mk_policy="const"),
    S.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048, window="blackman_harris"),
]


@pytest.mark.parametrize("p", CASES,
                         ids=lambda p: f"fs{int(p.fs)}_B{p.bins_per_octave}_L{p.slice_len}_{p.mk_policy}_{p.window}")
def test_host_layout_matches_oracle(lib, p):
    lay = S.layout(p)
    op = O.make_plan(O.SliCQParams(p.fs, p.fmin, p.fmax, p.bins_per_octave, p.slice_len,
                                   p.trans_len, p.min_filter_len, mk_policy=p.mk_policy,
                                   window=p.window))
    K = op.K
    assert lay["M"].shape[0] == K + 2
    chans = op.sys.channels[: K + 2]
    np.testing.assert_array_equal(lay["M"], [c.M for c in chans])
    np.testing.assert_array_equal(lay["len"], [c.length for c in chans])
    np.testing.assert_array_equal(lay["j0"], [c.j0 for c in chans])
    np.testing.assert_array_equal(lay["off"], op.offsets)
    np.testing.assert_allclose(lay["xi"], op.sys.xi[: K + 2], rtol=1e-13)
    np.testing.assert_allclose(lay["omega"], op.sys.Omega[: K + 2], rtol=1e-13)
    assert lay["coefs_per_slice"] == op.coefs_per_slice


@pytest.mark.parametrize("kw,code", [
    (dict(fmin=0.0), 1), (dict(fmax=10.0), 1), (dict(slice_len=6000), 1),
    (dict(trans_len=3), 1), (dict(trans_len=8192), 1), (dict(bins_per_octave=0), 1),
    (dict(slice_len=1024, trans_len=256), 6), (dict(slice_cluster=3), 1),
    (dict(fmin=23000.0, fmax=30000.0), 1),
    (dict(mk_policy="mult4"), 6),   # mixed-radix band lengths are not built
])
def test_invalid_parameters_are_rejected(lib, kw, code):
    base = dict(fs=44100.0, fmin=50.0, fmax=22050.0, bins_per_octave=12, slice_len=8192,
                trans_len=2048)
    base.update(kw)
    p = S.SliCQParams(**base)
    cp = p.to_c()
    n = ctypes.c_int32()
    c = ctypes.c_int64()
    assert lib.slicq_layout(ctypes.byref(cp), ctypes.byref(n), ctypes.byref(c)) == code


def test_precision_values(lib):
    """slicq_params.precision: the three defined values build a layout (the
    split-precision ones with the same channels), anything else is EINVAL."""
    base = dict(fs=44100.0, fmin=50.0, fmax=22050.0, bins_per_octave=12, slice_len=8192,
                trans_len=2048)
    counts = []
    for prec in ("fp32", "split_fp16", "split_bf16"):
        cp = S.SliCQParams(**base, precision=prec).to_c()
        n, c = ctypes.c_int32(), ctypes.c_int64()
        assert lib.slicq_layout(ctypes.byref(cp), ctypes.byref(n), ctypes.byref(c)) == 0
        counts.append((n.value, c.value))
    assert counts[0] == counts[1] == counts[2]
    for bad in (3, -1, 7):
        cp = S.SliCQParams(**base).to_c()
        cp.precision = bad
        n, c = ctypes.c_int32(), ctypes.c_int64()
        assert lib.slicq_layout(ctypes.byref(cp), ctypes.byref(n), ctypes.byref(c)) == 1


def test_selftest_and_tuning_reject_bad_arguments(lib):
    """Argument checks that need no device: a non-positive wait limit, a
    null plan."""
    lib.slicq_selftest_wait.restype = ctypes.c_int
    lib.slicq_selftest_wait.argtypes = [ctypes.c_int, ctypes.c_int64]
    assert lib.slicq_selftest_wait(0, 0) == 1
    assert lib.slicq_plan_tuning(None, None, None, None) == 1
    assert lib.slicq_plan_check(None) == 1


def test_null_pointers(lib):
    assert lib.slicq_layout(None, None, None) == 1
    assert lib.slicq_plan_info(None, None, None) == 1
    assert lib.slicq_num_slices(None, 100) == 0
    assert lib.slicq_forward(None, None, 1, 1, None, 0, None, 0, None) == 1
    assert lib.slicq_inverse(None, None, 1, 1, None, None, 0, None) == 1
    assert lib.slicq_adjoint(None, None, 1, 1, None, None, 0, None) == 1
    assert lib.slicq_spectrogram(None, None, 1, 1, None, 0, None) == 1


def test_two_layer_views_match_oracle():
    """two_layer: views of the coefficient tensor that place every slice's
    coefficients where the oracle's 2-layer array (Sec. 4.1) has them."""
    torch = pytest.importorskip("torch")
    p = S.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512)
    op = O.make_plan(O.SliCQParams(p.fs, p.fmin, p.fmax, p.bins_per_octave, p.slice_len, p.trans_len))
    x = np.random.default_rng(3).standard_normal(7000)
    c = O.slicq_forward(x, op)
    ct = torch.from_numpy(c)
    lay = S.layout(p)
    for k in (0, 5, op.K, op.K + 1):
        M = int(lay["M"][k])
        s0, s1 = S.two_layer(ct, int(lay["off"][k]), M)
        # views of the coefficients, not copies
        assert s0.untyped_storage().data_ptr() == ct.untyped_storage().data_ptr()
        assert s1.untyped_storage().data_ptr() == ct.untyped_storage().data_ptr()
        ref = O.two_layer_view(c, op, k)            # [2, S M / 2]
        total = ref.shape[1]
        # layer 1 row q starts at time q M; layer 0 row q at q M - M/2
        got1 = s1.reshape(-1).numpy()
        got0 = np.roll(s0.reshape(-1).numpy(), -M // 2)
        np.testing.assert_array_equal(got1, ref[1])
        np.testing.assert_array_equal(got0, ref[0])
        assert got1.shape[0] == total


def test_channel_views_split_packed_coefficients():
    """channel_views: views of channel k = 0..K+1 that equal the oracle's
    per-channel coefficients of every slice."""
    torch = pytest.importorskip("torch")
    p = S.SliCQParams(16000.0, 50.0, 8000.0, 24, 2048, 512)
    op = O.make_plan(O.SliCQParams(p.fs, p.fmin, p.fmax, p.bins_per_octave, p.slice_len, p.trans_len))
    x = np.random.default_rng(4).standard_normal(5000)
    c = O.slicq_forward(x, op)
    ct = torch.from_numpy(c)
    lay = S.layout(p)
    views = S.channel_views(ct, lay["off"], lay["M"])
    assert len(views) == op.K + 2
    xs = O.slicq_slices(x, op)
    for k, v in enumerate(views):
        assert v.untyped_storage().data_ptr() == ct.untyped_storage().data_ptr()
        for m in (0, xs.shape[0] - 1):
            ref = O.nsgt_analysis(xs[m], op.sys, [k])[0]
            np.testing.assert_allclose(v[m].numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max() + 1e-300)
    assert S.SliCQ is S.SliCQPlan


def test_without_a_gpu_calls_fail_with_a_status(lib):
    """No device: plan creation and the device self-test return SLICQ_ECUDA
    (no crash, no fallback), and the Python plan raises."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cp = S.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048).to_c()
    h = ctypes.c_void_p()
    assert lib.slicq_plan_create(ctypes.byref(cp), 0, ctypes.byref(h)) == 3
    assert not h.value
    assert lib.slicq_selftest_wait(0, 1000) == 3
    with pytest.raises(Exception):
        S.SliCQPlan(S.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048))
