"""Python binding of libslicq (argument marshalling only).

Every step of the transform runs in the library's CUDA kernels; this module
only checks shapes and dtypes, allocates outputs and workspaces with PyTorch
and passes raw pointers and the current CUDA stream through the C ABI of
``include/slicq.h``.  Importing it loads ``lib/libslicq.so`` and raises if the
library is missing: there is no fallback implementation.

    plan = SliCQPlan(SliCQParams(fs=44100, fmin=32.7, fmax=22050,
                                 bins_per_octave=48, slice_len=65536,
                                 trans_len=16384))
    c = plan.forward(x)          # x: float32 [batch, n] on the GPU
    y = plan.inverse(c, n)       # perfect reconstruction (Prop. 3)
    g = plan.adjoint(c, n)       # Re(A^H c), the gradient of the analysis

Citations: Holighaus, Doerfler, Velasco, Grill, arXiv:1210.0084 —
Algorithms 1-4, Proposition 2 (dual windows), Table 1 (channel layout).
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Dict, Optional, Tuple

import numpy as np

__all__ = [
    "SliCQParams", "SliCQPlan", "SliCQError", "SliCQFunction", "slicq_transform",
    "layout", "lib_path", "load_library", "STATUS", "SliCQBatch", "SliCQStream",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
STATUS = {0: "SLICQ_OK", 1: "SLICQ_EINVAL", 2: "SLICQ_ENOMEM", 3: "SLICQ_ECUDA",
          4: "SLICQ_ESIZE", 5: "SLICQ_ETIMEOUT", 6: "SLICQ_EUNSUPPORTED"}


def lib_path() -> str:
    return os.environ.get("SLICQ_LIB", os.path.join(_PKG, "lib", "libslicq.so"))


class SliCQError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("fs", ctypes.c_double), ("fmin", ctypes.c_double), ("fmax", ctypes.c_double),
                ("bins_per_octave", ctypes.c_int32), ("min_filter_len", ctypes.c_int32),
                ("slice_len", ctypes.c_int64), ("trans_len", ctypes.c_int64),
                ("window", ctypes.c_int32), ("mk_policy", ctypes.c_int32),
                ("slice_cluster", ctypes.c_int32), ("precision", ctypes.c_int32)]


_lib = None


def load_library():
    """Load libslicq.so once (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise OSError(f"libslicq.so not built at {path}; run "
                      "`python -m paper_1210_0084_gb300.build`")
    L = ctypes.CDLL(path)
    P, I32, I64, VP, SZ = (ctypes.POINTER(_Params), ctypes.c_int32, ctypes.c_int64,
                           ctypes.c_void_p, ctypes.c_size_t)
    sig = {
        "slicq_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "slicq_abi_version": (I32, []),
        "slicq_layout": (ctypes.c_int, [P, ctypes.POINTER(I32), ctypes.POINTER(I64)]),
        "slicq_layout_tables": (ctypes.c_int, [P, I32, VP, VP, VP, VP, VP, VP]),
        "slicq_plan_create": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(VP)]),
        "slicq_plan_destroy": (None, [VP]),
        "slicq_plan_info": (ctypes.c_int, [VP, ctypes.POINTER(I32), ctypes.POINTER(I64)]),
        "slicq_plan_check": (ctypes.c_int, [VP]),
        "slicq_selftest_wait": (ctypes.c_int, [ctypes.c_int, I64]),
        "slicq_plan_tuning": (ctypes.c_int, [VP, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                             ctypes.POINTER(I32)]),
        "slicq_num_slices": (I64, [VP, I64]),
        "slicq_workspace_size": (ctypes.c_int, [VP, I64, I64, ctypes.POINTER(SZ)]),
        "slicq_forward": (ctypes.c_int, [VP, VP, I64, I64, VP, I64, VP, SZ, VP]),
        "slicq_inverse": (ctypes.c_int, [VP, VP, I64, I64, VP, VP, SZ, VP]),
        "slicq_adjoint": (ctypes.c_int, [VP, VP, I64, I64, VP, VP, SZ, VP]),
        "slicq_plan_table": (ctypes.c_int, [VP, I32, VP, I64, ctypes.POINTER(I64)]),
        "slicq_trace_enable": (ctypes.c_int, [VP, I32]),
        "slicq_spectrogram": (ctypes.c_int, [VP, VP, I64, I64, VP, I64, VP]),
        "slicq_inverse_modified": (ctypes.c_int, [VP, VP, I64, I64, I32, VP, VP, VP, SZ, VP]),
        "slicq_stream_create": (ctypes.c_int, [VP, ctypes.POINTER(VP)]),
        "slicq_stream_destroy": (None, [VP]),
        "slicq_stream_hop": (I64, [VP]),
        "slicq_stream_forward": (ctypes.c_int, [VP, VP, VP, VP]),
        "slicq_stream_inverse": (ctypes.c_int, [VP, VP, VP, VP]),
        "slicq_stream_reset": (ctypes.c_int, [VP, VP]),
        "slicq_batch_create": (ctypes.c_int, [VP, I32, VP, VP, I32, ctypes.POINTER(VP)]),
        "slicq_batch_destroy": (None, [VP]),
        "slicq_batch_layout": (ctypes.c_int, [VP, VP, VP, VP, ctypes.POINTER(I64), ctypes.POINTER(I64),
                                              ctypes.POINTER(SZ)]),
        "slicq_batch_forward": (ctypes.c_int, [VP, VP, VP, VP, SZ, VP]),
        "slicq_batch_inverse": (ctypes.c_int, [VP, VP, VP, VP, SZ, VP]),
        "slicq_trace_read": (ctypes.c_int, [VP, VP, VP, I32, ctypes.POINTER(I32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, what: str):
    if status != 0:
        raise SliCQError(status, what)


@dataclass(frozen=True)
class SliCQParams:
    """Parameters of one sliCQ system (Table 1 and Sec. 4; see slicq.h)."""

    fs: float
    fmin: float
    fmax: float
    bins_per_octave: int
    slice_len: int
    trans_len: int
    min_filter_len: int = 16
    slice_cluster: int = 0
    mk_policy: str = "pow2"   # "pow2" or "const" (rectangular representation)
    window: str = "hann"      # "hann" or "blackman_harris"
    precision: str = "fp32"   # "fp32", "split_fp16" or "split_bf16" (band DFT stages)

    def to_c(self) -> _Params:
        mk = {"pow2": 0, "mult4": 1, "const": 2}[self.mk_policy]
        win = {"hann": 0, "blackman_harris": 1}[self.window]
        prec = {"fp32": 0, "split_fp16": 1, "split_bf16": 2}[self.precision]
        return _Params(float(self.fs), float(self.fmin), float(self.fmax),
                       int(self.bins_per_octave), int(self.min_filter_len),
                       int(self.slice_len), int(self.trans_len), win, mk,
                       int(self.slice_cluster), prec)


def layout(p: SliCQParams) -> Dict[str, np.ndarray]:
    """Host-only channel layout (no GPU): M, off, j0, len, xi, omega per channel."""
    L = load_library()
    cp = p.to_c()
    nch = ctypes.c_int32()
    cps = ctypes.c_int64()
    _check(L.slicq_layout(ctypes.byref(cp), ctypes.byref(nch), ctypes.byref(cps)), "slicq_layout")
    n = nch.value
    out = {"M": np.zeros(n, np.int32), "off": np.zeros(n, np.int64), "j0": np.zeros(n, np.int64),
           "len": np.zeros(n, np.int32), "xi": np.zeros(n, np.float64),
           "omega": np.zeros(n, np.float64)}
    _check(L.slicq_layout_tables(ctypes.byref(cp), n, *(out[k].ctypes.data for k in
                                                         ("M", "off", "j0", "len", "xi", "omega"))),
           "slicq_layout_tables")
    out["coefs_per_slice"] = int(cps.value)
    return out


class SliCQPlan:
    """A plan on one CUDA device: channel layout and FP64-derived tables."""

    def __init__(self, params: SliCQParams, device: Optional[int] = None):
        import torch
        self._torch = torch
        self.params = params
        self.lib = load_library()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        cp = params.to_c()
        _check(self.lib.slicq_plan_create(ctypes.byref(cp), self.device, ctypes.byref(h)),
               "slicq_plan_create")
        self._h = h
        nch = ctypes.c_int32()
        cps = ctypes.c_int64()
        _check(self.lib.slicq_plan_info(h, ctypes.byref(nch), ctypes.byref(cps)), "slicq_plan_info")
        self.n_channels = nch.value
        self.coefs_per_slice = cps.value
        self._work: Dict[Tuple[int, int], "torch.Tensor"] = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                self.lib.slicq_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    # ------------------------------------------------------------------ info
    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def slice_cluster(self) -> int:
        """CTAs per slice the plan's slice kernels run (measured choice when
        the parameters leave it at 0)."""
        c = ctypes.c_int32()
        _check(self.lib.slicq_plan_tuning(self._h, ctypes.byref(c), None, None), "slicq_plan_tuning")
        return c.value

    def check(self):
        """Synchronise and raise SliCQError if a launch of this plan reported a
        device-side failure (a split-precision tensor-core wait that gave up)."""
        _check(self.lib.slicq_plan_check(self._h), "slicq_plan_check")

    def num_slices(self, n: int) -> int:
        return int(self.lib.slicq_num_slices(self._h, int(n)))

    def workspace_bytes(self, n: int, batch: int) -> int:
        sz = ctypes.c_size_t()
        _check(self.lib.slicq_workspace_size(self._h, int(n), int(batch), ctypes.byref(sz)),
               "slicq_workspace_size")
        return sz.value

    def workspace(self, n: int, batch: int):
        """Device workspace for (n, batch) on the current stream, cached on the
        plan: calls on different streams get different workspaces, so they may
        run concurrently."""
        key = (int(n), int(batch), self._torch.cuda.current_stream(self.device).cuda_stream)
        w = self._work.get(key)
        if w is None:
            nb = self.workspace_bytes(n, batch)
            w = self._torch.zeros(max(nb, 256), dtype=self._torch.uint8,
                                  device=f"cuda:{self.device}")
            self._work[key] = w
        return w

    def table(self, which: int) -> np.ndarray:
        """Copy of a plan table (0 analysis, 1 synthesis, 2 adjoint windows, 3 Tukey)."""
        cap = 1 << 26
        buf = np.zeros(cap, np.float32)
        n = ctypes.c_int64()
        _check(self.lib.slicq_plan_table(self._h, int(which), buf.ctypes.data, cap, ctypes.byref(n)),
               "slicq_plan_table")
        return buf[: n.value].copy()

    KERNEL_NAMES = ("slice_forward", "band_analysis", "band_synthesis", "slice_inverse",
                    "band_boundary", "slice_ola", "spectrogram")

    def trace(self, enable: bool = True):
        """Start (or stop) recording CUDA events around every kernel launch."""
        _check(self.lib.slicq_trace_enable(self._h, 1 if enable else 0), "slicq_trace_enable")

    def trace_read(self, cap: int = 4096):
        """[(kernel name, ms)] of the launches traced since the last read."""
        kid = np.zeros(cap, np.int32)
        ms = np.zeros(cap, np.float32)
        n = ctypes.c_int32()
        _check(self.lib.slicq_trace_read(self._h, kid.ctypes.data, ms.ctypes.data, cap,
                                         ctypes.byref(n)), "slicq_trace_read")
        return [(self.KERNEL_NAMES[k], float(t)) for k, t in zip(kid[: n.value], ms[: n.value])]

    # ------------------------------------------------------------ transforms
    def _stream(self):
        return ctypes.c_void_p(self._torch.cuda.current_stream(self.device).cuda_stream)

    def _as_batch(self, x):
        t = self._torch
        if x.dtype != t.float32 or not x.is_cuda:
            raise TypeError("expected a float32 CUDA tensor")
        squeeze = x.dim() == 1
        x2 = x.reshape(1, -1) if squeeze else x
        if x2.dim() != 2:
            raise ValueError("expected [n] or [batch, n]")
        return x2.contiguous(), squeeze

    def forward(self, x, out=None):
        """Coefficients complex64 [batch, S, coefs_per_slice] (Algorithm 3)."""
        t = self._torch
        x2, squeeze = self._as_batch(x)
        batch, n = x2.shape
        S = self.num_slices(n)
        if out is None:
            out = t.empty((batch, S, self.coefs_per_slice), dtype=t.complex64, device=x2.device)
        w = self.workspace(n, batch)
        _check(self.lib.slicq_forward(self._h, x2.data_ptr(), n, batch, out.data_ptr(), out.numel(),
                                      w.data_ptr(), w.numel(), self._stream()), "slicq_forward")
        return out[0] if squeeze else out

    def _synth(self, fn, c, n, out, what):
        t = self._torch
        if c.dtype != t.complex64 or not c.is_cuda:
            raise TypeError("expected complex64 CUDA coefficients")
        squeeze = c.dim() == 2
        c3 = c.unsqueeze(0) if squeeze else c
        batch = c3.shape[0]
        S = self.num_slices(n)
        if tuple(c3.shape[1:]) != (S, self.coefs_per_slice):
            raise ValueError(f"coefficients must be [batch, {S}, {self.coefs_per_slice}]")
        c3 = c3.contiguous()
        if out is None:
            out = t.empty((batch, n), dtype=t.float32, device=c3.device)
        w = self.workspace(n, batch)
        _check(fn(self._h, c3.data_ptr(), int(n), batch, out.data_ptr(), w.data_ptr(), w.numel(),
                  self._stream()), what)
        return out[0] if squeeze else out

    def inverse(self, c, n: int, out=None):
        """Real signal [batch, n] from coefficients (Algorithm 4, canonical dual)."""
        return self._synth(self.lib.slicq_inverse, c, n, out, "slicq_inverse")

    def adjoint(self, c, n: int, out=None):
        """Re(A^H c) [batch, n]: the gradient of the analysis map."""
        return self._synth(self.lib.slicq_adjoint, c, n, out, "slicq_adjoint")

    def inverse_modified(self, c, n: int, shift: int = 0, mask=None, out=None):
        """Real signal from modified coefficients (Sec. 6): channel k takes
        channel k - shift, modulated to its own centre frequency, then times
        ``mask`` (float32, same shape as ``c``); see slicq_inverse_modified."""
        t = self._torch
        squeeze = c.dim() == 2
        c3 = (c.unsqueeze(0) if squeeze else c).contiguous()
        batch = c3.shape[0]
        mptr = None
        if mask is not None:
            m3 = (mask.unsqueeze(0) if mask.dim() == 2 else mask).contiguous()
            if m3.dtype != t.float32 or tuple(m3.shape) != tuple(c3.shape):
                raise ValueError("mask must be float32 with the coefficients' shape")
            mptr = m3.data_ptr()
        if out is None:
            out = t.empty((batch, n), dtype=t.float32, device=c3.device)
        w = self.workspace(n, batch)
        _check(self.lib.slicq_inverse_modified(self._h, c3.data_ptr(), int(n), batch, int(shift), mptr,
                                               out.data_ptr(), w.data_ptr(), w.numel(), self._stream()),
               "slicq_inverse_modified")
        return out[0] if squeeze else out

    def spectrogram(self, c, n: int, out=None):
        """sliCQ spectrogram |s^0 + s^1|^2 (Sec. 4.1), float32
        [batch, S * coefs_per_slice / 2]; channel k's S M_k / 2 time indices
        start at S off_k / 2 (see ``spectrogram_blocks``)."""
        t = self._torch
        if c.dtype != t.complex64 or not c.is_cuda:
            raise TypeError("expected complex64 CUDA coefficients")
        squeeze = c.dim() == 2
        c3 = (c.unsqueeze(0) if squeeze else c).contiguous()
        batch = c3.shape[0]
        S = self.num_slices(n)
        if tuple(c3.shape[1:]) != (S, self.coefs_per_slice):
            raise ValueError(f"coefficients must be [batch, {S}, {self.coefs_per_slice}]")
        if out is None:
            out = t.empty((batch, S * (self.coefs_per_slice // 2)), dtype=t.float32, device=c3.device)
        _check(self.lib.slicq_spectrogram(self._h, c3.data_ptr(), int(n), batch, out.data_ptr(),
                                          out.numel(), self._stream()), "slicq_spectrogram")
        return out[0] if squeeze else out

    def channels(self, c):
        """Per-channel views [..., S, M_k] of packed coefficients (see ``channel_views``)."""
        lay = layout(self.params)
        return channel_views(c, lay["off"], lay["M"])

    def two_layer(self, c, k: int):
        """(s0, s1) of channel k as views of the coefficients (see ``two_layer``)."""
        lay = layout(self.params)
        return two_layer(c, int(lay["off"][k]), int(lay["M"][k]))

    def spectrogram_blocks(self, spec, n: int):
        """Per-channel views [.., S M_k / 2] of a spectrogram from ``spectrogram``."""
        lay = layout(self.params)
        S = self.num_slices(n)
        return [spec[..., S * int(o) // 2: S * (int(o) + int(m)) // 2]
                for o, m in zip(lay["off"], lay["M"])]


def channel_views(c, offsets, lengths):
    """Per-channel views of packed coefficients (no copy): for c of shape
    [..., S, coefs_per_slice] the list of c[..., off_k:off_k + M_k], i.e. the
    coefficients c^m_{n,k} of channel k as [..., S, M_k] (Algorithm 3's
    output as a list over k = 0..K+1)."""
    return [c[..., int(o):int(o) + int(m)] for o, m in zip(offsets, lengths)]


def two_layer(c, off_k: int, M_k: int):
    """The 2-layer array s^l_{n,k} of Sec. 4.1 for one channel, as views of
    the coefficients (no copy).

    c is [batch, S, coefs_per_slice] (or [S, coefs_per_slice]); channel k
    occupies columns off_k .. off_k + M_k - 1 of every slice.  Slice m's
    coefficient n^s sits in layer l = m mod 2 at time index
    ((m - 1) M_k / 2 + n^s) mod (S M_k / 2); slices of one parity tile the
    time axis.  Returns (s0, s1), each [..., S/2, M_k] with s^l[q, n^s] =
    slice l + 2q: s1 row q covers time indices q M_k .. q M_k + M_k - 1, s0
    row q covers q M_k - M_k/2 .. q M_k + M_k/2 - 1 (row 0's first half wraps
    to the end).  s0 + s1 at equal time indices is the sliCQ spectrogram's
    argument."""
    blk = c[..., off_k:off_k + M_k]
    return blk[..., 0::2, :], blk[..., 1::2, :]


# The transform object under the name the PyTorch layer of the design uses.
SliCQ = SliCQPlan


def _autograd():
    import torch

    class _SliCQFunction(torch.autograd.Function):
        """Forward sliCQ with the hand-written adjoint kernel as its backward."""

        @staticmethod
        def forward(ctx, x, plan: SliCQPlan):
            ctx.plan = plan
            ctx.n = x.shape[-1]
            ctx.shape = x.shape
            return plan.forward(x)

        @staticmethod
        def backward(ctx, grad_c):
            g = ctx.plan.adjoint(grad_c.contiguous(), ctx.n)
            return g.reshape(ctx.shape), None

    return _SliCQFunction


_FN = None


def SliCQFunction():
    """The torch.autograd.Function class (created lazily so that importing this
    module does not import torch)."""
    global _FN
    if _FN is None:
        _FN = _autograd()
    return _FN


def slicq_transform(x, plan: SliCQPlan):
    """Differentiable forward sliCQ of a float32 CUDA tensor [batch, n]."""
    return SliCQFunction().apply(x, plan)


class SliCQStream:
    """Streaming sliCQ of one plan: N = slice_len / 2 samples per call.

    ``forward(block)`` takes the next N samples (float32 CUDA) and returns
    slice m (complex64 [coefs_per_slice]); ``inverse(c)`` takes one slice's
    coefficients and returns the N output samples (m-1)N + a0 + 1 .. mN + a0.
    """

    def __init__(self, plan: SliCQPlan):
        import torch
        self._torch = torch
        self.plan = plan
        self.lib = plan.lib
        h = ctypes.c_void_p()
        _check(self.lib.slicq_stream_create(plan.handle, ctypes.byref(h)), "slicq_stream_create")
        self._h = h
        self.hop = int(self.lib.slicq_stream_hop(plan.handle))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.slicq_stream_destroy(h)
            self._h = None

    def _stream(self):
        return ctypes.c_void_p(self._torch.cuda.current_stream(self.plan.device).cuda_stream)

    def forward(self, block, out=None):
        t = self._torch
        if block.dtype != t.float32 or not block.is_cuda or block.numel() != self.hop:
            raise ValueError(f"expected {self.hop} float32 CUDA samples")
        block = block.contiguous()
        if out is None:
            out = t.empty(self.plan.coefs_per_slice, dtype=t.complex64, device=block.device)
        _check(self.lib.slicq_stream_forward(self._h, block.data_ptr(), out.data_ptr(), self._stream()),
               "slicq_stream_forward")
        return out

    def inverse(self, coef, out=None):
        t = self._torch
        if coef.dtype != t.complex64 or not coef.is_cuda or coef.numel() != self.plan.coefs_per_slice:
            raise ValueError("expected one slice of complex64 CUDA coefficients")
        coef = coef.contiguous()
        if out is None:
            out = t.empty(self.hop, dtype=t.float32, device=coef.device)
        _check(self.lib.slicq_stream_inverse(self._h, coef.data_ptr(), out.data_ptr(), self._stream()),
               "slicq_stream_inverse")
        return out

    def reset(self):
        _check(self.lib.slicq_stream_reset(self._h, self._stream()), "slicq_stream_reset")


class SliCQBatch:
    """A ragged batch: clips of different lengths over several plans of one
    slice geometry, transformed in one call (plans as concurrent branches)."""

    def __init__(self, plans, clip_plan, clip_samples):
        import torch
        self._torch = torch
        self.plans = list(plans)
        self.lib = load_library()
        self.device = self.plans[0].device
        n = len(clip_plan)
        self.n_clips = n
        self.clip_plan = np.asarray(clip_plan, np.int32)
        self.clip_samples = np.asarray(clip_samples, np.int64)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(self.lib.slicq_batch_create(arr, len(self.plans), self.clip_plan.ctypes.data,
                                           self.clip_samples.ctypes.data, n, ctypes.byref(h)),
               "slicq_batch_create")
        self._h = h
        self.sig_off = np.zeros(n, np.int64)
        self.coef_off = np.zeros(n, np.int64)
        self.slices = np.zeros(n, np.int64)
        st, ct = ctypes.c_int64(), ctypes.c_int64()
        wb = ctypes.c_size_t()
        _check(self.lib.slicq_batch_layout(h, self.sig_off.ctypes.data, self.coef_off.ctypes.data,
                                           self.slices.ctypes.data, ctypes.byref(st), ctypes.byref(ct),
                                           ctypes.byref(wb)), "slicq_batch_layout")
        self.sig_total, self.coef_total, self.work_bytes = st.value, ct.value, wb.value
        self.work = torch.zeros(max(self.work_bytes, 256), dtype=torch.uint8, device=f"cuda:{self.device}")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                self.lib.slicq_batch_destroy(h)
            except Exception:
                pass
            self._h = None

    def pack(self, signals):
        """Concatenate per-clip float32 arrays into the batch's signal layout."""
        t = self._torch
        buf = t.zeros(self.sig_total, dtype=t.float32, device=f"cuda:{self.device}")
        for c, x in enumerate(signals):
            xt = t.as_tensor(np.asarray(x, np.float32)).to(buf.device)
            buf[self.sig_off[c]: self.sig_off[c] + self.clip_samples[c]] = xt
        return buf

    def clip_signal(self, sig, c):
        return sig[self.sig_off[c]: self.sig_off[c] + self.clip_samples[c]]

    def clip_coefs(self, coef, c):
        cps = self.plans[self.clip_plan[c]].coefs_per_slice
        o = int(self.coef_off[c])
        return coef[o: o + int(self.slices[c]) * cps].view(int(self.slices[c]), cps)

    def _stream(self):
        return ctypes.c_void_p(self._torch.cuda.current_stream(self.device).cuda_stream)

    def forward(self, sig, out=None):
        t = self._torch
        if out is None:
            out = t.empty(self.coef_total, dtype=t.complex64, device=sig.device)
        _check(self.lib.slicq_batch_forward(self._h, sig.data_ptr(), out.data_ptr(), self.work.data_ptr(),
                                            self.work.numel(), self._stream()), "slicq_batch_forward")
        return out

    def inverse(self, coef, out=None):
        t = self._torch
        if out is None:
            out = t.zeros(self.sig_total, dtype=t.float32, device=coef.device)
        _check(self.lib.slicq_batch_inverse(self._h, coef.data_ptr(), out.data_ptr(), self.work.data_ptr(),
                                            self.work.numel(), self._stream()), "slicq_batch_inverse")
        return out
