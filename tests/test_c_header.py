"""The boundary is a C ABI: a plain C99 program includes include/slicq.h,
links libslicq.so and calls the host-only entry points (no GPU needed)."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1210_0084_gb300 import slicq as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stdio.h>
#include "slicq.h"

int main(void) {
  slicq_params p = {0};
  p.fs = 44100.0; p.fmin = 50.0; p.fmax = 22050.0; p.bins_per_octave = 12;
  p.min_filter_len = 16; p.slice_len = 8192; p.trans_len = 2048;
  p.window = SLICQ_WIN_HANN; p.mk_policy = SLICQ_MK_POW2; p.precision = SLICQ_PREC_FP32;
  int32_t nch = 0; int64_t cps = 0;
  if (slicq_layout(&p, &nch, &cps) != SLICQ_OK) return 1;
  p.slice_len = 6000;
  slicq_status bad = slicq_layout(&p, &nch, &cps);
  p.slice_len = 8192;
  printf("%d %d %lld %d %s\n", (int)slicq_abi_version(), (int)nch, (long long)cps, (int)bad,
         slicq_status_string(SLICQ_ETIMEOUT));
  return 0;
}
"""


def test_c_program_uses_the_header_and_library(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda_inc = None
    for d in ("/usr/local/cuda/include", os.path.join(os.environ.get("CUDA_HOME", ""), "include")):
        if d and os.path.exists(os.path.join(d, "cuda_runtime_api.h")):
            cuda_inc = d
            break
    if cuda_inc is None:
        pytest.skip("no CUDA headers")
    lib = S.lib_path()
    if not os.path.exists(lib):
        pytest.skip("library not built")
    src = tmp_path / "use_slicq.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_slicq"
    libdir = os.path.dirname(lib)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                    str(src), "-o", str(exe), "-L", libdir, "-lslicq", f"-Wl,-rpath,{libdir}"],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    lay = S.layout(S.SliCQParams(44100.0, 50.0, 22050.0, 12, 8192, 2048))
    assert int(out[0]) == 2
    assert int(out[1]) == lay["M"].shape[0]
    assert int(out[2]) == int(np.sum(lay["M"]))
    assert int(out[3]) == 1  # SLICQ_EINVAL: slice length not a power of two
    assert len(out) >= 5
