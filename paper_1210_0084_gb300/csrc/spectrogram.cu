// sliCQ spectrogram (Sec. 4.1): |s^0 + s^1|^2 of the 2-layer array.
//
// Slice m's coefficient n of channel k sits in layer m mod 2 at time index
// t = n + (m-1) M_k/2 (circular in S M_k/2).  With H = M_k/2 and t = qH + r
// (r < H) the two slices covering t are q + 1 (n = r, the first half of its
// channel-k coefficients) and q (n = H + r, the second half), so
//   spec_k[t] = |c[q+1][off_k + r] + c[q][off_k + H + r]|^2   (slices mod S).
// A thread computes one t: every coefficient is read once, and the
// plan's half-coefficient table gives the channel of thread i.
#include "fft_common.cuh"
#include "internal.h"

namespace slicq {
namespace {

__global__ void __launch_bounds__(256) spectrogram_kernel(const float2* __restrict__ coef, float* out,
                                                          const int2* __restrict__ half_chan, int64_t cps,
                                                          int S, int64_t row_base) {
  pdl_launch_dependents();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // half-coefficient of a slice
  const int2 ch = i < cps / 2 ? __ldg(half_chan + i) : make_int2(0, 1);
  pdl_wait();  // the coefficients
  if (i >= cps / 2) return;
  const int64_t row = row_base + blockIdx.y;  // b S + q
  const int64_t b = row / S;
  const int q = (int)(row - b * S);
  const int off = ch.x;
  const int H = 1 << (ch.y - 1);
  const int r = (int)(i - off / 2);
  const int q1 = q + 1 == S ? 0 : q + 1;
  const float2* cb = coef + b * S * cps;
  const float2 x1 = __ldcs(cb + q1 * cps + off + r);
  const float2 x0 = __ldcs(cb + q * cps + off + H + r);
  const float2 v = c_add(x0, x1);
  out[b * (S * cps / 2) + (int64_t)S * (off / 2) + (int64_t)q * H + r] = v.x * v.x + v.y * v.y;
}

}  // namespace

cudaError_t launch_spectrogram(const slicq_plan* pl, const float2* coef, int64_t S, int64_t batch,
                               float* out, cudaStream_t st) {
  const int64_t cps = pl->coefs_per_slice;
  const unsigned bx = (unsigned)((cps / 2 + 255) / 256);
  const int64_t rows = batch * S;
  for (int64_t r0 = 0; r0 < rows; r0 += kMaxGridY) {
    dim3 grid(bx, (unsigned)(rows - r0 < kMaxGridY ? rows - r0 : kMaxGridY));
    const cudaError_t e = launch_pdl(spectrogram_kernel, grid, dim3(256), 0, st, coef, out,
                                     (const int2*)pl->d_half_chan, cps, (int)S, r0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace slicq
