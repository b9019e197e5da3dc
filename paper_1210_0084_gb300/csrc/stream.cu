// Streaming sliCQ (real-time mode, bounded delay): one slice per call.
//
// Forward: slice m covers input samples [(m-1)N, (m+1)N) (Algorithm 3), so
// every N new samples complete one slice.  The stream keeps the last 2N
// samples in a device ring (time t at t mod 2N); the new block overwrites the
// older half, and the slice kernel reads the ring as a clip of length 2N with
// slice index m mod 2, whose circular indexing then addresses exactly the 2N
// samples of slice m.  Samples before the start are zero.
//
// Inverse: slice m contributes to output samples mN + d, |d| < a0 + M
// (a0 = (N - M)/2, Algorithm 4).  Once slice m is in, every sample up to
// mN + a0 is complete, so each call emits the N samples
// (m-1)N + a0 + 1 .. mN + a0: the transition shared with slice m-1 (its
// side kept from the previous call plus this slice's side) and this slice's
// direct region.  The output ring holds 2N samples; the emitted block is
// copied to the caller's buffer.  Before the first slice the earlier side of
// the transition is zero.
#include <new>

#include "internal.h"

using namespace slicq;

struct slicq_stream {
  const slicq_plan* pl = nullptr;
  int64_t m_fwd = 0, m_inv = 0;  // slices processed by each direction
  void* mem = nullptr;           // one device allocation
  size_t mem_bytes = 0;
  float* ring_in = nullptr;      // 2N input samples
  float* ring_out = nullptr;     // 2N output samples
  RowDesc* rows = nullptr;       // [2]: the ring as a clip of 2N samples, slice index 0 and 1
  void* work = nullptr;          // workspace laid out for two rows (two transition slots)
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace of one slice row whose transition patch has the two alternating slots.
Workspace stream_workspace(const slicq_stream* s) {
  Workspace ws;
  workspace_layout_rows(s->pl, 2, s->work, &ws);
  ws.S = 1;
  return ws;
}

template <class Fn>
slicq_status on_plan_device(const slicq_plan* pl, Fn fn) {
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return SLICQ_ECUDA;
  if (cur != pl->device && cudaSetDevice(pl->device) != cudaSuccess) return SLICQ_ECUDA;
  const cudaError_t e = fn();
  if (cur != pl->device) cudaSetDevice(cur);
  return e == cudaSuccess ? SLICQ_OK : (e == cudaErrorMemoryAllocation ? SLICQ_ENOMEM : SLICQ_ECUDA);
}

}  // namespace

extern "C" {

slicq_status slicq_stream_create(const slicq_plan* plan, slicq_stream** out) {
  if (!plan || !out) return SLICQ_EINVAL;
  *out = nullptr;
  slicq_stream* s = new (std::nothrow) slicq_stream();
  if (!s) return SLICQ_ENOMEM;
  s->pl = plan;
  const int64_t N = plan->N;
  const size_t o_in = 0;
  const size_t o_out = align256(o_in + sizeof(float) * 2 * N);
  const size_t o_rows = align256(o_out + sizeof(float) * 2 * N);
  const size_t o_work = align256(o_rows + sizeof(RowDesc) * 2);
  s->mem_bytes = o_work + workspace_layout_rows(plan, 2, nullptr, nullptr);
  const slicq_status st = on_plan_device(plan, [&] {
    cudaError_t e = cudaMalloc(&s->mem, s->mem_bytes);
    if (e != cudaSuccess) return e;
    char* b = static_cast<char*>(s->mem);
    s->ring_in = reinterpret_cast<float*>(b + o_in);
    s->ring_out = reinterpret_cast<float*>(b + o_out);
    s->rows = reinterpret_cast<RowDesc*>(b + o_rows);
    s->work = b + o_work;
    const RowDesc rows[2] = {RowDesc{0, (int32_t)(2 * N), (int32_t)(2 * N), 2, 0, 0},
                             RowDesc{0, (int32_t)(2 * N), (int32_t)(2 * N), 2, 1, 0}};
    e = cudaMemset(s->mem, 0, s->mem_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(s->rows, rows, sizeof(rows), cudaMemcpyHostToDevice);
    return e;
  });
  if (st != SLICQ_OK) {
    if (s->mem) on_plan_device(plan, [&] { return cudaFree(s->mem); });
    delete s;
    return st;
  }
  *out = s;
  return SLICQ_OK;
}

void slicq_stream_destroy(slicq_stream* s) {
  if (!s) return;
  if (s->mem) on_plan_device(s->pl, [&] { return cudaFree(s->mem); });
  delete s;
}

slicq_status slicq_stream_reset(slicq_stream* s, cudaStream_t stream) {
  if (!s) return SLICQ_EINVAL;
  s->m_fwd = s->m_inv = 0;
  const int64_t N = s->pl->N;
  return on_plan_device(s->pl, [&] {
    // the rings and the transition sides; the row tables stay
    cudaError_t e = cudaMemsetAsync(s->ring_in, 0, sizeof(float) * 2 * N, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ring_out, 0, sizeof(float) * 2 * N, stream);
    if (e == cudaSuccess) {
      const Workspace ws = stream_workspace(s);
      e = cudaMemsetAsync(ws.ola_patch, 0, sizeof(float) * 2 * 2 * ((s->pl->params.trans_len + 3) & ~int64_t(3)),
                          stream);
    }
    return e;
  });
}

slicq_status slicq_stream_forward(slicq_stream* s, const float* d_in, float* d_coef, cudaStream_t stream) {
  if (!s || !d_in || !d_coef) return SLICQ_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_coef) & 7) != 0) return SLICQ_EINVAL;
  const slicq_plan* pl = s->pl;
  const int64_t N = pl->N;
  const int mm = (int)(s->m_fwd & 1);
  const slicq_status st = on_plan_device(pl, [&] {
    // the new block [mN, (m+1)N) goes to ring half m mod 2
    cudaError_t e = cudaMemcpyAsync(s->ring_in + mm * N, d_in, sizeof(float) * N, cudaMemcpyDeviceToDevice, stream);
    const Workspace ws = stream_workspace(s);
    if (e == cudaSuccess) e = launch_slice_forward(pl, s->ring_in, 2 * N, 1, ws, stream, s->rows + mm);
    if (e == cudaSuccess) e = launch_band_analysis(pl, ws, 1, reinterpret_cast<float2*>(d_coef), stream);
    return e;
  });
  if (st == SLICQ_OK) ++s->m_fwd;
  return st;
}

slicq_status slicq_stream_inverse(slicq_stream* s, const float* d_coef, float* d_out, cudaStream_t stream) {
  if (!s || !d_coef || !d_out) return SLICQ_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_coef) & 7) != 0) return SLICQ_EINVAL;
  const slicq_plan* pl = s->pl;
  const int64_t N = pl->N;
  const int64_t a0 = (N - pl->params.trans_len) / 2;
  const int mm = (int)(s->m_inv & 1);
  const slicq_status st = on_plan_device(pl, [&] {
    const Workspace ws = stream_workspace(s);
    cudaError_t e = launch_band_synthesis(pl, reinterpret_cast<const float2*>(d_coef), 1, kSynthInverse, ws, stream);
    if (e == cudaSuccess) e = launch_band_boundaries(pl, 1, ws, stream);
    // direct region into the ring, both transition sides into their slots
    if (e == cudaSuccess) e = launch_slice_inverse(pl, 2 * N, 1, kSynthInverse, ws, s->ring_out, stream, s->rows + mm);
    // the transition shared with slice m - 1 (row of slice m - 1)
    if (e == cudaSuccess) e = launch_slice_ola(pl, 2 * N, 1, ws, s->ring_out, stream, s->rows + (1 - mm));
    // emit (m-1)N + a0 + 1 .. mN + a0 (ring positions mod 2N)
    const int64_t start = (((s->m_inv - 1) * N + a0 + 1) % (2 * N) + 2 * N) % (2 * N);
    const int64_t first = std::min<int64_t>(N, 2 * N - start);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_out, s->ring_out + start, sizeof(float) * first, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess && first < N)
      e = cudaMemcpyAsync(d_out + first, s->ring_out, sizeof(float) * (N - first), cudaMemcpyDeviceToDevice, stream);
    return e;
  });
  if (st == SLICQ_OK) ++s->m_inv;
  return st;
}

int64_t slicq_stream_hop(const slicq_plan* plan) { return plan ? plan->N : 0; }

}  // extern "C"
