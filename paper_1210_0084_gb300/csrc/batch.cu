// Ragged batches: many clips of different lengths, sample rates and bins
// per octave in one call.
//
// Clips that share a plan form one flat list of slice rows; a row table tells
// the slice kernels which clip (offset, length) and slice index each row is.
// The band kernels already work on flat rows.  Each plan's kernel chain runs
// on its own stream, forked from and joined back to the caller's stream with
// events, so the chains of different plans run concurrently.  Capturing one
// call in a CUDA graph therefore records the whole batch, plans as parallel
// branches, for a single-launch replay.
#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

using namespace slicq;

namespace {
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct SubBatch {
  const slicq_plan* pl = nullptr;
  int64_t rows = 0;
  int64_t coef_off = 0;      // complex values
  size_t work_off = 0, work_bytes = 0;
  RowDesc* d_rows = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};
}  // namespace

struct slicq_batch {
  int device = 0;
  int n_clips = 0;
  std::vector<SubBatch> subs;
  std::vector<int64_t> sig_off, coef_off, slices;
  int64_t sig_total = 0, coef_total = 0;
  size_t work_total = 0;
  void* d_rows = nullptr;
  cudaEvent_t fork = nullptr;
};

namespace {
void destroy(slicq_batch* b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  for (auto& s : b->subs) {
    if (s.st) cudaStreamDestroy(s.st);
    if (s.done) cudaEventDestroy(s.done);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_rows) cudaFree(b->d_rows);
  cudaSetDevice(cur);
  delete b;
}

template <class Fn>
slicq_status run(const slicq_batch* b, cudaStream_t stream, Fn per_plan) {
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return SLICQ_ECUDA;
  if (cur != b->device && cudaSetDevice(b->device) != cudaSuccess) return SLICQ_ECUDA;
  cudaError_t e = cudaEventRecord(b->fork, stream);
  for (size_t i = 0; e == cudaSuccess && i < b->subs.size(); ++i) {
    const SubBatch& sb = b->subs[i];
    if (sb.rows == 0) continue;
    e = cudaStreamWaitEvent(sb.st, b->fork, 0);
    if (e == cudaSuccess) e = per_plan(sb);
    if (e == cudaSuccess) e = cudaEventRecord(sb.done, sb.st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, sb.done, 0);
  }
  if (cur != b->device) cudaSetDevice(cur);
  return e == cudaSuccess ? SLICQ_OK : SLICQ_ECUDA;
}
}  // namespace

extern "C" {

slicq_status slicq_batch_create(const slicq_plan* const* plans, int32_t n_plans, const int32_t* clip_plan,
                                const int64_t* clip_samples, int32_t n_clips, slicq_batch** out) {
  if (!plans || n_plans < 1 || !clip_plan || !clip_samples || n_clips < 1 || !out) return SLICQ_EINVAL;
  *out = nullptr;
  for (int p = 0; p < n_plans; ++p) {
    if (!plans[p]) return SLICQ_EINVAL;
    if (plans[p]->device != plans[0]->device || plans[p]->N != plans[0]->N ||
        plans[p]->params.trans_len != plans[0]->params.trans_len)
      return SLICQ_EUNSUPPORTED;  // one slice geometry per batch
  }
  for (int c = 0; c < n_clips; ++c)
    if (clip_plan[c] < 0 || clip_plan[c] >= n_plans || clip_samples[c] < 1) return SLICQ_EINVAL;
  slicq_batch* b = new (std::nothrow) slicq_batch();
  if (!b) return SLICQ_ENOMEM;
  b->device = plans[0]->device;
  b->n_clips = n_clips;
  b->sig_off.assign(n_clips, 0);
  b->coef_off.assign(n_clips, 0);
  b->slices.assign(n_clips, 0);
  const int64_t L2 = 2 * plans[0]->N;
  int64_t off = 0;
  for (int c = 0; c < n_clips; ++c) {  // clips in order, 16-byte aligned starts
    b->sig_off[c] = off;
    const int64_t L = L2 * ((clip_samples[c] + L2 - 1) / L2);
    if (L >= (int64_t(1) << 31)) { delete b; return SLICQ_EUNSUPPORTED; }
    b->slices[c] = 2 * L / L2;
    off += (clip_samples[c] + 3) & ~int64_t(3);
  }
  b->sig_total = off;
  // rows, coefficients and workspace grouped by plan
  std::vector<std::vector<RowDesc>> rows(n_plans);
  b->subs.resize(n_plans);
  int64_t coef = 0;
  size_t work = 0;
  for (int p = 0; p < n_plans; ++p) {
    SubBatch& sb = b->subs[p];
    sb.pl = plans[p];
    sb.coef_off = coef;
    for (int c = 0; c < n_clips; ++c) {
      if (clip_plan[c] != p) continue;
      b->coef_off[c] = coef + sb.rows * plans[p]->coefs_per_slice;
      const int64_t S = b->slices[c];
      for (int64_t m = 0; m < S; ++m)
        rows[p].push_back(RowDesc{b->sig_off[c], (int32_t)clip_samples[c], (int32_t)(S * L2 / 2),
                                  (int32_t)S, (int32_t)m, sb.rows});
      sb.rows += S;
    }
    coef += sb.rows * plans[p]->coefs_per_slice;
    sb.work_off = work;
    sb.work_bytes = workspace_layout_rows(plans[p], std::max<int64_t>(sb.rows, 1), nullptr, nullptr);
    work = align256(work + sb.work_bytes);
  }
  b->coef_total = coef;
  b->work_total = work;
  // device row tables and per-plan streams
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  size_t total_rows = 0;
  for (auto& r : rows) total_rows += r.size();
  cudaError_t e = cudaMalloc(&b->d_rows, sizeof(RowDesc) * std::max<size_t>(total_rows, 1));
  size_t ro = 0;
  for (int p = 0; e == cudaSuccess && p < n_plans; ++p) {
    SubBatch& sb = b->subs[p];
    sb.d_rows = reinterpret_cast<RowDesc*>(b->d_rows) + ro;
    if (!rows[p].empty())
      e = cudaMemcpy(sb.d_rows, rows[p].data(), sizeof(RowDesc) * rows[p].size(), cudaMemcpyHostToDevice);
    ro += rows[p].size();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sb.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sb.done, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  cudaSetDevice(cur);
  if (e != cudaSuccess) {
    destroy(b);
    return e == cudaErrorMemoryAllocation ? SLICQ_ENOMEM : SLICQ_ECUDA;
  }
  *out = b;
  return SLICQ_OK;
}

void slicq_batch_destroy(slicq_batch* batch) { destroy(batch); }

slicq_status slicq_batch_layout(const slicq_batch* b, int64_t* h_sig_off, int64_t* h_coef_off,
                                int64_t* h_slices, int64_t* sig_total, int64_t* coef_total,
                                size_t* work_bytes) {
  if (!b) return SLICQ_EINVAL;
  for (int c = 0; c < b->n_clips; ++c) {
    if (h_sig_off) h_sig_off[c] = b->sig_off[c];
    if (h_coef_off) h_coef_off[c] = b->coef_off[c];
    if (h_slices) h_slices[c] = b->slices[c];
  }
  if (sig_total) *sig_total = b->sig_total;
  if (coef_total) *coef_total = b->coef_total;
  if (work_bytes) *work_bytes = b->work_total;
  return SLICQ_OK;
}

slicq_status slicq_batch_forward(const slicq_batch* b, const float* d_sig, float* d_coef, void* d_work,
                                 size_t work_bytes, cudaStream_t stream) {
  if (!b || !d_sig || !d_coef || !d_work) return SLICQ_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_work) & 255) || (reinterpret_cast<uintptr_t>(d_coef) & 7) ||
      (reinterpret_cast<uintptr_t>(d_sig) & 15))
    return SLICQ_EINVAL;
  if (work_bytes < b->work_total) return SLICQ_ESIZE;
  return run(b, stream, [&](const SubBatch& sb) {
    Workspace ws;
    workspace_layout_rows(sb.pl, sb.rows, (char*)d_work + sb.work_off, &ws);
    float2* coef = reinterpret_cast<float2*>(d_coef) + sb.coef_off;
    cudaError_t e = launch_slice_forward(sb.pl, d_sig, 0, 1, ws, sb.st, sb.d_rows);
    if (e == cudaSuccess) e = launch_band_analysis(sb.pl, ws, 1, coef, sb.st);
    return e;
  });
}

slicq_status slicq_batch_inverse(const slicq_batch* b, const float* d_coef, float* d_sig_out, void* d_work,
                                 size_t work_bytes, cudaStream_t stream) {
  if (!b || !d_sig_out || !d_coef || !d_work) return SLICQ_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_work) & 255) || (reinterpret_cast<uintptr_t>(d_coef) & 7) ||
      (reinterpret_cast<uintptr_t>(d_sig_out) & 15))
    return SLICQ_EINVAL;
  if (work_bytes < b->work_total) return SLICQ_ESIZE;
  return run(b, stream, [&](const SubBatch& sb) {
    Workspace ws;
    workspace_layout_rows(sb.pl, sb.rows, (char*)d_work + sb.work_off, &ws);
    const float2* coef = reinterpret_cast<const float2*>(d_coef) + sb.coef_off;
    cudaError_t e = launch_band_synthesis(sb.pl, coef, 1, kSynthInverse, ws, sb.st);
    if (e == cudaSuccess) e = launch_band_boundaries(sb.pl, 1, ws, sb.st);
    if (e == cudaSuccess) e = launch_slice_inverse(sb.pl, 0, 1, kSynthInverse, ws, d_sig_out, sb.st, sb.d_rows);
    if (e == cudaSuccess) e = launch_slice_ola(sb.pl, 0, 1, ws, d_sig_out, sb.st, sb.d_rows);
    return e;
  });
}

}  // extern "C"
