// C ABI of libslicq: argument checking, workspace partition and the launch
// sequence of each entry point.  See include/slicq.h for the contract.
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"

namespace slicq {
slicq_status build_tables(slicq_plan* pl);

namespace {
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

slicq_status from_cuda(cudaError_t e) { return e == cudaSuccess ? SLICQ_OK : SLICQ_ECUDA; }

constexpr int kTraceSlots = 4096;

void trace_release(const slicq_plan* pl) {
  for (cudaEvent_t e : pl->trace.ev) cudaEventDestroy(e);
  pl->trace.ev.clear();
  pl->trace.kid.clear();
  pl->trace.n = 0;
  pl->trace.on = false;
}

// Launch `fn` (returning cudaError_t) between two trace events when tracing.
template <class Fn>
cudaError_t traced(const slicq_plan* pl, int32_t kid, cudaStream_t st, Fn fn) {
  auto& tr = pl->trace;
  const bool rec = tr.on && tr.n < kTraceSlots;
  if (rec) cudaEventRecord(tr.ev[2 * tr.n], st);
  const cudaError_t e = fn();
  if (rec) {
    cudaEventRecord(tr.ev[2 * tr.n + 1], st);
    tr.kid[tr.n] = kid;
    ++tr.n;
  }
  return e;
}

void free_plan(slicq_plan* pl) {
  if (!pl) return;
  trace_release(pl);
  if (pl->d_arena) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(pl->device);
    cudaFree(pl->d_arena);
    cudaSetDevice(cur);
  }
  delete pl;
}

// Run fn with the plan's device current, restoring the caller's device.
template <class Fn>
slicq_status on_device(const slicq_plan* pl, Fn fn) {
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return SLICQ_ECUDA;
  if (cur != pl->device && cudaSetDevice(pl->device) != cudaSuccess) return SLICQ_ECUDA;
  const slicq_status st = fn();
  if (cur != pl->device) cudaSetDevice(cur);
  return st;
}
}  // namespace

size_t workspace_layout(const slicq_plan* pl, int64_t n, int64_t batch, void* base, Workspace* ws) {
  Workspace w;
  const int64_t L2 = 2 * pl->N;
  w.L = L2 * std::max<int64_t>(1, (n + L2 - 1) / L2);
  w.S = w.L / pl->N;
  w.spec_stride = pl->N + 2;
  const int64_t slices = batch * w.S;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
  const size_t o_spec = take(sizeof(float2) * slices * w.spec_stride);
  const size_t o_bp = take(sizeof(float2) * slices * std::max(pl->ovl_total, 1));
  const size_t o_op = take(sizeof(float) * slices * 2 * ((pl->params.trans_len + 3) & ~int64_t(3)));
  w.bytes = off;
  if (base) {
    char* b = (char*)base;
    w.spec = (float2*)(b + o_spec);
    w.band_patch = (float2*)(b + o_bp);
    w.ola_patch = (float*)(b + o_op);
  }
  if (ws) *ws = w;
  return off;
}

size_t workspace_layout_rows(const slicq_plan* pl, int64_t rows, void* base, Workspace* ws) {
  Workspace w;
  w.S = rows;
  w.L = 0;
  w.spec_stride = pl->N + 2;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
  const size_t o_spec = take(sizeof(float2) * rows * w.spec_stride);
  const size_t o_bp = take(sizeof(float2) * rows * std::max(pl->ovl_total, 1));
  const size_t o_op = take(sizeof(float) * rows * 2 * ((pl->params.trans_len + 3) & ~int64_t(3)));
  w.bytes = off;
  if (base) {
    char* b = (char*)base;
    w.spec = (float2*)(b + o_spec);
    w.band_patch = (float2*)(b + o_bp);
    w.ola_patch = (float*)(b + o_op);
  }
  if (ws) *ws = w;
  return off;
}

}  // namespace slicq

using namespace slicq;

extern "C" {

const char* slicq_status_string(slicq_status s) {
  switch (s) {
    case SLICQ_OK: return "SLICQ_OK";
    case SLICQ_EINVAL: return "SLICQ_EINVAL: invalid parameter or null pointer";
    case SLICQ_ENOMEM: return "SLICQ_ENOMEM: allocation failed";
    case SLICQ_ECUDA: return "SLICQ_ECUDA: CUDA runtime error";
    case SLICQ_ESIZE: return "SLICQ_ESIZE: buffer too small";
    case SLICQ_ETIMEOUT: return "SLICQ_ETIMEOUT: bounded device wait gave up";
    case SLICQ_EUNSUPPORTED: return "SLICQ_EUNSUPPORTED: parameters outside this build";
  }
  return "SLICQ_UNKNOWN";
}

int32_t slicq_abi_version(void) { return SLICQ_ABI_VERSION; }

slicq_status slicq_layout(const slicq_params* p, int32_t* n_channels, int64_t* coefs_per_slice) {
  if (!p) return SLICQ_EINVAL;
  slicq_plan tmp;
  const slicq_status st = build_layout(p, &tmp);
  if (st != SLICQ_OK) return st;
  if (n_channels) *n_channels = tmp.n_channels;
  if (coefs_per_slice) *coefs_per_slice = tmp.coefs_per_slice;
  return SLICQ_OK;
}

slicq_status slicq_layout_tables(const slicq_params* p, int32_t n_channels, int32_t* h_M,
                                 int64_t* h_off, int64_t* h_j0, int32_t* h_len, double* h_xi,
                                 double* h_omega) {
  if (!p) return SLICQ_EINVAL;
  slicq_plan tmp;
  const slicq_status st = build_layout(p, &tmp);
  if (st != SLICQ_OK) return st;
  if (n_channels < tmp.n_channels) return SLICQ_ESIZE;
  for (int k = 0; k < tmp.n_channels; ++k) {
    const BandDesc& b = tmp.bands[k];
    if (h_M) h_M[k] = 1 << b.log2M;
    if (h_off) h_off[k] = b.coef_off;
    if (h_j0) h_j0[k] = b.j0;
    if (h_len) h_len[k] = b.len;
    if (h_xi) h_xi[k] = tmp.xi[k];
    if (h_omega) h_omega[k] = tmp.omega[k];
  }
  return SLICQ_OK;
}

slicq_status slicq_plan_create(const slicq_params* p, int device, slicq_plan** out) {
  if (!p || !out) return SLICQ_EINVAL;
  *out = nullptr;
  slicq_plan* pl = new (std::nothrow) slicq_plan();
  if (!pl) return SLICQ_ENOMEM;
  slicq_status st = build_layout(p, pl);
  if (st != SLICQ_OK) { delete pl; return st; }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    delete pl;
    return device < 0 ? SLICQ_EINVAL : SLICQ_ECUDA;
  }
  pl->device = device;
  st = on_device(pl, [&] { return build_tables(pl); });
  if (st != SLICQ_OK) { free_plan(pl); return st; }
  *out = pl;
  return SLICQ_OK;
}

void slicq_plan_destroy(slicq_plan* plan) { free_plan(plan); }

slicq_status slicq_plan_tuning(const slicq_plan* plan, int32_t* slice_cluster, int32_t* band_ctas_analysis,
                               int32_t* band_ctas_synthesis) {
  if (!plan) return SLICQ_EINVAL;
  if (slice_cluster) *slice_cluster = plan->C;
  if (band_ctas_analysis) *band_ctas_analysis = plan->n_cta_a;
  if (band_ctas_synthesis) *band_ctas_synthesis = plan->n_cta_s;
  return SLICQ_OK;
}

slicq_status slicq_plan_check(const slicq_plan* plan) {
  if (!plan) return SLICQ_EINVAL;
  return on_device(plan, [&]() -> slicq_status {
    if (cudaDeviceSynchronize() != cudaSuccess) return SLICQ_ECUDA;
    int flag = 0;
    if (cudaMemcpy(&flag, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SLICQ_ECUDA;
    if (!flag) return SLICQ_OK;
    const int zero = 0;
    if (cudaMemcpy(plan->d_err, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return SLICQ_ECUDA;
    return SLICQ_ETIMEOUT;
  });
}

slicq_status slicq_plan_info(const slicq_plan* plan, int32_t* n_channels, int64_t* coefs_per_slice) {
  if (!plan) return SLICQ_EINVAL;
  if (n_channels) *n_channels = plan->n_channels;
  if (coefs_per_slice) *coefs_per_slice = plan->coefs_per_slice;
  return SLICQ_OK;
}

int64_t slicq_num_slices(const slicq_plan* plan, int64_t n_samples) {
  if (!plan || n_samples < 1) return 0;
  const int64_t L2 = 2 * plan->N;
  return 2 * ((n_samples + L2 - 1) / L2);
}

slicq_status slicq_workspace_size(const slicq_plan* plan, int64_t n_samples, int64_t batch, size_t* bytes) {
  if (!plan || !bytes || n_samples < 1 || batch < 1) return SLICQ_EINVAL;
  *bytes = workspace_layout(plan, n_samples, batch, nullptr, nullptr);
  return SLICQ_OK;
}

static slicq_status check_common(const slicq_plan* plan, int64_t n, int64_t batch, const void* a,
                                 const void* b, void* work, size_t work_bytes, Workspace* ws) {
  if (!plan || !a || !b || !work || n < 1 || batch < 1) return SLICQ_EINVAL;
  if ((reinterpret_cast<uintptr_t>(work) & 255) != 0) return SLICQ_EINVAL;
  const size_t need = workspace_layout(plan, n, batch, work, ws);
  if (ws->L >= (int64_t(1) << 31)) return SLICQ_EUNSUPPORTED;  // positions are 32-bit
  if (work_bytes < need) return SLICQ_ESIZE;
  return SLICQ_OK;
}

slicq_status slicq_forward(const slicq_plan* plan, const float* d_f, int64_t n_samples, int64_t batch,
                           float* d_coef, int64_t coef_capacity, void* d_work, size_t work_bytes,
                           cudaStream_t stream) {
  Workspace ws;
  slicq_status st = check_common(plan, n_samples, batch, d_f, d_coef, d_work, work_bytes, &ws);
  if (st != SLICQ_OK) return st;
  if ((reinterpret_cast<uintptr_t>(d_coef) & 7) != 0) return SLICQ_EINVAL;
  if (coef_capacity < batch * ws.S * plan->coefs_per_slice) return SLICQ_ESIZE;
  return on_device(plan, [&] {
    cudaError_t e = traced(plan, 0, stream, [&] {
      return launch_slice_forward(plan, d_f, n_samples, batch, ws, stream); });
    if (e == cudaSuccess)
      e = traced(plan, 1, stream, [&] {
        return launch_band_analysis(plan, ws, batch, reinterpret_cast<float2*>(d_coef), stream); });
    return from_cuda(e);
  });
}

static slicq_status synthesis(const slicq_plan* plan, const float* d_coef, int64_t n_samples, int64_t batch,
                              float* d_out, void* d_work, size_t work_bytes, cudaStream_t stream,
                              SynthKind kind, const SynthModify* mod = nullptr) {
  Workspace ws;
  slicq_status st = check_common(plan, n_samples, batch, d_coef, d_out, d_work, work_bytes, &ws);
  if (st != SLICQ_OK) return st;
  if ((reinterpret_cast<uintptr_t>(d_coef) & 7) != 0) return SLICQ_EINVAL;
  return on_device(plan, [&] {
    cudaError_t e = traced(plan, 2, stream, [&] {
      return launch_band_synthesis(plan, reinterpret_cast<const float2*>(d_coef), batch, kind, ws, stream,
                                   nullptr, mod); });
    if (e == cudaSuccess && !plan->shared.empty())
      e = traced(plan, 4, stream, [&] { return launch_band_boundaries(plan, batch, ws, stream); });
    if (e == cudaSuccess)
      e = traced(plan, 3, stream, [&] {
        return launch_slice_inverse(plan, n_samples, batch, kind, ws, d_out, stream); });
    if (e == cudaSuccess)
      e = traced(plan, 5, stream, [&] { return launch_slice_ola(plan, n_samples, batch, ws, d_out, stream); });
    return from_cuda(e);
  });
}

slicq_status slicq_inverse(const slicq_plan* plan, const float* d_coef, int64_t n_samples, int64_t batch,
                           float* d_out, void* d_work, size_t work_bytes, cudaStream_t stream) {
  return synthesis(plan, d_coef, n_samples, batch, d_out, d_work, work_bytes, stream, kSynthInverse);
}

slicq_status slicq_adjoint(const slicq_plan* plan, const float* d_coef, int64_t n_samples, int64_t batch,
                           float* d_out, void* d_work, size_t work_bytes, cudaStream_t stream) {
  return synthesis(plan, d_coef, n_samples, batch, d_out, d_work, work_bytes, stream, kSynthAdjoint);
}

slicq_status slicq_inverse_modified(const slicq_plan* plan, const float* d_coef, int64_t n_samples,
                                    int64_t batch, int32_t channel_shift, const float* d_mask, float* d_out,
                                    void* d_work, size_t work_bytes, cudaStream_t stream) {
  if (!plan) return SLICQ_EINVAL;
  if (channel_shift != 0 && plan->params.mk_policy != SLICQ_MK_CONST) return SLICQ_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_mask) & 3) != 0) return SLICQ_EINVAL;
  const SynthModify mod{channel_shift, d_mask};
  return synthesis(plan, d_coef, n_samples, batch, d_out, d_work, work_bytes, stream, kSynthInverse, &mod);
}

slicq_status slicq_spectrogram(const slicq_plan* plan, const float* d_coef, int64_t n_samples, int64_t batch,
                               float* d_out, int64_t out_capacity, cudaStream_t stream) {
  if (!plan || !d_coef || !d_out || n_samples < 1 || batch < 1) return SLICQ_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_coef) & 7) != 0) return SLICQ_EINVAL;
  const int64_t S = slicq_num_slices(plan, n_samples);
  if (S * plan->N >= (int64_t(1) << 31)) return SLICQ_EUNSUPPORTED;  // positions are 32-bit
  if (out_capacity < batch * S * (plan->coefs_per_slice / 2)) return SLICQ_ESIZE;
  return on_device(plan, [&] {
    return from_cuda(traced(plan, 6, stream, [&] {
      return launch_spectrogram(plan, reinterpret_cast<const float2*>(d_coef), S, batch, d_out, stream); }));
  });
}

slicq_status slicq_plan_table(const slicq_plan* plan, int32_t which, float* h_out, int64_t count,
                              int64_t* n_out) {
  if (!plan || !h_out) return SLICQ_EINVAL;
  const float* src = nullptr;
  int64_t n = 0;
  switch (which) {
    case 0: src = plan->d_ga; n = plan->win_total; break;
    case 1: src = plan->d_gs; n = plan->win_total; break;
    case 2: src = plan->d_gadj; n = plan->win_total; break;
    case 3: src = plan->d_hw; n = plan->params.trans_len + 1; break;
    default: return SLICQ_EINVAL;
  }
  if (count < n) return SLICQ_ESIZE;
  if (n_out) *n_out = n;
  return on_device(plan, [&] {
    return from_cuda(cudaMemcpy(h_out, src, sizeof(float) * n, cudaMemcpyDeviceToHost));
  });
}

slicq_status slicq_trace_enable(const slicq_plan* plan, int32_t enable) {
  if (!plan) return SLICQ_EINVAL;
  return on_device(plan, [&] {
    trace_release(plan);
    if (!enable) return SLICQ_OK;
    auto& tr = plan->trace;
    tr.ev.resize(2 * kTraceSlots);
    tr.kid.assign(kTraceSlots, -1);
    for (auto& e : tr.ev)
      if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; trace_release(plan); return SLICQ_ECUDA; }
    tr.on = true;
    return SLICQ_OK;
  });
}

slicq_status slicq_trace_read(const slicq_plan* plan, int32_t* h_kernel, float* h_ms, int32_t cap,
                              int32_t* n_out) {
  if (!plan || !n_out) return SLICQ_EINVAL;
  return on_device(plan, [&] {
    auto& tr = plan->trace;
    const int n = std::min(tr.n, std::max(cap, 0));
    for (int i = 0; i < n; ++i) {
      float ms = 0.f;
      if (cudaEventSynchronize(tr.ev[2 * i + 1]) != cudaSuccess ||
          cudaEventElapsedTime(&ms, tr.ev[2 * i], tr.ev[2 * i + 1]) != cudaSuccess)
        return SLICQ_ECUDA;
      if (h_kernel) h_kernel[i] = tr.kid[i];
      if (h_ms) h_ms[i] = ms;
    }
    *n_out = n;
    tr.n = 0;
    return SLICQ_OK;
  });
}

}  // extern "C"
