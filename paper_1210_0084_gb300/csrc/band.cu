// Band stage launchers, the FP32 band kernels and the boundary kernel that
// adds the partial sums of bins several band groups share.  The kernels
// themselves are in band_kernels.cuh.
#include "band_kernels.cuh"

namespace slicq {
namespace {

// Bins covered by several groups: spectrum = the groups' partial sums in
// group order.  Thread i takes the i-th shared bin in kBoundarySlices
// consecutive slices.
constexpr int kBoundarySlices = 4;

__global__ void __launch_bounds__(256) band_boundary_kernel(BandArgs a, int nshared, int64_t total) {
  pdl_launch_dependents();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int4 sb = i < nshared ? __ldg(a.shared + i) : make_int4(0, 0, 0, 0);
  pdl_wait();
  if (i >= nshared) return;
  const int64_t s0 = (a.slice_base + blockIdx.y) * kBoundarySlices;
  float2 v[kBoundarySlices];
#pragma unroll
  for (int u = 0; u < kBoundarySlices; ++u) {
    v[u] = make_float2(0.f, 0.f);
    if (s0 + u < total) {
      const float2* row = a.patch + (s0 + u) * (int64_t)a.ovl_total + sb.y;
      v[u] = __ldcs(row);
      for (int j = 1; j < sb.z; ++j) v[u] = c_add(v[u], __ldcs(row + j));
    }
  }
#pragma unroll
  for (int u = 0; u < kBoundarySlices; ++u)
    if (s0 + u < total) a.spec[(s0 + u) * a.spec_stride + sb.x] = v[u];
}

BandArgs make_args(const slicq_plan* pl, const Workspace& ws, const float* win) {
  BandArgs a{};
  a.bands = pl->d_bands;
  a.groups = pl->d_groups;
  a.thread_band = pl->d_thread_band;
  a.slot_base = pl->d_slot_base;
  a.shared = pl->d_shared;
  a.win = win;
  a.twband = pl->d_twband;
  a.tw4096 = pl->d_tw4096;
  a.spec = ws.spec;
  a.spec_stride = ws.spec_stride;
  a.cps = pl->coefs_per_slice;
  a.patch = ws.band_patch;
  a.ovl_total = pl->ovl_total;
  a.N = (int)pl->N;
  a.err = pl->d_err;
  return a;
}

// The persistent band kernels of the plan's precision.
BandKernels kernels_of(const slicq_plan* pl) {
  switch (pl->params.precision) {
    case SLICQ_PREC_SPLIT_FP16: return band_kernels_split_fp16();
    case SLICQ_PREC_SPLIT_BF16: return band_kernels_split_bf16();
    default: return {band_analysis_persistent_kernel<kPrecFP32>, band_synthesis_persistent_kernel<kPrecFP32>};
  }
}

}  // namespace

int band_ctas_per_sm(const slicq_plan* pl, bool synthesis) {
  int n = 0;
  const BandKernels bk = kernels_of(pl);
  const void* k = synthesis ? (const void*)bk.synthesis : (const void*)bk.analysis;
  const int smem = synthesis ? pl->band_smem_s : pl->band_smem_p;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBandThreads, smem) != cudaSuccess)
    return 1;
  return std::max(1, n);
}

cudaError_t launch_band_analysis(const slicq_plan* pl, const Workspace& ws, int64_t batch,
                                 float2* coef, cudaStream_t st, long long* cycles) {
  BandArgs a = make_args(pl, ws, pl->d_ga);
  a.coef = coef;
  a.cycles = cycles;
  a.total = batch * ws.S;
  const BandKernel kern = kernels_of(pl).analysis;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->band_smem_p);
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, dim3(pl->n_cta_a), dim3(kBandThreads),
                    (size_t)pl->band_smem_p, st, a, (const int2*)pl->d_cta_map_a, (const int*)pl->d_lanes_a);
}

cudaError_t launch_band_synthesis(const slicq_plan* pl, const float2* coef, int64_t batch,
                                  SynthKind kind, const Workspace& ws, cudaStream_t st,
                                  long long* cycles, const SynthModify* mod) {
  BandArgs a = make_args(pl, ws, kind == kSynthInverse ? pl->d_gs : pl->d_gadj);
  a.coef = const_cast<float2*>(coef);
  a.cycles = cycles;
  if (mod && (mod->shift != 0 || mod->mask)) {
    a.modify = 1;
    a.shift = mod->shift;
    a.mask = mod->mask;
    a.K = pl->K;
    a.S_clip = (int)ws.S;
    a.jc = pl->d_jc;
  }
  a.total = batch * ws.S;
  const BandKernel kern = kernels_of(pl).synthesis;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->band_smem_s);
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, dim3(pl->n_cta_s), dim3(kBandThreads),
                    (size_t)pl->band_smem_s, st, a, (const int2*)pl->d_cta_map_s, (const int*)pl->d_lanes_s);
}

cudaError_t launch_band_boundaries(const slicq_plan* pl, int64_t batch, const Workspace& ws,
                                   cudaStream_t st) {
  const int nshared = (int)pl->shared.size();
  if (nshared == 0) return cudaSuccess;
  BandArgs a = make_args(pl, ws, nullptr);
  const int64_t total = batch * ws.S;
  const int64_t chunks = (total + kBoundarySlices - 1) / kBoundarySlices;
  for (int64_t c0 = 0; c0 < chunks; c0 += kMaxGridY) {
    a.slice_base = c0;
    dim3 grid((unsigned)((nshared + 255) / 256), (unsigned)(chunks - c0 < kMaxGridY ? chunks - c0 : kMaxGridY));
    const cudaError_t e = launch_pdl(band_boundary_kernel, grid, dim3(256), 0, st, a, nshared, total);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace slicq
