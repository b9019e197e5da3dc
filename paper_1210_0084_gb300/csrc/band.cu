// Band stage of the sliCQ: one CTA per (slice, group of consecutive channels).
//
// Analysis (Algorithm 1, inner loop): for channel k with support J_k and
// M_k coefficients, y[r] = sum_{j in J_k, j = r mod M_k} X[j] g_k[j] / sqrt(2N)
// (periodisation of f_hat * conj(g_k)), then c = unnormalised backward
// DFT_{M_k}(y), which gives c_{n,k} = <f_hat, M_{-n a_k} g_k> (eq. CQ_coeff).
// The window multiply and the fold are the pass-1 loads of the transform;
// the slice spectrum X (bins 0..N of the real-input spectrum) comes from the
// slice kernel, bins beyond N are read as conjugates.
//
// Synthesis (Algorithm 2, loop over k and line "sum_k f_k g~_k"): Y = forward
// DFT_{M_k}(c_k), then the half spectrum receives Y[j mod M_k] w g~_k[j] at
// j and its conjugate at -j (when those bins lie in 0..N).  Channels are
// accumulated in shared memory colour by colour (channels of one colour have
// disjoint footprints), so every bin is summed in a fixed order; bins shared
// with the neighbouring group are combined by whichever of the two CTAs
// arrives second (a + b == b + a), so the result is deterministic and no
// zero-fill pass is needed.
#include <cooperative_groups.h>

#include "fft_common.cuh"
#include "internal.h"

namespace slicq {
namespace {

struct BandArgs {
  const BandDesc* __restrict__ bands;
  const GroupDesc* __restrict__ groups;
  const BoundaryDesc* __restrict__ bounds;
  const int16_t* __restrict__ thread_band;
  const float* __restrict__ win;   // window table of this launch
  TwiddleTables tw;
  float2* spec;                    // [slice][spec_stride]
  int64_t slice_base;              // first slice of this launch
  int64_t spec_stride;
  float2* coef;                    // [slice][cps]
  int64_t cps;
  float2* patch;                   // [slice][G-1][2][max_ovl]
  uint32_t* cnt;                   // [slice][G-1]
  int G, max_ovl;
  int N, log2N2;                   // N and log2(2N)
};

// ------------------------------------------------------------ analysis ---

template <int LOGM>
__device__ __forceinline__ void analysis_pass1(const BandArgs& a, const BandDesc& bd, int tt,
                                               const float2* __restrict__ X, float2* buf) {
  constexpr int M = 1 << LOGM;
  const int twoN = 2 * a.N;
  const float* __restrict__ g = a.win + bd.win_off;
  auto load = [&](int idx) -> float2 {
    const int o = (idx - bd.j0) & (M - 1);
    if (o >= bd.len) return make_float2(0.f, 0.f);
    int b = bd.j0 + o;
    if (b >= twoN) b -= twoN;
    const float2 x = (b <= a.N) ? X[b] : c_conj(X[twoN - b]);
    return c_scale(x, __ldg(g + o));
  };
  team_pass1<LOGM, +1>(tt, buf, load);
}

template <int LOGM>
__device__ __forceinline__ void analysis_pass2(const BandArgs& a, const BandDesc& bd, int tt,
                                               const float2* buf, float2* __restrict__ out) {
  using T = Team<LOGM>;
  float2 res[T::HELD];
  team_pass2<LOGM, +1>(tt, buf, a.tw, a.log2N2 - LOGM, res);
#pragma unroll
  for (int i = 0; i < T::J2; ++i)
#pragma unroll
    for (int r = 0; r < T::R2; ++r)
      __stcs(out + team_out_index<LOGM>(tt, i, r), res[i * T::R2 + r]);
}

__global__ void __launch_bounds__(kBandThreads) band_analysis_kernel(BandArgs a) {
  extern __shared__ float2 sm[];
  const int g = blockIdx.x;
  const int64_t s = a.slice_base + blockIdx.y;
  const int t = threadIdx.x;
  const int k = a.thread_band[g * kBandThreads + t];
  BandDesc bd{};
  if (k >= 0) bd = a.bands[k];
  const int tt = t - bd.tofs;
  const float2* X = a.spec + s * a.spec_stride;
  float2* buf = sm + bd.smem_off;
  if (k >= 0) {
    switch (bd.log2M) {
      case 4: analysis_pass1<4>(a, bd, tt, X, buf); break;
      case 5: analysis_pass1<5>(a, bd, tt, X, buf); break;
      case 6: analysis_pass1<6>(a, bd, tt, X, buf); break;
      case 7: analysis_pass1<7>(a, bd, tt, X, buf); break;
      case 8: analysis_pass1<8>(a, bd, tt, X, buf); break;
      case 9: analysis_pass1<9>(a, bd, tt, X, buf); break;
      case 10: analysis_pass1<10>(a, bd, tt, X, buf); break;
    }
  }
  __syncthreads();
  if (k >= 0) {
    float2* out = a.coef + s * a.cps + bd.coef_off;
    switch (bd.log2M) {
      case 4: analysis_pass2<4>(a, bd, tt, buf, out); break;
      case 5: analysis_pass2<5>(a, bd, tt, buf, out); break;
      case 6: analysis_pass2<6>(a, bd, tt, buf, out); break;
      case 7: analysis_pass2<7>(a, bd, tt, buf, out); break;
      case 8: analysis_pass2<8>(a, bd, tt, buf, out); break;
      case 9: analysis_pass2<9>(a, bd, tt, buf, out); break;
      case 10: analysis_pass2<10>(a, bd, tt, buf, out); break;
    }
  }
}

// ----------------------------------------------------------- synthesis ---

// Barrier that threads may reach from different code locations (the band
// pipelines below are different template instances per band length; every
// thread of the CTA executes the same number of these barriers).
__device__ __forceinline__ void cta_sync() { asm volatile("barrier.sync 0;" ::: "memory"); }

// MIRROR = false: Y w g~ into bin j (if j <= N); true: its conjugate into -j.
template <int LOGM, bool MIRROR>
__device__ __forceinline__ void synthesis_accumulate(const BandArgs& a, const BandDesc& bd, int tt,
                                                     const float2* res, float2* acc, int acc_lo) {
  using T = Team<LOGM>;
  constexpr int M = 1 << LOGM;
  const int twoN = 2 * a.N;
  const float* __restrict__ g = a.win + bd.win_off;
#pragma unroll
  for (int i = 0; i < T::J2; ++i) {
#pragma unroll
    for (int r = 0; r < T::R2; ++r) {
      const int idx = team_out_index<LOGM>(tt, i, r);
      const int o = (idx - bd.j0) & (M - 1);
      if (o < bd.len) {
        int b = bd.j0 + o;
        if (b >= twoN) b -= twoN;
        const float2 v = c_scale(res[i * T::R2 + r], __ldg(g + o));
        if (!MIRROR) {
          if (b <= a.N) acc[b - acc_lo] = c_add(acc[b - acc_lo], v);
        } else {
          const int mb = b == 0 ? 0 : twoN - b;
          if (mb <= a.N) acc[mb - acc_lo] = c_add(acc[mb - acc_lo], c_conj(v));
        }
      }
    }
  }
}

// Hand a shared boundary to the neighbour or, if the neighbour already
// handed over its half, add both halves and store them.  side 0 = this
// group is left of the boundary.  No waiting: the first arriver leaves.
__device__ __forceinline__ void boundary_combine(const BandArgs& a, int64_t s, int bd, int side,
                                                 const float2* acc, int acc_lo, float2* spec,
                                                 int* s_flag) {
  const BoundaryDesc b = a.bounds[bd];
  const int64_t slot = s * (a.G - 1) + bd;
  float2* mine = a.patch + (slot * 2 + side) * a.max_ovl;
  const float2* other = a.patch + (slot * 2 + (1 - side)) * a.max_ovl;
  for (int h = b.lo + threadIdx.x; h < b.hi; h += blockDim.x) mine[h - b.lo] = acc[h - acc_lo];
  __threadfence();
  cta_sync();
  if (threadIdx.x == 0) {
    // 0 -> 1 for the first arriver, 1 -> 0 for the second (ready for the next call)
    const unsigned old = atomicInc(a.cnt + slot, 1u);
    *s_flag = (old == 1u);
  }
  cta_sync();
  if (*s_flag) {
    __threadfence();
    for (int h = b.lo + threadIdx.x; h < b.hi; h += blockDim.x)
      spec[h] = c_add(acc[h - acc_lo], __ldcg(other + (h - b.lo)));
  }
  cta_sync();
}

// The whole synthesis pipeline of one CTA as seen by one thread.  LOGM = 0
// is a thread without a band: it only takes part in the barriers and the
// CTA-wide loops.
template <int LOGM>
__device__ __forceinline__ void synthesis_pipeline(const BandArgs& a, const GroupDesc& gd,
                                                   const BandDesc& bd, int tt, int64_t s,
                                                   float2* sm, int* s_flag) {
  constexpr int LG = LOGM ? LOGM : 4;
  using T = Team<LG>;
  float2 res[T::HELD];
  float2* buf = sm + bd.smem_off;
  if (LOGM) {
    const float2* c = a.coef + s * a.cps + bd.coef_off;
    team_pass1<LG, -1>(tt, buf, [&](int idx) { return __ldcs(c + idx); });
  }
  cta_sync();
  if (LOGM) team_pass2<LG, -1>(tt, buf, a.tw, a.log2N2 - LG, res);
  cta_sync();
  // the whole shared buffer becomes the accumulator of bins [acc_lo, acc_hi)
  float2* acc = sm;
  const int nacc = gd.acc_hi - gd.acc_lo;
  for (int h = threadIdx.x; h < nacc; h += blockDim.x) acc[h] = make_float2(0.f, 0.f);
  cta_sync();
  for (int col = 0; col < gd.ncolor; ++col) {
    if (LOGM && bd.color == col) synthesis_accumulate<LG, false>(a, bd, tt, res, acc, gd.acc_lo);
    cta_sync();
    if (gd.any_mirror) {
      if (LOGM && bd.color == col && bd.mirror) synthesis_accumulate<LG, true>(a, bd, tt, res, acc, gd.acc_lo);
      cta_sync();
    }
  }
  float2* spec = a.spec + s * a.spec_stride;
  for (int h = gd.ex_lo + threadIdx.x; h < gd.ex_hi; h += blockDim.x) spec[h] = acc[h - gd.acc_lo];
  if (gd.left_bd >= 0) boundary_combine(a, s, gd.left_bd, 1, acc, gd.acc_lo, spec, s_flag);
  if (gd.right_bd >= 0) boundary_combine(a, s, gd.right_bd, 0, acc, gd.acc_lo, spec, s_flag);
}

__global__ void __launch_bounds__(kBandThreads) band_synthesis_kernel(BandArgs a) {
  extern __shared__ float2 sm[];
  __shared__ int s_flag;
  const int g = blockIdx.x;
  const int64_t s = a.slice_base + blockIdx.y;
  const int t = threadIdx.x;
  const int k = a.thread_band[g * kBandThreads + t];
  const GroupDesc gd = a.groups[g];
  BandDesc bd{};
  if (k >= 0) bd = a.bands[k];
  const int tt = t - bd.tofs;
  switch (k >= 0 ? bd.log2M : 0) {
    case 4: synthesis_pipeline<4>(a, gd, bd, tt, s, sm, &s_flag); break;
    case 5: synthesis_pipeline<5>(a, gd, bd, tt, s, sm, &s_flag); break;
    case 6: synthesis_pipeline<6>(a, gd, bd, tt, s, sm, &s_flag); break;
    case 7: synthesis_pipeline<7>(a, gd, bd, tt, s, sm, &s_flag); break;
    case 8: synthesis_pipeline<8>(a, gd, bd, tt, s, sm, &s_flag); break;
    case 9: synthesis_pipeline<9>(a, gd, bd, tt, s, sm, &s_flag); break;
    case 10: synthesis_pipeline<10>(a, gd, bd, tt, s, sm, &s_flag); break;
    default: synthesis_pipeline<0>(a, gd, bd, tt, s, sm, &s_flag); break;
  }
}

BandArgs make_args(const slicq_plan* pl, const Workspace& ws, const float* win) {
  BandArgs a{};
  a.bands = pl->d_bands;
  a.groups = pl->d_groups;
  a.bounds = pl->d_bounds;
  a.thread_band = pl->d_thread_band;
  a.win = win;
  a.tw = TwiddleTables{pl->d_tw_lo, pl->d_tw_hi, pl->tw_lb};
  a.spec = ws.spec;
  a.spec_stride = ws.spec_stride;
  a.cps = pl->coefs_per_slice;
  a.patch = ws.band_patch;
  a.cnt = ws.band_cnt;
  a.G = pl->G;
  a.max_ovl = pl->max_ovl;
  a.N = (int)pl->N;
  a.log2N2 = ilog2c((int)(2 * pl->N));
  return a;
}

}  // namespace

cudaError_t launch_band_analysis(const slicq_plan* pl, const Workspace& ws, int64_t batch,
                                 float2* coef, cudaStream_t st) {
  BandArgs a = make_args(pl, ws, pl->d_ga);
  a.coef = coef;
  cudaError_t e = cudaFuncSetAttribute(band_analysis_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, pl->band_smem);
  if (e != cudaSuccess) return e;
  const int64_t total = batch * ws.S;
  for (int64_t s0 = 0; s0 < total; s0 += kMaxGridY) {
    a.slice_base = s0;
    dim3 grid(pl->G, (unsigned)(total - s0 < kMaxGridY ? total - s0 : kMaxGridY));
    band_analysis_kernel<<<grid, kBandThreads, pl->band_smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_band_synthesis(const slicq_plan* pl, const float2* coef, int64_t batch,
                                  SynthKind kind, const Workspace& ws, cudaStream_t st) {
  BandArgs a = make_args(pl, ws, kind == kSynthInverse ? pl->d_gs : pl->d_gadj);
  a.coef = const_cast<float2*>(coef);
  cudaError_t e = cudaFuncSetAttribute(band_synthesis_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, pl->band_smem);
  if (e != cudaSuccess) return e;
  const int64_t total = batch * ws.S;
  for (int64_t s0 = 0; s0 < total; s0 += kMaxGridY) {
    a.slice_base = s0;
    dim3 grid(pl->G, (unsigned)(total - s0 < kMaxGridY ? total - s0 : kMaxGridY));
    band_synthesis_kernel<<<grid, kBandThreads, pl->band_smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace slicq
