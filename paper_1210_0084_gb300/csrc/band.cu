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
// DFT_{M_k}(c_k); each channel writes its weighted values Y[j mod M_k] w g~_k[j]
// (j in J_k) to shared memory; then every half-spectrum bin h = 0..N of the
// group sums, in a fixed order, the channels whose support covers h directly
// and the conjugates of those covering -h.  Bins shared with the neighbouring
// group are combined by whichever of the two CTAs arrives second
// (a + b == b + a), so the result is deterministic and needs no zero-fill.
#include "fft_common.cuh"
#include "internal.h"

namespace slicq {
namespace {

// Pass-2 twiddles of every band length M = 2^LOGM (LOGM = 4..10): entry
// (M - 16) + r R1 + j holds exp(-2 pi i j r / M), r < R2, j < R1, so that the
// threads of a team (consecutive j) read consecutive words.
constexpr int kTwSmall = 2032;

struct BandArgs {
  const BandDesc* __restrict__ bands;
  const GroupDesc* __restrict__ groups;
  const BoundaryDesc* __restrict__ bounds;
  const int16_t* __restrict__ thread_band;
  const int32_t* __restrict__ mirror_list;  // channels with mirrored bins, per group
  const float* __restrict__ win;     // window table of this launch
  const float2* __restrict__ twband; // pass-2 twiddle tables, kTwSmall entries
  const float2* __restrict__ tw4096; // exp(-2 pi i t / 4096), t < 4096 (three-pass lengths)
  float2* spec;                      // [slice][spec_stride]
  int64_t slice_base;                // first slice of this launch (per-slice kernels)
  int64_t total;                     // slices of the call (persistent kernel)
  int64_t spec_stride;
  float2* coef;                      // [slice][cps]
  int64_t cps;
  float2* patch;                     // [slice][G-1][2][max_ovl]
  uint32_t* cnt;                     // [slice][G-1]
  int G, max_ovl;
  int N;
};

__device__ __forceinline__ void load_twiddles(const BandArgs& a, float2* s_tw) {
  for (int i = threadIdx.x; i < kTwSmall; i += blockDim.x) s_tw[i] = __ldg(a.twband + i);
}

// exp(SIGN 2 pi i j r / 2^LOGM) from the shared pass-2 tables
template <int LOGM, int SIGN>
struct BandTw {
  const float2* s_tw;
  __device__ __forceinline__ float2 operator()(int j, int r) const {
    const float2 w = s_tw[((1 << LOGM) - 16) + r * Team<LOGM>::R1 + j];
    return SIGN < 0 ? w : c_conj(w);
  }
};

// --------------------------------------------------------------- cp.async ---
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// ------------------------------------------------------------ analysis ---
// Persistent form: CTA c keeps group cta_group[c] and walks the slices
// s = lane, lane + lanes, ... (lanes per group proportional to the group's
// work).  Each slice's footprint of the spectrum [fp_lo, fp_lo + fp_len) is
// one contiguous block; cp.async copies the next slice's block while the
// current one is transformed.  Shared memory: [twiddles M][footprint x 2]
// [team buffers].

// exp(SIGN 2 pi i e / n) for n | 4096, from the global W_4096 table (L1-resident)
template <int SIGN>
struct Tw4096 {
  const float2* __restrict__ t;
  __device__ __forceinline__ float2 operator()(int e, int n) const {
    const float2 w = __ldg(t + e * (4096 / n));
    return SIGN < 0 ? w : c_conj(w);
  }
};

// Three-pass transform of one band of length 2^LOGM (2048, 4096) by its team
// (several warps).  Every thread of the CTA calls this (the group holds
// channels of one length); threads without a channel only join the barriers.
// IN(idx) gives input element idx; OUT(idx, v) takes the result element idx
// (its writes may overwrite `buf`: a barrier separates them from the reads).
template <int LOGM, int SIGN, class In, class Out>
__device__ __forceinline__ void band_three_pass(bool active, int tt, float2* buf, const float2* tw4096,
                                                In in, Out out) {
  using T = Team3<LOGM>;
  constexpr int L = T::L;
  const Tw4096<SIGN> tw{tw4096};
  auto nosync = [] {};
  auto cta = [] { __syncthreads(); };
  if (active)
    stockham_pass<L, T::R0, 1, SIGN, T::TT>(tt, in, tw, nosync, [&](int i, float2 v) { buf[i] = v; });
  __syncthreads();
  if (active) {
    stockham_pass<L, T::R1, T::R0, SIGN, T::TT>(tt, [&](int i) { return buf[i]; }, tw, cta,
                                                [&](int i, float2 v) { buf[i] = v; });
  } else {
    __syncthreads();
  }
  __syncthreads();
  if (active) {
    stockham_pass<L, T::R2, T::R0 * T::R1, SIGN, T::TT>(tt, [&](int i) { return buf[i]; }, tw, cta, out);
  } else {
    __syncthreads();
  }
}

template <int LOGM>
__device__ void analysis_persistent(const BandArgs& a, const GroupDesc& gd, int lane, int lanes,
                                    int64_t total, float2* sm) {
  constexpr bool THREE = LOGM > kMaxTwoPassLog2;
  using T = Team<THREE ? 10 : LOGM>;
  constexpr int M = 1 << LOGM;
  constexpr int TT = THREE ? Team3<THREE ? LOGM : 11>::TT : T::TT;
  constexpr int BUFL = THREE ? Team3<THREE ? LOGM : 11>::BUF : T::BUF;
  const int t = threadIdx.x;
  const int nb = gd.band_end - gd.band_begin;
  const int bl = t / TT;
  const int tt = t - bl * TT;
  const bool active = bl < nb;
  const BandDesc bd = a.bands[gd.band_begin + (active ? bl : 0)];
  const int twoN = 2 * a.N;
  float2* s_tw = sm;
  float2* s_x0 = sm + M;
  float2* s_x1 = s_x0 + gd.fp_len;
  float2* buf = s_x1 + gd.fp_len + bl * BUFL;
  const float* __restrict__ g = a.win + bd.win_off;
  if (!THREE)
    for (int i = t; i < M; i += blockDim.x) s_tw[i] = __ldg(a.twband + (M - 16) + i);
  auto stage = [&](int64_t s, float2* dst) {
    const float2* src = a.spec + s * a.spec_stride + gd.fp_lo;
    for (int i = 2 * t; i < gd.fp_len; i += 2 * (int)blockDim.x) cp_async16(dst + i, src + i);
  };
  int64_t s = lane;
  if (s < total) stage(s, s_x0);
  cp_async_commit();
  for (int it = 0; s < total; s += lanes, ++it) {
    const float2* X = ((it & 1) ? s_x1 : s_x0) - gd.fp_lo;  // X[b] for b in the footprint
    if (s + lanes < total) stage(s + lanes, (it & 1) ? s_x0 : s_x1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();  // this slice's block (and, first time, the twiddles) are in
    // every load is issued; out-of-support residues get weight 0 (the
    // window table has padding after its last channel)
    auto load = [&](int idx) -> float2 {
      const int o = (idx - bd.j0) & (M - 1);
      const bool in = o < bd.len;
      const int oc = in ? o : 0;
      int b = bd.j0 + oc;
      if (b >= twoN) b -= twoN;
      const bool mir = b > a.N;
      float2 x = X[mir ? twoN - b : b];
      const float w = __ldg(g + oc);
      if (mir) x.y = -x.y;
      return c_scale(x, in ? w : 0.f);
    };
    if constexpr (THREE) {
      float2* out = a.coef + s * a.cps + bd.coef_off;
      band_three_pass<LOGM, +1>(active, tt, buf, a.tw4096, load,
                                [&](int i, float2 v) { __stcs(out + i, v); });
      __syncthreads();
      continue;
    }
    if (active) team_pass1<THREE ? 4 : LOGM, +1>(tt, buf, load);
    __syncwarp();  // a team lies inside one warp
    if (active) {
      float2 res[T::HELD];
      constexpr int LP = THREE ? 10 : LOGM;
      team_pass2<LP, +1>(tt, buf, [&](int j, int r) { return c_conj(s_tw[r * T::R1 + j]); }, res);
      float2* out = a.coef + s * a.cps + bd.coef_off;
#pragma unroll
      for (int i = 0; i < T::J2; ++i)
#pragma unroll
        for (int r = 0; r < T::R2; ++r) __stcs(out + team_out_index<LP>(tt, i, r), res[i * T::R2 + r]);
    }
    __syncthreads();  // the footprint buffer is refilled two slices later
  }
  cp_async_wait<0>();
}

__global__ void __launch_bounds__(kBandThreads, 1) band_analysis_persistent_kernel(
    BandArgs a, const int2* __restrict__ cta_map, const int* __restrict__ lanes_of) {
  extern __shared__ float2 sm[];
  const int2 gl = cta_map[blockIdx.x];  // (group, lane)
  const GroupDesc gd = a.groups[gl.x];
  const int lanes = lanes_of[gl.x];
  const int64_t total = a.total;
  switch (gd.log2M) {
    case 4: analysis_persistent<4>(a, gd, gl.y, lanes, total, sm); break;
    case 5: analysis_persistent<5>(a, gd, gl.y, lanes, total, sm); break;
    case 6: analysis_persistent<6>(a, gd, gl.y, lanes, total, sm); break;
    case 7: analysis_persistent<7>(a, gd, gl.y, lanes, total, sm); break;
    case 8: analysis_persistent<8>(a, gd, gl.y, lanes, total, sm); break;
    case 9: analysis_persistent<9>(a, gd, gl.y, lanes, total, sm); break;
    case 10: analysis_persistent<10>(a, gd, gl.y, lanes, total, sm); break;
    case 11: analysis_persistent<11>(a, gd, gl.y, lanes, total, sm); break;
    case 12: analysis_persistent<12>(a, gd, gl.y, lanes, total, sm); break;
  }
}

// ----------------------------------------------------------- synthesis ---

// Per-channel fields the gather needs, staged in shared memory.
struct GatherBand {
  int32_t dlo, dhi;   // direct bins [dlo, dhi] (dhi < 0: none)
  int32_t j0, base;   // support start on the circle, contribution offset in smem
};

template <int LOGM>
__device__ __forceinline__ void synthesis_pass1(int tt, const float2* __restrict__ c, float2* buf) {
  team_pass1<LOGM, -1>(tt, buf, [&](int idx) { return __ldcs(c + idx); });
}

template <int LOGM>
__device__ __forceinline__ void synthesis_pass2(int tt, const float2* s_tw, const float2* buf,
                                                float2* res) {
  team_pass2<LOGM, -1>(tt, buf, BandTw<LOGM, -1>{s_tw}, res);
}

// Weighted values Y[j mod M] w g~[j] stored at their support offsets o = j - j0.
template <int LOGM>
__device__ __forceinline__ void synthesis_weight(const BandArgs& a, const BandDesc& bd, int tt,
                                                 const float2* res, float2* contrib) {
  using T = Team<LOGM>;
  constexpr int M = 1 << LOGM;
  const float* __restrict__ g = a.win + bd.win_off;
#pragma unroll
  for (int i = 0; i < T::J2; ++i)
#pragma unroll
    for (int r = 0; r < T::R2; ++r) {
      const int idx = team_out_index<LOGM>(tt, i, r);
      const int o = (idx - bd.j0) & (M - 1);
      if (o < bd.len) contrib[o] = c_scale(res[i * T::R2 + r], __ldg(g + o));
    }
}

// Sum of all contributions to half-spectrum bin h, in a fixed order: direct
// channels from the highest covering one down, then the mirrored channels.
__device__ __forceinline__ float2 gather_bin(int h, int& last, int nb, const GatherBand* gb,
                                             const GroupDesc& gd, const BandDesc* __restrict__ bands,
                                             const int32_t* __restrict__ mirror_list,
                                             const float2* sm, int twoN) {
  while (last + 1 < nb && gb[last + 1].dlo <= h) ++last;
  float2 acc = make_float2(0.f, 0.f);
  for (int k = last; k >= 0; --k) {
    const GatherBand b = gb[k];
    if (b.dhi < 0) continue;          // channel without support
    if (b.dhi < h) break;             // dhi is non-decreasing over the group
    int o = h - b.j0;
    if (o < 0) o += twoN;
    acc = c_add(acc, sm[b.base + o]);
  }
  for (int i = 0; i < gd.nmirror; ++i) {
    const BandDesc bd = bands[mirror_list[gd.mirror_off + i]];
    if (h < bd.mlo || h > bd.mhi) continue;
    const int bm = h == 0 ? 0 : twoN - h;
    int o = bm - bd.j0;
    if (o < 0) o += twoN;
    if (o < bd.len) acc = c_add(acc, c_conj(sm[bd.smem_off + o]));
  }
  return acc;
}

__global__ void __launch_bounds__(kBandThreads) band_synthesis_kernel(BandArgs a) {
  extern __shared__ float2 sm[];
  __shared__ float2 s_tw[kTwSmall];
  __shared__ GatherBand s_gb[kBandThreads];
  __shared__ int s_flag;
  const int g = blockIdx.x;
  const int64_t s = a.slice_base + blockIdx.y;
  const int t = threadIdx.x;
  const int k = a.thread_band[g * kBandThreads + t];
  const GroupDesc gd = a.groups[g];
  const int nb = gd.band_end - gd.band_begin;
  BandDesc bd{};
  if (k >= 0) bd = a.bands[k];
  const int tt = t - bd.tofs;
  float2* buf = sm + bd.smem_off;
  const int twoN = 2 * a.N;

  load_twiddles(a, s_tw);
  if (t < nb) {
    const BandDesc b = a.bands[gd.band_begin + t];
    s_gb[t] = GatherBand{b.dlo, b.dhi, b.j0, b.smem_off};
  }
  __syncthreads();  // tables filled by all threads; the passes only sync per warp
  if (gd.log2M > kMaxTwoPassLog2) {
    // three-pass lengths: the team spans warps; its last pass writes Y w g~ at
    // the support offsets into the band's buffer
    const float2* c = a.coef + s * a.cps + bd.coef_off;
    auto in = [&](int idx) { return __ldcs(c + idx); };
    const float* __restrict__ g = a.win + bd.win_off;
    auto contrib = [&](int idx, float2 v) {  // weighted as in the two-pass path
      const int o = (idx - bd.j0) & ((1 << bd.log2M) - 1);
      if (o < bd.len) buf[o] = c_scale(v, __ldg(g + o));
    };
    if (gd.log2M == 11) band_three_pass<11, -1>(k >= 0, tt, buf, a.tw4096, in, contrib);
    else band_three_pass<12, -1>(k >= 0, tt, buf, a.tw4096, in, contrib);
  }
  if (k >= 0) {
    const float2* c = a.coef + s * a.cps + bd.coef_off;
    switch (bd.log2M) {
      case 4: synthesis_pass1<4>(tt, c, buf); break;
      case 5: synthesis_pass1<5>(tt, c, buf); break;
      case 6: synthesis_pass1<6>(tt, c, buf); break;
      case 7: synthesis_pass1<7>(tt, c, buf); break;
      case 8: synthesis_pass1<8>(tt, c, buf); break;
      case 9: synthesis_pass1<9>(tt, c, buf); break;
      case 10: synthesis_pass1<10>(tt, c, buf); break;
    }
  }
  __syncwarp();  // a team lies inside one warp
  float2 res[kPerThread];
  if (k >= 0) {
    switch (bd.log2M) {
      case 4: synthesis_pass2<4>(tt, s_tw, buf, res); break;
      case 5: synthesis_pass2<5>(tt, s_tw, buf, res); break;
      case 6: synthesis_pass2<6>(tt, s_tw, buf, res); break;
      case 7: synthesis_pass2<7>(tt, s_tw, buf, res); break;
      case 8: synthesis_pass2<8>(tt, s_tw, buf, res); break;
      case 9: synthesis_pass2<9>(tt, s_tw, buf, res); break;
      case 10: synthesis_pass2<10>(tt, s_tw, buf, res); break;
    }
  }
  __syncwarp();  // the team has read its pass buffer: reuse it for contributions
  if (k >= 0) {
    switch (bd.log2M) {
      case 4: synthesis_weight<4>(a, bd, tt, res, buf); break;
      case 5: synthesis_weight<5>(a, bd, tt, res, buf); break;
      case 6: synthesis_weight<6>(a, bd, tt, res, buf); break;
      case 7: synthesis_weight<7>(a, bd, tt, res, buf); break;
      case 8: synthesis_weight<8>(a, bd, tt, res, buf); break;
      case 9: synthesis_weight<9>(a, bd, tt, res, buf); break;
      case 10: synthesis_weight<10>(a, bd, tt, res, buf); break;
    }
  }
  __syncthreads();

  // gather bins [acc_lo, acc_hi); bins shared with a neighbour go to hand-off slots
  float2* spec = a.spec + s * a.spec_stride;
  int bl_hi = gd.acc_lo, br_lo = gd.acc_hi;
  float2* patch_l = nullptr;
  float2* patch_r = nullptr;
  if (gd.left_bd >= 0) {
    bl_hi = a.bounds[gd.left_bd].hi;
    patch_l = a.patch + ((s * (a.G - 1) + gd.left_bd) * 2 + 1) * a.max_ovl - gd.acc_lo;
  }
  if (gd.right_bd >= 0) {
    br_lo = a.bounds[gd.right_bd].lo;
    patch_r = a.patch + ((s * (a.G - 1) + gd.right_bd) * 2 + 0) * a.max_ovl - br_lo;
  }
  {
    int h = gd.acc_lo + t;
    int last = -1;
    if (h < gd.acc_hi) {  // last channel with dlo <= h (dlo is non-decreasing)
      int lo = 0, hi = nb - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_gb[mid].dlo <= h) lo = mid; else hi = mid - 1;
      }
      last = s_gb[lo].dlo <= h ? lo : -1;
    }
    for (; h < gd.acc_hi; h += blockDim.x) {
      const float2 v = gather_bin(h, last, nb, s_gb, gd, a.bands, a.mirror_list, sm, twoN);
      if (h < bl_hi) patch_l[h] = v;
      else if (h >= br_lo) patch_r[h] = v;
      else spec[h] = v;
    }
  }
  // hand-offs: the second CTA to arrive at a shared range stores the sums
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    const int bd_i = side == 0 ? gd.left_bd : gd.right_bd;
    if (bd_i < 0) continue;
    const BoundaryDesc b = a.bounds[bd_i];
    const int64_t slot = s * (a.G - 1) + bd_i;
    // barrier, then one thread fences and moves the counter (the pattern of
    // a grid-wide barrier): the CTA's slot writes are ordered before it
    __syncthreads();
    if (t == 0) {
      __threadfence();
      // 0 -> 1 for the first arriver, 1 -> 0 for the second (ready for the next call)
      const unsigned old = atomicInc(a.cnt + slot, 1u);
      __threadfence();
      s_flag = (old == 1u);
    }
    __syncthreads();
    if (s_flag) {
      const float2* p0 = a.patch + (slot * 2 + 0) * a.max_ovl;
      const float2* p1 = a.patch + (slot * 2 + 1) * a.max_ovl;
      for (int h = b.lo + t; h < b.hi; h += blockDim.x)
        spec[h] = c_add(__ldcg(p0 + (h - b.lo)), __ldcg(p1 + (h - b.lo)));
    }
  }
}

BandArgs make_args(const slicq_plan* pl, const Workspace& ws, const float* win) {
  BandArgs a{};
  a.bands = pl->d_bands;
  a.groups = pl->d_groups;
  a.bounds = pl->d_bounds;
  a.thread_band = pl->d_thread_band;
  a.mirror_list = pl->d_mirror_list;
  a.win = win;
  a.twband = pl->d_twband;
  a.tw4096 = pl->d_tw4096;
  a.spec = ws.spec;
  a.spec_stride = ws.spec_stride;
  a.cps = pl->coefs_per_slice;
  a.patch = ws.band_patch;
  a.cnt = ws.band_cnt;
  a.G = pl->G;
  a.max_ovl = pl->max_ovl;
  a.N = (int)pl->N;
  return a;
}

}  // namespace

cudaError_t launch_band_analysis(const slicq_plan* pl, const Workspace& ws, int64_t batch,
                                 float2* coef, cudaStream_t st) {
  BandArgs a = make_args(pl, ws, pl->d_ga);
  a.coef = coef;
  a.total = batch * ws.S;
  cudaError_t e = cudaFuncSetAttribute(band_analysis_persistent_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, pl->band_smem_p);
  if (e != cudaSuccess) return e;
  band_analysis_persistent_kernel<<<pl->n_cta_a, kBandThreads, pl->band_smem_p, st>>>(
      a, pl->d_cta_map, pl->d_lanes);
  return cudaGetLastError();
}

cudaError_t launch_band_synthesis(const slicq_plan* pl, const float2* coef, int64_t batch,
                                  SynthKind kind, const Workspace& ws, cudaStream_t st) {
  BandArgs a = make_args(pl, ws, kind == kSynthInverse ? pl->d_gs : pl->d_gadj);
  a.coef = const_cast<float2*>(coef);
  cudaError_t e = cudaFuncSetAttribute(band_synthesis_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, pl->band_smem_a);
  if (e != cudaSuccess) return e;
  const int64_t total = batch * ws.S;
  for (int64_t s0 = 0; s0 < total; s0 += kMaxGridY) {
    a.slice_base = s0;
    dim3 grid(pl->G, (unsigned)(total - s0 < kMaxGridY ? total - s0 : kMaxGridY));
    band_synthesis_kernel<<<grid, kBandThreads, pl->band_smem_a, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace slicq
