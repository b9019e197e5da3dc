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
// DFT_{M_k}(c_k); each channel's weighted values Y[j mod M_k] w g~_k[j]
// (j in J_k) belong to half-spectrum bin j for j <= N and, conjugated, to bin
// 2N - j for j >= N or j = 0 (the mirrored channel's term for a real signal).
// At plan time the channels of a group are coloured so that channels of one
// colour touch disjoint bins; each colour is an accumulator layer in shared
// memory that its channels fill with plain stores, and every bin is the sum
// of its layers in a fixed order.  Bins shared with the neighbouring group go
// to two patch rows that a second kernel adds (a + b): the result is
// deterministic without atomics.
//
// This header holds the kernels as templates over the arithmetic of the
// band transforms (kPrecFP32, or the split-precision tensor-core stages of
// tc_dft.cuh); each specialisation is instantiated in exactly one
// translation unit (band.cu, band_split16.cu, band_splitbf16.cu).
#pragma once

#include <algorithm>

#include "fft_common.cuh"
#include "internal.h"
#include "tc_dft.cuh"

namespace slicq {

// Pass-2 twiddles of every band length M = 2^LOGM (LOGM = 4..10): entry
// (M - 16) + r R1 + j holds exp(-2 pi i j r / M), r < R2, j < R1, so that the
// threads of a team (consecutive j) read consecutive words.

struct BandArgs {
  const BandDesc* __restrict__ bands;
  const GroupDesc* __restrict__ groups;
  const int16_t* __restrict__ thread_band;
  const int32_t* __restrict__ slot_base;    // [N+1] patch slot of bin h for group g: slot_base[h] + g
  const int4* __restrict__ shared;          // bins of several groups: (h, first slot, count, 0)
  const float* __restrict__ win;     // window table of this launch
  const float2* __restrict__ twband; // pass-2 twiddle tables of lengths 16..1024 (2032 entries)
  const float2* __restrict__ tw4096; // exp(-2 pi i t / 4096), t < 4096 (three-pass lengths)
  float2* spec;                      // [slice][spec_stride]
  int64_t slice_base;                // first slice of this launch (per-slice kernels)
  int64_t total;                     // slices of the call (persistent kernel)
  int64_t spec_stride;
  float2* coef;                      // [slice][cps]
  int64_t cps;
  float2* patch;                     // [slice][ovl_total] partial sums of shared bins
  int ovl_total;
  int N;
  long long* cycles;                 // optional: SM clocks of each CTA (plan calibration)
  // transposition and masking (synthesis only; see slicq_inverse_modified)
  int modify;                        // 0: plain synthesis
  int shift;                         // channel k = 1..K reads channel k - shift
  int K;
  int S_clip;                        // slices per clip (slice index m = row mod S_clip)
  const int32_t* __restrict__ jc;    // centre bin of each channel, round(xi_k 2N / xi_s)
  const float* __restrict__ mask;    // [row][cps] gains, or null
  int* err;                          // set to 1 if a tensor-core wait gave up (split precision)
};

// The two persistent band kernels of one precision.
using BandKernel = void (*)(BandArgs, const int2*, const int*);
struct BandKernels {
  BandKernel analysis;
  BandKernel synthesis;
};
BandKernels band_kernels_split_fp16();
BandKernels band_kernels_split_bf16();

namespace {

// --------------------------------------------------------------- cp.async ---
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
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

// A channel whose support J_k lies strictly between DC and Nyquist: no wrap
// around the circle, no mirrored bins, every bin its own half-spectrum bin.
__device__ __forceinline__ bool simple_channel(const BandDesc& bd, int N) {
  return bd.j0 > 0 && bd.j0 + bd.len - 1 < N;
}

template <int LOGM, int PREC>
__device__ void analysis_persistent(const BandArgs& a, const GroupDesc& gd, int lane, int lanes,
                                    int64_t total, float2* sm) {
  constexpr bool THREE = LOGM > kMaxTwoPassLog2;
  // split precision: the radix-R stages (R > 4) of two-pass lengths on the tensor cores
  constexpr bool TC = PREC != kPrecFP32 && !THREE && LOGM >= 5;
  using T = Team<THREE ? 10 : LOGM>;
  constexpr int M = 1 << LOGM;
  constexpr int TT = THREE ? Team3<THREE ? LOGM : 11>::TT : T::TT;
  constexpr int BUFL = THREE ? Team3<THREE ? LOGM : 11>::BUF : T::BUF;
  const int t = threadIdx.x;
  const int nb = gd.band_end - gd.band_begin;
  const int bl = t / TT;
  const bool active = bl < nb;
  const BandDesc bd = a.bands[gd.band_begin + (active ? bl : 0)];
  const int twoN = 2 * a.N;
  float2* s_tw = sm;
  float2* s_x0 = sm + M;
  float2* s_x1 = s_x0 + gd.fp_len;
  const int buf_off = M + 2 * gd.fp_len + bl * BUFL;
  const float* __restrict__ g = a.win + bd.win_off;
  const bool simple = simple_channel(bd, a.N);
  if (!THREE)
    for (int i = t; i < M; i += blockDim.x) s_tw[i] = __ldg(a.twband + (M - 16) + i);
  // tensor-core region after the team buffers, 128-byte aligned
  TcCtx tc{};
  if constexpr (TC)
    tc = tc_setup<LOGM, +1, PREC>(reinterpret_cast<unsigned char*>(sm) +
                                  ((((size_t)M + 2 * gd.fp_len + (size_t)nb * BUFL) * sizeof(float2) + 127) & ~(size_t)127));
  // window values of the pass-1 inputs, 0 outside the support: the same in
  // every slice (registers; two-pass lengths)
  float w[THREE ? 1 : T::J1][THREE ? 1 : T::R1];
  if constexpr (!THREE) {
    const int tt = t - bl * TT;
#pragma unroll
    for (int i = 0; i < T::J1; ++i)
#pragma unroll
      for (int r = 0; r < T::R1; ++r) {
        const int o = (tt + T::TT * i + r * T::R2 - bd.j0) & (M - 1);
        w[i][r] = o < bd.len ? __ldg(g + o) : 0.f;
      }
  }
  // The loop takes these integers through an empty asm each slice so that
  // the compiler recomputes the addresses instead of keeping all of them
  // live across the loop.
  struct Opaque {
    int tt, j0, len, buf;
  };
  const Opaque op0{t - bl * TT, bd.j0, bd.len, buf_off};
  auto opaque = [&]() {
    Opaque o = op0;
    asm volatile("" : "+r"(o.tt), "+r"(o.j0), "+r"(o.len), "+r"(o.buf));
    return o;
  };
  auto stage = [&](int64_t s, float2* dst) {
    const float2* src = a.spec + s * a.spec_stride + gd.fp_lo;
    for (int i = 2 * t; i < gd.fp_len; i += 2 * (int)blockDim.x) cp_async16(dst + i, src + i);
  };
  int64_t s = lane;
  pdl_wait();  // the slice spectra of the previous kernel
  if (s < total) stage(s, s_x0);
  cp_async_commit();
  for (int it = 0; s < total; s += lanes, ++it) {
    const float2* X = ((it & 1) ? s_x1 : s_x0) - gd.fp_lo;  // X[b] for b in the footprint
    if (s + lanes < total) stage(s + lanes, (it & 1) ? s_x0 : s_x1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();  // this slice's block (and, first time, the twiddles) are in
    const Opaque q = opaque();
    float2* buf = sm + q.buf;
    float2* out = a.coef + s * a.cps + bd.coef_off;
    // general input element idx: the bin of the residue (circular, mirrored
    // bins conjugated), weight 0 outside the support
    auto load_general = [&](int idx, float wv) -> float2 {
      const int o = (idx - q.j0) & (M - 1);
      const int oc = o < q.len ? o : 0;
      int b = q.j0 + oc;
      if (b >= twoN) b -= twoN;
      const bool mir = b > a.N;
      float2 x = X[mir ? twoN - b : b];
      if (mir) x.y = -x.y;
      return c_scale(x, wv);
    };
    if constexpr (THREE) {
      band_three_pass<LOGM, +1>(active, q.tt, buf, a.tw4096,
                                [&](int idx) {
                                  const int o = (idx - q.j0) & (M - 1);
                                  return load_general(idx, o < q.len ? __ldg(g + o) : 0.f);
                                },
                                [&](int i, float2 v) { __stcs(out + i, v); });
      __syncthreads();
      continue;
    } else {
      float2 v[T::J1][T::R1];
      if (active) {
        if (simple) {
#pragma unroll
          for (int i = 0; i < T::J1; ++i)
#pragma unroll
            for (int r = 0; r < T::R1; ++r) {
              const int o = (q.tt + T::TT * i + r * T::R2 - q.j0) & (M - 1);
              v[i][r] = c_scale(X[q.j0 + (o < q.len ? o : 0)], w[i][r]);
            }
        } else {
#pragma unroll
          for (int i = 0; i < T::J1; ++i)
#pragma unroll
            for (int r = 0; r < T::R1; ++r) v[i][r] = load_general(q.tt + T::TT * i + r * T::R2, w[i][r]);
        }
        if constexpr (!TC) team_pass1_regs<LOGM, +1>(q.tt, buf, v);
      }
      if constexpr (TC) {
        // both radix stages over the whole CTA (threads without a channel
        // pass zeros); the stores between them are those of the register path
        if (!active) {
#pragma unroll
          for (int i = 0; i < T::J1; ++i)
#pragma unroll
            for (int r = 0; r < T::R1; ++r) v[i][r] = make_float2(0.f, 0.f);
        }
        if (!tc_dft<T::R1, T::J1, +1, PREC>(v, tc, tc.b1)) break;
        if (active) {
#pragma unroll
          for (int i = 0; i < T::J1; ++i)
#pragma unroll
            for (int r = 0; r < T::R1; ++r) buf[T::pad1(q.tt + T::TT * i, r)] = v[i][r];
        }
        __syncwarp();  // a team lies inside one warp
        float2 u[T::J2][T::R2];
#pragma unroll
        for (int i = 0; i < T::J2; ++i) {
          const int j = q.tt + T::TT * i;
#pragma unroll
          for (int r = 0; r < T::R2; ++r) {
            float2 x = make_float2(0.f, 0.f);
            if (active) {
              x = buf[T::pad2(j, r)];
              if (r > 0) x = c_mul(x, c_conj(s_tw[r * T::R1 + j]));
            }
            u[i][r] = x;
          }
        }
        if (!tc_dft<T::R2, T::J2, +1, PREC>(u, tc, tc.b2)) break;
        if (active) {
#pragma unroll
          for (int i = 0; i < T::J2; ++i)
#pragma unroll
            for (int r = 0; r < T::R2; ++r) __stcs(out + team_out_index<LOGM>(q.tt, i, r), u[i][r]);
        }
      } else {
        __syncwarp();  // a team lies inside one warp
        if (active) {
          float2 res[T::HELD];
          team_pass2<LOGM, +1>(q.tt, buf, [&](int j, int r) { return c_conj(s_tw[r * T::R1 + j]); }, res);
#pragma unroll
          for (int i = 0; i < T::J2; ++i)
#pragma unroll
            for (int r = 0; r < T::R2; ++r) __stcs(out + team_out_index<LOGM>(q.tt, i, r), res[i * T::R2 + r]);
        }
      }
      __syncthreads();  // the footprint buffer is refilled two slices later
    }
  }
  cp_async_wait<0>();
  if constexpr (TC) tc_teardown(tc, a.err);
}

template <int PREC>
__global__ void __launch_bounds__(kBandThreads, 1) band_analysis_persistent_kernel(
    BandArgs a, const int2* __restrict__ cta_map, const int* __restrict__ lanes_of) {
  extern __shared__ __align__(128) float2 sm[];
  pdl_launch_dependents();
  const int2 gl = cta_map[blockIdx.x];  // (group, lane)
  const GroupDesc gd = a.groups[gl.x];
  const int lanes = lanes_of[gl.x];
  const int64_t total = a.total;
  const long long t0 = clock64();
  switch (gd.log2M) {
    case 4: analysis_persistent<4, PREC>(a, gd, gl.y, lanes, total, sm); break;
    case 5: analysis_persistent<5, PREC>(a, gd, gl.y, lanes, total, sm); break;
    case 6: analysis_persistent<6, PREC>(a, gd, gl.y, lanes, total, sm); break;
    case 7: analysis_persistent<7, PREC>(a, gd, gl.y, lanes, total, sm); break;
    case 8: analysis_persistent<8, PREC>(a, gd, gl.y, lanes, total, sm); break;
    case 9: analysis_persistent<9, PREC>(a, gd, gl.y, lanes, total, sm); break;
    case 10: analysis_persistent<10, PREC>(a, gd, gl.y, lanes, total, sm); break;
    case 11: analysis_persistent<11, kPrecFP32>(a, gd, gl.y, lanes, total, sm); break;
    case 12: analysis_persistent<12, kPrecFP32>(a, gd, gl.y, lanes, total, sm); break;
  }
  if (a.cycles) {
    __syncthreads();
    if (threadIdx.x == 0) a.cycles[blockIdx.x] = clock64() - t0;
  }
}

// ----------------------------------------------------------- synthesis ---
// Persistent form: CTA c keeps group cta_group[c] and walks the slices
// s = lane, lane + lanes, ...  Shared memory: [pass-2 twiddles (two-pass
// lengths)][team buffers][accumulator layers].  Per slice: pass 1, pass 2
// (while the next slice's coefficients load into registers), weighted
// values to the layers, then every bin of the group to the spectrum or a
// patch row.

// Zeroes n complex values at p (p 16-byte aligned) with 16-byte stores.
__device__ __forceinline__ void zero_layers(float2* p, int n) {
  float4* q = reinterpret_cast<float4*>(p);
  const int n4 = n >> 1;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = threadIdx.x; i < n4; i += kBandThreads) q[i] = z;
  if ((n & 1) && threadIdx.x == 0) p[n - 1] = make_float2(0.f, 0.f);
}

// Where slice s's bins of group g go: the spectrum row, or, for a bin other
// groups also cover, the group's slot of that bin in the slice's patch row.
struct BinSink {
  float2* spec;
  float2* row;
  const int32_t* __restrict__ slot;
  int g, ex_lo, ex_hi;
  __device__ __forceinline__ BinSink(const BandArgs& a, const GroupDesc& gd, int gi, int64_t s) {
    spec = a.spec + s * a.spec_stride;
    row = a.patch + s * (int64_t)a.ovl_total;
    slot = a.slot_base;
    g = gi;
    ex_lo = gd.ex_lo;
    ex_hi = gd.ex_hi;
  }
  __device__ __forceinline__ void put(int h, float2 v) const {
    if (h >= ex_lo && h < ex_hi) spec[h] = v;
    else row[__ldg(slot + h) + g] = v;
  }
};

// Bins [acc_lo, acc_hi): the sum of the NL layers in layer order (NL = 0:
// nl layers).  The bins a layer's channels cover are the same in every
// slice and are overwritten by every slice's stores; the others stay zero
// from the initial zeroing, so the layers need no clearing between slices.
template <int NL>
__device__ __forceinline__ void write_bins(const GroupDesc& gd, const float2* lay, int nl, int acc_n,
                                           const BinSink& out) {
  for (int h = gd.acc_lo + (int)threadIdx.x; h < gd.acc_hi; h += kBandThreads) {
    const float2* p = lay + (h - gd.acc_lo);
    float2 v = p[0];
    if (NL > 0) {
#pragma unroll
      for (int l = 1; l < NL; ++l) v = c_add(v, p[l * acc_n]);
    } else {
      for (int l = 1; l < nl; ++l) v = c_add(v, p[l * acc_n]);
    }
    out.put(h, v);
  }
}

__device__ __forceinline__ void write_bins_n(const GroupDesc& gd, const float2* lay, int nl, int acc_n,
                                             const BinSink& out) {
  switch (nl) {
    case 1: write_bins<1>(gd, lay, nl, acc_n, out); break;
    case 2: write_bins<2>(gd, lay, nl, acc_n, out); break;
    case 3: write_bins<3>(gd, lay, nl, acc_n, out); break;
    case 4: write_bins<4>(gd, lay, nl, acc_n, out); break;
    default: write_bins<0>(gd, lay, nl, acc_n, out); break;
  }
}

// The channel's two layers, indexed by bin: direct colours come first, then
// the mirrored ones (a channel without direct or mirrored bins never writes
// the corresponding one).
struct ChannelLayers {
  float2* dl;
  float2* ml;
  __device__ __forceinline__ ChannelLayers(const BandDesc& bd, const GroupDesc& gd, float2* lay, int acc_n) {
    const int nd = gd.nphases & 0xFFFF;
    const int dli = bd.phases & 0xFFFF, mli = bd.phases >> 16;
    dl = lay + (dli == kNoPhase ? 0 : dli) * acc_n - gd.acc_lo;
    ml = lay + (mli == kNoPhase ? 0 : nd + mli) * acc_n - gd.acc_lo;
  }
  // value y of support bin b (0 <= b < 2N) to its direct and mirrored bins
  __device__ __forceinline__ void put(int b, float2 y, int N, int twoN) const {
    if (b <= N) dl[b] = y;
    if (b == 0 || b >= N) ml[b == 0 ? 0 : twoN - b] = c_conj(y);
  }
};

// Transposition: channel k = 1..K takes channel k - shift (none: src < 0)
// modulated by the centre-bin difference dj (the coefficients keep their
// absolute frequency); the plateaus k = 0, K+1 keep their own.
struct ModSource {
  int src;  // coefficient offset of the source channel in a slice, -1: zeros
  int dj;
};

__device__ __forceinline__ ModSource mod_source(const BandArgs& a, int k, int own_off) {
  if (!a.modify || a.shift == 0 || k == 0 || k == a.K + 1) return ModSource{own_off, 0};
  const int src = k - a.shift;
  if (src < 1 || src > a.K) return ModSource{-1, 0};
  return ModSource{a.bands[src].coef_off, a.jc[k] - a.jc[src]};
}

// coefficient idx of channel k (offset own_off) in slice row s, modified:
// times exp(2 pi i dj t / 2N) at t = (m-1)N + idx 2N/M, i.e.
// (-1)^(dj (m-1)) exp(2 pi i (dj idx mod M) / M), then times the mask
__device__ __forceinline__ float2 mod_value(const BandArgs& a, const ModSource& ms, int M, int own_off,
                                            int64_t s, int idx, float2 v) {
  if (ms.dj != 0) {
    const int64_t m = s % a.S_clip;
    const int e = (int)((((int64_t)ms.dj % M + M) % M * idx) & (M - 1));
    float sn, cs;
    sincospif(2.0f * (float)e / (float)M, &sn, &cs);
    if ((ms.dj & 1) && ((m - 1) & 1)) { cs = -cs; sn = -sn; }
    v = c_mul(v, make_float2(cs, sn));
  }
  if (a.mask) v = c_scale(v, __ldg(a.mask + s * a.cps + own_off + idx));
  return v;
}

template <int LOGM, int PREC>
__device__ void synthesis_two_pass(const BandArgs& a, const GroupDesc& gd, int gi, int k, int lane, int lanes,
                                   int64_t total, float2* sm) {
  // split precision: the radix-R stages (R > 4) on the tensor cores
  constexpr bool TC = PREC != kPrecFP32 && LOGM >= 5;
  using T = Team<LOGM>;
  constexpr int M = 1 << LOGM;
  const int t = threadIdx.x;
  const int nb = gd.band_end - gd.band_begin;
  const bool active = k >= 0;
  BandDesc bd{};
  if (active) bd = a.bands[k];
  const int twoN = 2 * a.N;
  const int acc_n = gd.acc_hi - gd.acc_lo;
  const int nl = (gd.nphases & 0xFFFF) + (gd.nphases >> 16);
  const int lay_off = (M + nb * T::BUF + 1) & ~1;
  float2* lay = sm + lay_off;
  const bool simple = simple_channel(bd, a.N);

  for (int i = t; i < M; i += kBandThreads) sm[i] = __ldg(a.twband + (M - 16) + i);
  zero_layers(lay, nl * acc_n);
  // tensor-core region after the accumulator layers, 128-byte aligned
  TcCtx tc{};
  if constexpr (TC)
    tc = tc_setup<LOGM, -1, PREC>(reinterpret_cast<unsigned char*>(sm) +
                                  ((((size_t)lay_off + (size_t)nl * acc_n) * sizeof(float2) + 127) & ~(size_t)127));
  // window values of the held outputs: the same in every slice (registers)
  float w[T::HELD];
  {
    const float* __restrict__ g = a.win + bd.win_off;
    const int tt = t - bd.tofs;
#pragma unroll
    for (int i = 0; i < T::J2; ++i)
#pragma unroll
      for (int r = 0; r < T::R2; ++r) {
        const int o = (team_out_index<LOGM>(tt, i, r) - bd.j0) & (M - 1);
        w[i * T::R2 + r] = active && o < bd.len ? __ldg(g + o) : 0.f;
      }
  }
  // The loop body derives every address from these integers again in each
  // slice: passed through an empty asm, they look new to the compiler, which
  // would otherwise compute all of them once before the loop and keep them
  // live in registers across it.
  struct Opaque {
    int tt, j0, len, buf, dl, ml;
  };
  const ChannelLayers cl0(bd, gd, lay, acc_n);
  const Opaque op0{t - bd.tofs, bd.j0, bd.len, M + bd.smem_off, (int)(cl0.dl - sm), (int)(cl0.ml - sm)};
  auto opaque = [&]() {
    Opaque o = op0;
    asm volatile("" : "+r"(o.tt), "+r"(o.j0), "+r"(o.len), "+r"(o.buf), "+r"(o.dl), "+r"(o.ml));
    return o;
  };
  // slice s's coefficients into the team buffer at their natural positions;
  // each thread copies exactly the elements it reads in pass 1
  const ModSource ms = mod_source(a, k, bd.coef_off);
  auto fetch = [&](const Opaque& q, int64_t s) {
    float2* buf = sm + q.buf;
    if (ms.src < 0) {  // transposed from outside 1..K: zeros
#pragma unroll
      for (int i = 0; i < T::J1; ++i)
#pragma unroll
        for (int r = 0; r < T::R1; ++r) buf[q.tt + T::TT * i + r * T::R2] = make_float2(0.f, 0.f);
      return;
    }
    const float2* c = a.coef + s * a.cps + ms.src;
#pragma unroll
    for (int i = 0; i < T::J1; ++i)
#pragma unroll
      for (int r = 0; r < T::R1; ++r) {
        const int idx = q.tt + T::TT * i + r * T::R2;
        cp_async8(buf + idx, c + idx);
      }
  };
  int64_t s = lane;
  pdl_wait();  // the coefficients (and the previous kernel's use of the workspace)
  if (active && s < total) fetch(opaque(), s);
  cp_async_commit();
  __syncthreads();  // twiddles staged, layers zeroed
  for (; s < total; s += lanes) {
    const Opaque q = opaque();
    float2* buf = sm + q.buf;
    float2 res[T::HELD];
    float2 v[T::J1][T::R1];
    cp_async_wait<0>();  // this thread's copies have landed
    if (active) {
#pragma unroll
      for (int i = 0; i < T::J1; ++i)
#pragma unroll
        for (int r = 0; r < T::R1; ++r) v[i][r] = buf[q.tt + T::TT * i + r * T::R2];
      if (a.modify) {
#pragma unroll
        for (int i = 0; i < T::J1; ++i)
#pragma unroll
          for (int r = 0; r < T::R1; ++r)
            v[i][r] = mod_value(a, ms, M, bd.coef_off, s, q.tt + T::TT * i + r * T::R2, v[i][r]);
      }
    }
    __syncwarp();  // the team has read its inputs: pass 1 overwrites them
    if constexpr (TC) {
      // both radix stages over the whole CTA (threads without a channel pass
      // zeros); the stores between them are those of the register path
      if (!active) {
#pragma unroll
        for (int i = 0; i < T::J1; ++i)
#pragma unroll
          for (int r = 0; r < T::R1; ++r) v[i][r] = make_float2(0.f, 0.f);
      }
      if (!tc_dft<T::R1, T::J1, -1, PREC>(v, tc, tc.b1)) break;
      if (active) {
#pragma unroll
        for (int i = 0; i < T::J1; ++i)
#pragma unroll
          for (int r = 0; r < T::R1; ++r) buf[T::pad1(q.tt + T::TT * i, r)] = v[i][r];
      }
      __syncwarp();
      float2 u[T::J2][T::R2];
#pragma unroll
      for (int i = 0; i < T::J2; ++i) {
        const int j = q.tt + T::TT * i;
#pragma unroll
        for (int r = 0; r < T::R2; ++r) {
          float2 x = make_float2(0.f, 0.f);
          if (active) {
            x = buf[T::pad2(j, r)];
            if (r > 0) x = c_mul(x, sm[r * T::R1 + j]);
          }
          u[i][r] = x;
        }
      }
      if (!tc_dft<T::R2, T::J2, -1, PREC>(u, tc, tc.b2)) break;
#pragma unroll
      for (int i = 0; i < T::J2; ++i)
#pragma unroll
        for (int r = 0; r < T::R2; ++r) res[i * T::R2 + r] = u[i][r];
    } else {
      if (active) team_pass1_regs<LOGM, -1>(q.tt, buf, v);
      __syncwarp();
      if (active) team_pass2<LOGM, -1>(q.tt, buf, [&](int j, int r) { return sm[r * T::R1 + j]; }, res);
    }
    __syncwarp();  // the team has read its buffer: refill it with the next slice
    if (active && s + lanes < total) fetch(q, s + lanes);
    cp_async_commit();
    __syncthreads();  // the previous slice's write-out has read the layers
    if (active) {
      float2* dl = sm + q.dl;
      float2* ml = sm + q.ml;
      if (simple) {
#pragma unroll
        for (int i = 0; i < T::J2; ++i)
#pragma unroll
          for (int r = 0; r < T::R2; ++r) {
            const int o = (team_out_index<LOGM>(q.tt, i, r) - q.j0) & (M - 1);
            if (o < q.len) dl[q.j0 + o] = c_scale(res[i * T::R2 + r], w[i * T::R2 + r]);
          }
      } else {
#pragma unroll
        for (int i = 0; i < T::J2; ++i)
#pragma unroll
          for (int r = 0; r < T::R2; ++r) {
            const int o = (team_out_index<LOGM>(q.tt, i, r) - q.j0) & (M - 1);
            int b = q.j0 + o;
            if (b >= twoN) b -= twoN;
            if (o < q.len) {
              const float2 y = c_scale(res[i * T::R2 + r], w[i * T::R2 + r]);
              if (b <= a.N) dl[b] = y;
              if (b == 0 || b >= a.N) ml[b == 0 ? 0 : twoN - b] = c_conj(y);
            }
          }
      }
    }
    __syncthreads();
    write_bins_n(gd, lay, nl, acc_n, BinSink(a, gd, gi, s));
  }
  cp_async_wait<0>();
  if constexpr (TC) tc_teardown(tc, a.err);
}

// Three-pass lengths (2048, 4096): the team spans warps and its last pass
// writes Y w g~ at the support offsets of its buffer; windows and twiddles
// come from global memory (L1-resident).
template <int LOGM>
__device__ void synthesis_three_pass(const BandArgs& a, const GroupDesc& gd, int gi, int k, int lane, int lanes,
                                     int64_t total, float2* sm) {
  constexpr int M = 1 << LOGM;
  const int t = threadIdx.x;
  const int nb = gd.band_end - gd.band_begin;
  const bool active = k >= 0;
  BandDesc bd{};
  if (active) bd = a.bands[k];
  const int tt = t - bd.tofs;
  const int twoN = 2 * a.N;
  const int acc_n = gd.acc_hi - gd.acc_lo;
  const int nl = (gd.nphases & 0xFFFF) + (gd.nphases >> 16);
  float2* buf = sm + bd.smem_off;
  float2* lay = sm + ((nb * (M + 1) + 1) & ~1);
  const ChannelLayers cl(bd, gd, lay, acc_n);
  const float* __restrict__ gw = a.win + bd.win_off;
  zero_layers(lay, nl * acc_n);  // the transform's first barrier orders this
  pdl_wait();
  const ModSource ms = mod_source(a, k, bd.coef_off);
  for (int64_t s = lane; s < total; s += lanes) {
    const float2* c = a.coef + s * a.cps + ms.src;
    auto in = [&](int idx) {
      if (!a.modify) return __ldcs(c + idx);
      const float2 v = ms.src < 0 ? make_float2(0.f, 0.f) : __ldcs(c + idx);
      return mod_value(a, ms, M, bd.coef_off, s, idx, v);
    };
    auto contrib = [&](int idx, float2 v) {
      const int o = (idx - bd.j0) & (M - 1);
      if (o < bd.len) buf[o] = c_scale(v, __ldg(gw + o));
    };
    band_three_pass<LOGM, -1>(active, tt, buf, a.tw4096, in, contrib);
    __syncthreads();  // weighted values in the buffers; previous write-out done
    if (active) {
      for (int o = tt; o < bd.len; o += M / kPerThread) {
        int b = bd.j0 + o;
        if (b >= twoN) b -= twoN;
        cl.put(b, buf[o], a.N, twoN);
      }
    }
    __syncthreads();
    write_bins_n(gd, lay, nl, acc_n, BinSink(a, gd, gi, s));
  }
}

template <int PREC>
__global__ void __launch_bounds__(kBandThreads, 1) band_synthesis_persistent_kernel(
    BandArgs a, const int2* __restrict__ cta_map, const int* __restrict__ lanes_of) {
  extern __shared__ __align__(128) float2 sm[];
  pdl_launch_dependents();
  const int2 gl = cta_map[blockIdx.x];  // (group, lane)
  const GroupDesc gd = a.groups[gl.x];
  const int lanes = lanes_of[gl.x];
  const int k = a.thread_band[gl.x * kBandThreads + threadIdx.x];
  const int64_t total = a.total;
  const long long t0 = clock64();
  switch (gd.log2M) {
    case 4: synthesis_two_pass<4, PREC>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
    case 5: synthesis_two_pass<5, PREC>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
    case 6: synthesis_two_pass<6, PREC>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
    case 7: synthesis_two_pass<7, PREC>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
    case 8: synthesis_two_pass<8, PREC>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
    case 9: synthesis_two_pass<9, PREC>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
    case 10: synthesis_two_pass<10, PREC>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
    case 11: synthesis_three_pass<11>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
    case 12: synthesis_three_pass<12>(a, gd, gl.x, k, gl.y, lanes, total, sm); break;
  }
  if (a.cycles) {
    __syncthreads();
    if (threadIdx.x == 0) a.cycles[blockIdx.x] = clock64() - t0;
  }
}

}  // namespace
}  // namespace slicq
