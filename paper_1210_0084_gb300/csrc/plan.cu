// Plan construction: the integer layout on the host and the window, dual
// window and twiddle tables in FP64 on the device (stored as float32).
//
//   Table 1 (Sec. 3)       centre frequencies xi_k and bandwidths Omega_k,
//                          K the smallest integer with xi_K >= xi_max,
//                          decreased while xi_K >= xi_s / 2.
//   Sec. 3 sampling        g_k[j] = H((j xi_s / 2N - xi_k) / Omega_k) with a
//                          Hann H on ]-1/2, 1/2[ and flat plateaus for k = 0
//                          and K + 1; Omega_k widened to min_filter_len bins
//                          for k = 1..K (Sec. 5.2).
//   eq. framecond1         M_k >= |J_k| (next power of two, at least 16).
//   Prop. 2                d[j] = sum over all 2K+2 channels of M_k g_k[j]^2
//                          (channels K+2..2K+1 are the mirrors g_k[-j]) and
//                          g~_k = g_k / d, eq. painlessframe2.
//   Sec. 4.2               Tukey transition h_0 = cos^2(pi u / 2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "fft_common.cuh"
#include "internal.h"
#include "tc_dft.cuh"

namespace slicq {

namespace {

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2_64(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}

}  // namespace

slicq_status build_layout(const slicq_params* p, slicq_plan* pl) {
  if (!p || !pl) return SLICQ_EINVAL;
  if (!(p->fs > 0) || !(p->fmin > 0) || !(p->fmax > p->fmin) || p->bins_per_octave < 1 ||
      p->min_filter_len < 1 || !std::isfinite(p->fs) || !std::isfinite(p->fmax))
    return SLICQ_EINVAL;
  if (p->window != SLICQ_WIN_HANN && p->window != SLICQ_WIN_BLACKMAN_HARRIS) return SLICQ_EINVAL;
  if (p->mk_policy == SLICQ_MK_MULT4) return SLICQ_EUNSUPPORTED;  // band FFTs are radix-2
  if (p->mk_policy != SLICQ_MK_POW2 && p->mk_policy != SLICQ_MK_CONST) return SLICQ_EINVAL;
  if (p->precision != SLICQ_PREC_FP32 && p->precision != SLICQ_PREC_SPLIT_FP16 &&
      p->precision != SLICQ_PREC_SPLIT_BF16)
    return SLICQ_EINVAL;
  const int64_t L2 = p->slice_len;
  if (!is_pow2(L2)) return SLICQ_EINVAL;
  if (L2 < 2048 || L2 > 131072) return SLICQ_EUNSUPPORTED;
  const int64_t N = L2 / 2;
  const int64_t Mtr = p->trans_len;
  if (Mtr < 2 || (Mtr & 1) || Mtr >= N) return SLICQ_EINVAL;
  if (p->slice_cluster != 0 && (!is_pow2(p->slice_cluster) || p->slice_cluster > 8))
    return SLICQ_EINVAL;
  pl->params = *p;
  pl->N = N;

  // ---- Table 1
  const int B = p->bins_per_octave;
  const double Q = 1.0 / (std::pow(2.0, 1.0 / B) - std::pow(2.0, -1.0 / B));
  int64_t K = (int64_t)std::ceil(B * std::log2(p->fmax / p->fmin) - 1e-9) + 1;
  while (K >= 1 && p->fmin * std::pow(2.0, (double)(K - 1) / B) >= p->fs / 2) --K;
  if (K < 1) return SLICQ_EINVAL;
  if (K > 30000) return SLICQ_EUNSUPPORTED;
  pl->K = (int)K;
  const int nch = (int)K + 2;
  pl->n_channels = nch;
  pl->xi.assign(nch, 0.0);
  pl->omega.assign(nch, 0.0);
  const double floor_bw = p->min_filter_len * p->fs / (double)L2;
  for (int k = 1; k <= K; ++k) {
    pl->xi[k] = p->fmin * std::pow(2.0, (double)(k - 1) / B);
    pl->omega[k] = std::max(pl->xi[k] / Q, floor_bw);
  }
  pl->xi[0] = 0.0;
  pl->omega[0] = 2.0 * p->fmin;
  pl->xi[K + 1] = p->fs / 2.0;
  pl->omega[K + 1] = p->fs - 2.0 * pl->xi[K];

  // ---- supports J_k: integers j with |(j xi_s / 2N - xi_k) / Omega_k| < 1/2
  pl->bands.assign(nch, BandDesc{});
  pl->jlo.assign(nch, 0);
  int64_t coef_off = 0, win_off = 0;
  std::vector<int> foot_lo(nch), foot_hi(nch);
  std::vector<int32_t> cover(N + 2, 0);
  auto support = [&](int k, int64_t& first, int64_t& count) -> bool {
    const double centre = pl->xi[k] * (double)L2 / p->fs;
    const double half = pl->omega[k] * (double)L2 / (2.0 * p->fs);
    const int64_t lo = (int64_t)std::floor(centre - half) - 1;
    const int64_t hi = (int64_t)std::ceil(centre + half) + 1;
    first = 0;
    count = 0;
    for (int64_t j = lo; j <= hi; ++j) {
      const double t = ((double)j * p->fs / (double)L2 - pl->xi[k]) / pl->omega[k];
      if (std::fabs(t) < 0.5) {
        if (count == 0) first = j;
        if (j != first + count) return false;  // support must be an interval
        ++count;
      }
    }
    if (count == 0) first = (int64_t)std::llround(centre);  // degenerate plateau: a zero window of one bin
    return true;
  };
  // rectangular representation: every M_k is the largest pow2 length
  int64_t const_M = 0;
  if (p->mk_policy == SLICQ_MK_CONST) {
    int64_t widest = 0;
    for (int k = 0; k < nch; ++k) {
      int64_t first, count;
      if (!support(k, first, count)) return SLICQ_EINVAL;
      widest = std::max(widest, count);
    }
    const_M = 16;
    while (const_M < widest) const_M <<= 1;
  }
  for (int k = 0; k < nch; ++k) {
    int64_t first = 0, count = 0;
    if (!support(k, first, count)) return SLICQ_EINVAL;
    int64_t M = 16;
    while (M < count) M <<= 1;
    if (const_M) M = const_M;
    if (M > L2) return SLICQ_EINVAL;
    if (M > (int64_t(1) << kMaxBandLog2)) return SLICQ_EUNSUPPORTED;
    BandDesc& bd = pl->bands[k];
    bd.j0 = (int32_t)(((first % L2) + L2) % L2);
    bd.len = (int32_t)count;
    bd.log2M = ilog2_64(M);
    bd.coef_off = (int32_t)coef_off;
    bd.win_off = (int32_t)win_off;
    pl->jlo[k] = first;
    coef_off += M;
    win_off += count;
    // half-spectrum footprint: direct bins b <= N, mirrored bins 2N - b for b >= N or b = 0
    int dlo = (int)N + 1, dhi = -1, mlo = (int)N + 1, mhi = -1;
    for (int64_t o = 0; o < count; ++o) {
      const int64_t b = (bd.j0 + o) % L2;
      if (b <= N) {
        if (dhi >= 0 && b != dhi + 1) return SLICQ_EUNSUPPORTED;  // direct part must be an interval
        dlo = std::min<int>(dlo, (int)b);
        dhi = (int)b;
        cover[b] += 1;
      }
      if (b == 0 || b >= N) {
        const int64_t h = (L2 - b) % L2;
        mlo = std::min<int>(mlo, (int)h);
        mhi = std::max<int>(mhi, (int)h);
        cover[h] += 1;
      }
    }
    bd.dlo = dlo;
    bd.dhi = dhi;
    bd.mlo = mlo;
    bd.mhi = mhi;
    foot_lo[k] = std::min(dhi >= 0 ? dlo : (int)N + 1, mhi >= 0 ? mlo : (int)N + 1);
    foot_hi[k] = std::max(dhi, mhi);
    if (count == 0) foot_lo[k] = foot_hi[k] = -1;
  }
  for (int64_t h = 0; h <= N; ++h)
    if (cover[h] == 0) return SLICQ_EINVAL;  // eq. painlessframe1 fails: d[h] = 0
  if (coef_off > (int64_t)1 << 30) return SLICQ_EUNSUPPORTED;
  pl->coefs_per_slice = coef_off;
  pl->win_total = win_off;

  // ---- band groups: consecutive channels, <= kBandThreads threads each
  pl->groups.clear();
  pl->thread_band.clear();
  size_t smem_p = 0, syn_max = 0;  // bytes
  // split precision: a two-pass group of M >= 32 also holds its tensor-core
  // region (operands, DFT matrices, mbarrier), 128-byte aligned after the
  // rest of its shared memory
  const bool split = p->precision != SLICQ_PREC_FP32;
  auto tc_bytes = [&](int lm) { return split && lm >= 5 && lm <= kMaxTwoPassLog2 ? tc_region_bytes(lm) : 0; };
  auto with_tc = [&](size_t cplx, int lm) {
    const int tb = tc_bytes(lm);
    return tb ? ((cplx * sizeof(float2) + 127) & ~(size_t)127) + (size_t)tb : cplx * sizeof(float2);
  };
  pl->cost_a.clear();
  pl->cost_s.clear();
  {
    int k = 0;
    while (k < nch) {
      GroupDesc gd{};
      gd.band_begin = k;
      int threads = 0, smem = 0;
      // synthesis layers: greedy interval colouring of the direct ranges and
      // of the mirrored ranges; channels of one colour touch disjoint bins, so
      // each colour is one accumulator layer written with plain stores
      std::vector<int> dend, mend;  // last bin taken by each colour
      auto colour = [](std::vector<int>& ends, int lo, int hi) {
        for (size_t c = 0; c < ends.size(); ++c)
          if (ends[c] < lo) { ends[c] = hi; return (int)c; }
        ends.push_back(hi);
        return (int)ends.size() - 1;
      };
      int flo = (int)N + 1, fhi = -1;  // the group's footprint so far
      while (k < nch) {
        const int lm = pl->bands[k].log2M;
        const int M = 1 << lm;
        const int need_t = M >= kPerThread ? M / kPerThread : 1;
        const int need_s = lm > kMaxTwoPassLog2 ? M + 1                 // Team3<lm>::BUF
                                                : M + (M >> ((lm + 1) / 2)) + 1;  // Team<lm>::BUF
        if (threads + need_t > kBandThreads) break;
        // one band length per group: every warp of the CTA runs the same code
        if (k > gd.band_begin && lm != pl->bands[gd.band_begin].log2M) break;
        BandDesc& d = pl->bands[k];
        std::vector<int> de = dend, me = mend;
        const int dp = d.dhi >= 0 ? colour(de, d.dlo, d.dhi) : kNoPhase;
        const int mp = d.mhi >= 0 ? colour(me, d.mlo, d.mhi) : kNoPhase;
        const int nlo = foot_hi[k] >= 0 ? std::min(flo, foot_lo[k]) : flo;
        const int nhi = std::max(fhi, foot_hi[k]);
        const int acc_n = nhi >= nlo ? nhi - nlo + 1 : 0;
        const int lay = (int)(de.size() + me.size()) * acc_n;
        // synthesis shared memory: [pass-2 twiddles][team buffers][layers]
        const int need = ((lm > kMaxTwoPassLog2 ? 0 : M) + smem + need_s + 1 & ~1) + lay;
        if (k > gd.band_begin && with_tc((size_t)need, lm) > (size_t)kSynSmemBudget * sizeof(float2)) break;
        if (de.size() >= (size_t)kNoPhase || me.size() >= (size_t)kNoPhase) return SLICQ_EUNSUPPORTED;
        dend.swap(de);
        mend.swap(me);
        flo = nlo;
        fhi = nhi;
        d.phases = dp | (mp << 16);
        d.tofs = threads;
        d.smem_off = smem;
        threads += need_t;
        smem += need_s;
        ++k;
      }
      gd.band_end = k;
      gd.nphases = (int)dend.size() | ((int)mend.size() << 16);
      int alo = (int)N + 1, ahi = -1;
      int prev_dlo = 0, prev_dhi = -1;
      for (int b = gd.band_begin; b < gd.band_end; ++b) {
        BandDesc& d = pl->bands[b];
        if (foot_hi[b] >= 0) {
          alo = std::min(alo, foot_lo[b]);
          ahi = std::max(ahi, foot_hi[b]);
        }
        if (d.dhi < 0) {  // no direct bins: keep dlo monotone, mark empty
          d.dlo = prev_dlo;
        } else {
          if (d.dlo < prev_dlo || d.dhi < prev_dhi) return SLICQ_EUNSUPPORTED;
          prev_dlo = d.dlo;
          prev_dhi = d.dhi;
        }
      }
      if (ahi < 0) return SLICQ_EINVAL;
      gd.acc_lo = alo;
      gd.acc_hi = ahi + 1;
      gd.log2M = pl->bands[gd.band_begin].log2M;
      gd.fp_lo = alo & ~1;
      gd.fp_len = (gd.acc_hi - gd.fp_lo + 1) & ~1;
      {
        const int M = 1 << gd.log2M;
        const int nb = gd.band_end - gd.band_begin;
        const int bufl = gd.log2M > kMaxTwoPassLog2 ? M + 1
                                                    : M + (M >> ((gd.log2M + 1) / 2)) + 1;
        // synthesis: [pass-2 twiddles (two-pass lengths)][team buffers][layers]
        const int lay = ((gd.nphases & 0xFFFF) + (gd.nphases >> 16)) * (gd.acc_hi - gd.acc_lo);
        syn_max = std::max(syn_max, with_tc((size_t)((((gd.log2M > kMaxTwoPassLog2 ? 0 : M) + nb * bufl + 1) & ~1) + lay),
                                            gd.log2M));
        smem_p = std::max(smem_p, with_tc((size_t)(M + 2 * gd.fp_len + nb * bufl), gd.log2M));
        // estimated cycles per slice of one persistent CTA (a fixed part for
        // staging and barriers, the team transforms of the busiest warp
        // count times active warps, and the bin write-out); fitted to
        // per-CTA clock measurements of both kernels on GB300
        {
          const int thr = nb * (M >= kPerThread ? M / kPerThread : 1);
          const double fft = (double)((thr + 31) / 32) * std::min(M, kPerThread) * (gd.log2M + 4);
          const double rows = (double)((gd.acc_hi - gd.acc_lo + kBandThreads - 1) / kBandThreads);
          const double nl = (double)((gd.nphases & 0xFFFF) + (gd.nphases >> 16));
          const double fp_rows = (double)((gd.fp_len + kBandThreads - 1) / kBandThreads);
          pl->cost_a.push_back(2700.0 + 1.1 * fft + 6.5 * fp_rows * 16.0);
          pl->cost_s.push_back(5200.0 + 1.9 * fft + 3.5 * rows * 8.0 * (nl + 1.0));
        }
      }
      (void)smem;
      pl->groups.push_back(gd);
      std::vector<int16_t> tb(kBandThreads, (int16_t)-1);
      for (int b = gd.band_begin; b < gd.band_end; ++b) {
        const int M = 1 << pl->bands[b].log2M;
        const int nt = M >= kPerThread ? M / kPerThread : 1;
        for (int i = 0; i < nt; ++i) tb[pl->bands[b].tofs + i] = (int16_t)b;
      }
      pl->thread_band.insert(pl->thread_band.end(), tb.begin(), tb.end());
    }
  }
  const int G = (int)pl->groups.size();
  pl->G = G;
  // ---- bins covered by more than one group.  Groups are ordered and their
  // ranges [acc_lo, acc_hi) move monotonically, so the groups covering a bin
  // are a contiguous run first(h) .. first(h) + count(h) - 1.  A shared bin
  // gets one patch slot per covering group, in group order: group g writes
  // its partial sum of bin h to slot slot_base[h] + g of the slice's row.
  for (int g = 0; g + 1 < G; ++g) {
    const GroupDesc& a = pl->groups[g];
    const GroupDesc& b = pl->groups[g + 1];
    if (b.acc_lo < a.acc_lo || b.acc_hi < a.acc_hi) return SLICQ_EUNSUPPORTED;
  }
  if (pl->groups.front().acc_lo != 0 || pl->groups.back().acc_hi != N + 1) return SLICQ_EINVAL;
  {
    std::vector<int32_t> first(N + 1, -1), count(N + 1, 0);
    for (int g = 0; g < G; ++g)
      for (int h = pl->groups[g].acc_lo; h < pl->groups[g].acc_hi; ++h) {
        if (first[h] < 0) first[h] = g;
        ++count[h];
      }
    pl->slot_base.assign(N + 1, -1);
    pl->shared.clear();
    int32_t off = 0;
    for (int h = 0; h <= N; ++h) {
      if (count[h] == 0) return SLICQ_EINVAL;  // eq. painlessframe1: every bin is covered
      if (count[h] > 1) {
        pl->slot_base[h] = off - first[h];
        pl->shared.push_back(make_int4(h, off, count[h], 0));
        off += count[h];
      }
    }
    pl->ovl_total = off;
  }
  // bins of group g that no other group covers: [ex_lo, ex_hi)
  for (int g = 0; g < G; ++g) {
    GroupDesc& gd = pl->groups[g];
    gd.ex_lo = g > 0 ? std::max(gd.acc_lo, pl->groups[g - 1].acc_hi) : gd.acc_lo;
    gd.ex_hi = g + 1 < G ? std::min(gd.acc_hi, pl->groups[g + 1].acc_lo) : gd.acc_hi;
    if (gd.ex_hi < gd.ex_lo) gd.ex_hi = gd.ex_lo;
  }
  // per-slice band kernels: one team buffer per channel of the group
  if (syn_max > 220 * 1024 || smem_p > 220 * 1024) return SLICQ_EUNSUPPORTED;
  pl->band_smem_s = (int)syn_max;
  pl->band_smem_p = (int)smem_p;
  if (pl->band_smem_p > 220 * 1024) return SLICQ_EUNSUPPORTED;
  if (pl->band_smem_s > 220 * 1024) return SLICQ_EUNSUPPORTED;

  // ---- slice FFT geometry: N = P Q, cluster of C CTAs, <= 256 threads each
  const int logN = ilog2_64(N);
  pl->logP = logN / 2;
  pl->logQ = logN - pl->logP;
  int C = p->slice_cluster;
  if (C == 0) {
    C = 1;
    while (N / C > kSlicePer * kSliceMaxThreads) C <<= 1;
  }
  if (N / C > kSlicePer * kSliceMaxThreads || (1 << pl->logP) < C || N / (kSlicePer * C) < 1 || C > 8)
    return SLICQ_EUNSUPPORTED;
  pl->tw_lb = (ilog2_64(L2) + 1) / 2;
  set_slice_cluster(pl, C);
  return SLICQ_OK;
}

// Slice-kernel geometry for a cluster of C CTAs: the shared-memory layout
// [pass / exchange buffers][twiddle tables] of one CTA.
void set_slice_cluster(slicq_plan* pl, int C) {
  pl->C = C;
  const int P = 1 << pl->logP, Qn = 1 << pl->logQ;
  const int R2p = P / (1 << ((pl->logP + 1) / 2));
  const int R2q = Qn / (1 << ((pl->logQ + 1) / 2));
  const int cs1 = (Qn / C) * (P + R2p + 1);
  const int xs1 = (Qn / C) * (P + 1);
  const int cs3 = (P / C) * (Qn + R2q + 1);
  const int zs3 = (P / C) * (Qn + 1);
  pl->slice_tw_off = std::max(std::max(cs1, xs1), std::max(cs3, zs3));
  const int ntw = (1 << pl->tw_lb) + (int)((2 * pl->N) >> pl->tw_lb);
  // + the pass-2 tables of lengths P and Q and exp(-pi i v / Q), v < Q
  pl->slice_smem = (pl->slice_tw_off + ntw + P + 2 * Qn) * (int)sizeof(float2);
}

// ----------------------------------------------------- FP64 table kernels ---

namespace {

struct WinJob {
  int64_t jlo;     // unwrapped first support sample
  double xi, omega;
  int32_t len, win_off, plateau, M, j0, pair;  // pair: channel has a mirror
};

// H((j xi_s / 2N - xi_k) / Omega_k): Hann cos^2(pi t), or the 4-term
// Blackman-Harris window of F. J. Harris (Proc. IEEE 66(1), 1978),
// a0 - a1 cos 2 pi x + a2 cos 4 pi x - a3 cos 6 pi x on x in [0, 1], centred
// (x = t + 1/2: the odd terms change sign); plateaus are flat.
__device__ double window_value(const WinJob& w, int64_t j, double fs, double L2, int shape) {
  if (w.plateau) return 1.0;
  const double t = ((double)j * fs / L2 - w.xi) / w.omega;
  if (fabs(t) >= 0.5) return 0.0;
  if (shape == SLICQ_WIN_BLACKMAN_HARRIS)
    return 0.35875 + 0.48829 * cospi(2.0 * t) + 0.14128 * cospi(4.0 * t) + 0.01168 * cospi(6.0 * t);
  const double c = cospi(t);
  return c * c;
}

// g_k on its support, FP64
__global__ void k_windows(const WinJob* jobs, int nch, int64_t total, double fs, double L2, int shape,
                          double* g64) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  int lo = 0, hi = nch - 1;  // last job with win_off <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (jobs[mid].win_off <= i) lo = mid; else hi = mid - 1;
  }
  const WinJob w = jobs[lo];
  g64[i] = window_value(w, w.jlo + (i - w.win_off), fs, L2, shape);
}

// d[j] = sum_k M_k (g_k[j]^2 + [k has a mirror] g_k[-j]^2) over the circle
__global__ void k_diagonal(const WinJob* jobs, int nch, const double* g64, int64_t L2, double* d) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= L2) return;
  double acc = 0.0;
  for (int k = 0; k < nch; ++k) {
    const WinJob w = jobs[k];
    int64_t o = j - w.j0;
    if (o < 0) o += L2;
    if (o < w.len) {
      const double g = g64[w.win_off + o];
      acc += (double)w.M * g * g;
    }
    if (w.pair) {
      int64_t om = (L2 - j) % L2 - w.j0;
      if (om < 0) om += L2;
      if (om < w.len) {
        const double g = g64[w.win_off + om];
        acc += (double)w.M * g * g;
      }
    }
  }
  d[j] = acc;
}

// analysis, synthesis (dual) and adjoint tables, float32
__global__ void k_duals(const WinJob* jobs, int nch, int64_t total, const double* g64,
                        const double* d, int64_t L2, float* ga, float* gs, float* gadj,
                        int* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  int lo = 0, hi = nch - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (jobs[mid].win_off <= i) lo = mid; else hi = mid - 1;
  }
  const WinJob w = jobs[lo];
  const int64_t b = (w.j0 + (i - w.win_off)) % L2;
  const double g = g64[i];
  const double s = 1.0 / sqrt((double)L2);
  const double dj = d[b];
  if (!(dj > 0.0)) { *bad = 1; return; }
  const double weight = w.pair ? 1.0 : 0.5;  // self-mirror channels 0 and K+1
  ga[i] = (float)(g * s);
  gs[i] = (float)(weight * g / dj * s);
  gadj[i] = (float)(0.5 * g * s);
}

// exp(-2 pi i t / L2): fine table t < 2^lb, coarse table (t << lb); the
// pass-2 tables of the band lengths 16..1024 ([r][j] per length); and the
// four-step twiddles exp(-2 pi i q u / N) at [u Q + q]
__global__ void k_twiddles(int64_t L2, int lb, int logQ, float2* lo, float2* hi, float2* tband,
                           float2* t4, float2* t4096) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nlo = int64_t(1) << lb;
  const int64_t nhi = L2 >> lb;
  const int64_t N = L2 / 2;
  double s, c;
  if (i < nlo) {
    sincospi(-2.0 * (double)i / (double)L2, &s, &c);
    lo[i] = make_float2((float)c, (float)s);
  }
  if (i < nhi) {
    sincospi(-2.0 * (double)(i << lb) / (double)L2, &s, &c);
    hi[i] = make_float2((float)c, (float)s);
  }
  if (i < 2032) {
    int lm = 4;
    while (((int64_t(1) << (lm + 1)) - 16) <= i) ++lm;
    const int64_t M = int64_t(1) << lm;
    const int64_t R1 = int64_t(1) << ((lm + 1) / 2);
    const int64_t e = i - (M - 16);
    const int64_t r = e / R1, j = e % R1;
    sincospi(-2.0 * (double)((j * r) % M) / (double)M, &s, &c);
    tband[i] = make_float2((float)c, (float)s);
  }
  if (i < 4096) {
    sincospi(-2.0 * (double)i / 4096.0, &s, &c);
    t4096[i] = make_float2((float)c, (float)s);
  }
  if (i < N) {
    const int64_t u = i >> logQ, q = i & ((int64_t(1) << logQ) - 1);
    sincospi(-2.0 * (double)((q * u) % N) / (double)N, &s, &c);
    t4[i] = make_float2((float)c, (float)s);
  }
}

// h_0 over a whole slice, j = 0..2N-1 (the slice kernel's input weights)
__global__ void k_slice_window(int64_t N, int64_t M, float* h0) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= 2 * N) return;
  const int64_t d = j > N ? j - N : N - j;
  const int64_t a0 = (N - M) / 2;
  double v = 0.0;
  if (d <= a0) {
    v = 1.0;
  } else if (2 * d < N + M) {
    const double c = cospi(0.5 * (double)(d - a0) / (double)M);
    v = c * c;
  }
  h0[j] = (float)v;
}

// Tukey transition h_0 at |j - N| = (N - M)/2 + o, o = 0..M
__global__ void k_tukey(int64_t M, float* hw) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o > M) return;
  const double c = cospi(0.5 * (double)o / (double)M);
  hw[o] = (float)(c * c);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// One lane each, then every further CTA (up to `ctas`) to the group whose
// estimated time per lane, cost / lanes, is largest.
std::vector<int> balance_lanes(const std::vector<double>& cost, int ctas) {
  const int G = (int)cost.size();
  std::vector<int> lanes(G, 1);
  for (int c = G; c < ctas; ++c) {
    int best = 0;
    for (int g = 1; g < G; ++g)
      if (cost[g] * lanes[best] > cost[best] * lanes[g]) best = g;
    ++lanes[best];
  }
  return lanes;
}

// CTA -> (group, lane) for the given lanes per group.
std::vector<int2> lane_map(const std::vector<int>& lanes) {
  std::vector<int2> map;
  for (int g = 0; g < (int)lanes.size(); ++g)
    for (int y = 0; y < lanes[g]; ++y) map.push_back(make_int2(g, y));
  return map;
}

cudaError_t upload_lanes(slicq_plan* pl, bool synthesis, const std::vector<int>& lanes) {
  const std::vector<int2> map = lane_map(lanes);
  cudaError_t e = cudaMemcpy(synthesis ? pl->d_cta_map_s : pl->d_cta_map_a, map.data(),
                             sizeof(int2) * map.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(synthesis ? pl->d_lanes_s : pl->d_lanes_a, lanes.data(), sizeof(int) * lanes.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) (synthesis ? pl->n_cta_s : pl->n_cta_a) = (int)map.size();
  return e;
}

// Lanes per group from measured costs: both persistent band kernels run on
// zeros (the timing does not depend on the values) with the same number of
// lanes per group, first once to warm caches and clocks (one slice per
// lane), then five times with eight slices per lane; a group's cost is the
// median over the five runs of its CTAs' SM clocks per slice.  The plan
// keeps its estimated lanes if any step fails.
void calibrate_lanes(slicq_plan* pl) {
  constexpr int kRuns = 5;
  const int G = pl->G;
  // the same lanes per group for both kernels, within both kernels' slots
  const int per = std::max(1, std::min(pl->slots_a, pl->slots_s) / G);
  const std::vector<int> equal(G, per);
  const int64_t S = 8 * (int64_t)per;
  Workspace ws;
  const size_t wbytes = workspace_layout_rows(pl, S, nullptr, &ws);
  const size_t cbytes = sizeof(float2) * (size_t)(S * pl->coefs_per_slice);
  const int ncta = per * G;
  void* work = nullptr;
  float2* coef = nullptr;
  long long* d_cyc = nullptr;
  bool ok = cudaMalloc(&work, wbytes) == cudaSuccess && cudaMalloc(&coef, cbytes) == cudaSuccess &&
            cudaMalloc(&d_cyc, sizeof(long long) * 2 * ncta * kRuns) == cudaSuccess;
  ok = ok && cudaMemset(work, 0, wbytes) == cudaSuccess && cudaMemset(coef, 0, cbytes) == cudaSuccess;
  ok = ok && upload_lanes(pl, false, equal) == cudaSuccess && upload_lanes(pl, true, equal) == cudaSuccess;
  for (int run = 0; ok && run <= kRuns; ++run) {  // run 0 warms up (and is overwritten)
    const int64_t rows = run == 0 ? per : S;
    workspace_layout_rows(pl, rows, work, &ws);
    long long* c = d_cyc + (size_t)std::max(run - 1, 0) * 2 * ncta;
    // each kernel alone on the device: a kernel started early under
    // programmatic dependent launch would count its wait as work
    ok = launch_band_analysis(pl, ws, 1, coef, 0, c) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
         launch_band_synthesis(pl, coef, 1, kSynthInverse, ws, 0, c + ncta) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
  }
  ok = ok && cudaDeviceSynchronize() == cudaSuccess;
  std::vector<long long> cyc(2 * (size_t)ncta * kRuns, 0);
  ok = ok && cudaMemcpy(cyc.data(), d_cyc, sizeof(long long) * cyc.size(), cudaMemcpyDeviceToHost) == cudaSuccess;
  if (ok) {
    for (int kind = 0; kind < 2; ++kind) {  // 0 analysis, 1 synthesis
      std::vector<double> cost(G, 0.0);
      for (int g = 0; g < G; ++g) {
        double c[kRuns];
        for (int run = 0; run < kRuns; ++run) {
          c[run] = 0.0;
          for (int y = 0; y < per; ++y)
            c[run] += (double)cyc[((size_t)run * 2 + kind) * ncta + (size_t)g * per + y];
        }
        std::sort(c, c + kRuns);
        cost[g] = std::max(1.0, c[kRuns / 2] / (double)S);  // each lane ran S / per slices
      }
      (kind ? pl->cost_s : pl->cost_a) = cost;
    }
  }
  cudaFree(work);
  cudaFree(coef);
  cudaFree(d_cyc);
  // measured costs when the runs succeeded, the estimates otherwise
  upload_lanes(pl, false, balance_lanes(pl->cost_a, pl->slots_a));
  upload_lanes(pl, true, balance_lanes(pl->cost_s, pl->slots_s));
}

// Slice cluster size from measurement (slice_cluster = 0): each valid C, from
// the smallest that fits (N / C <= kSlicePer kSliceMaxThreads) up to 8, runs
// the forward and inverse slice kernels (with the transition overlap-add) on
// zeros over 2 x SMs slices: one warm-up run, then three timed runs; the
// plan keeps the C with the smallest median.  It keeps the smallest C if any
// step fails.
void tune_slice_cluster(slicq_plan* pl) {
  if (pl->params.slice_cluster != 0) return;
  std::vector<int> cands;
  for (int C = pl->C; C <= 8 && C <= (1 << pl->logP); C <<= 1) cands.push_back(C);
  if (cands.size() < 2) return;
  const int64_t L2 = 2 * pl->N;
  const int64_t n = (int64_t)pl->num_sms * L2;  // 2 x SMs slices
  const int C0 = pl->C;
  Workspace ws;
  const size_t wbytes = workspace_layout(pl, n, 1, nullptr, &ws);
  float* x = nullptr;
  float* y = nullptr;
  void* work = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMalloc(&x, sizeof(float) * n) == cudaSuccess && cudaMalloc(&y, sizeof(float) * n) == cudaSuccess &&
            cudaMalloc(&work, wbytes) == cudaSuccess && cudaMemset(x, 0, sizeof(float) * n) == cudaSuccess &&
            cudaMemset(work, 0, wbytes) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
            cudaEventCreate(&e1) == cudaSuccess;
  if (ok) workspace_layout(pl, n, 1, work, &ws);
  int best = C0;
  float best_ms = 0.f;
  for (size_t i = 0; ok && i < cands.size(); ++i) {
    set_slice_cluster(pl, cands[i]);
    float t[3];
    for (int run = 0; ok && run < 4; ++run) {
      ok = cudaEventRecord(e0, 0) == cudaSuccess && launch_slice_forward(pl, x, n, 1, ws, 0) == cudaSuccess &&
           launch_slice_inverse(pl, n, 1, kSynthInverse, ws, y, 0) == cudaSuccess &&
           launch_slice_ola(pl, n, 1, ws, y, 0) == cudaSuccess && cudaEventRecord(e1, 0) == cudaSuccess &&
           cudaEventSynchronize(e1) == cudaSuccess;
      if (ok && run > 0) ok = cudaEventElapsedTime(&t[run - 1], e0, e1) == cudaSuccess;
    }
    if (!ok) break;
    std::sort(t, t + 3);
    if (i == 0 || t[1] < best_ms) {
      best_ms = t[1];
      best = cands[i];
    }
  }
  cudaFree(x);
  cudaFree(y);
  cudaFree(work);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  set_slice_cluster(pl, ok ? best : C0);
}

}  // namespace

slicq_status build_tables(slicq_plan* pl) {
  const int nch = pl->n_channels;
  const int64_t L2 = 2 * pl->N;
  const int64_t Mtr = pl->params.trans_len;
  // arena layout
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align256(off + bytes); return o; };
  const size_t o_bands = take(sizeof(BandDesc) * nch);
  const size_t o_groups = take(sizeof(GroupDesc) * pl->G);
  const size_t o_tb = take(sizeof(int16_t) * pl->thread_band.size());
  const size_t o_slot = take(sizeof(int32_t) * pl->slot_base.size());
  const size_t o_shared = take(sizeof(int4) * std::max<size_t>(pl->shared.size(), 1));
  // spectrogram: half-coefficient i of a slice -> (off_k, log2 M_k) of its channel
  std::vector<int2> half(pl->coefs_per_slice / 2);
  for (int k = 0; k < nch; ++k) {
    const BandDesc& b = pl->bands[k];
    for (int r = 0; r < (1 << (b.log2M - 1)); ++r) half[b.coef_off / 2 + r] = make_int2(b.coef_off, b.log2M);
  }
  const size_t o_half = take(sizeof(int2) * std::max<size_t>(half.size(), 1));
  // transposition: centre bin of each channel (rounded to even on ties)
  std::vector<int32_t> jc(nch);
  for (int k = 0; k < nch; ++k) jc[k] = (int32_t)std::nearbyint(pl->xi[k] * (double)L2 / pl->params.fs);
  const size_t o_jc = take(sizeof(int32_t) * nch);
  const size_t o_ga = take(sizeof(float) * (pl->win_total + 32));  // + padding
  const size_t o_gs = take(sizeof(float) * (pl->win_total + 32));  // + padding
  const size_t o_gadj = take(sizeof(float) * (pl->win_total + 32));  // + padding
  // persistent band kernels: as many CTAs as the SMs hold at once (at least
  // one per group), lanes (CTAs) per group chosen so that the estimated time
  // of a lane, cost / lanes, is as even as possible
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) == cudaSuccess && sms > 0)
      pl->num_sms = sms;
  }
  // (these estimates from the group sizes are replaced by measured costs in
  // calibrate_lanes once the tables exist)
  pl->slots_a = pl->num_sms * band_ctas_per_sm(pl, false);
  pl->slots_s = pl->num_sms * band_ctas_per_sm(pl, true);
  std::vector<int> lanes_a = balance_lanes(pl->cost_a, pl->slots_a);
  std::vector<int> lanes_s = balance_lanes(pl->cost_s, pl->slots_s);
  std::vector<int2> map_a = lane_map(lanes_a), map_s = lane_map(lanes_s);
  pl->n_cta_a = (int)map_a.size();
  pl->n_cta_s = (int)map_s.size();
  const size_t map_cap = (size_t)std::max(pl->G, std::max(pl->slots_a, pl->slots_s));  // sum of lanes at most
  const size_t o_map_a = take(sizeof(int2) * map_cap);
  const size_t o_lanes_a = take(sizeof(int) * pl->G);
  const size_t o_map_s = take(sizeof(int2) * map_cap);
  const size_t o_lanes_s = take(sizeof(int) * pl->G);
  const size_t o_hw = take(sizeof(float) * (Mtr + 1));
  const size_t o_h0 = take(sizeof(float) * L2);
  const size_t o_twlo = take(sizeof(float2) * (size_t(1) << pl->tw_lb));
  const size_t o_twhi = take(sizeof(float2) * (L2 >> pl->tw_lb));
  const size_t o_twband = take(sizeof(float2) * 2032);
  const size_t o_tw4 = take(sizeof(float2) * pl->N);
  const size_t o_tw4096 = take(sizeof(float2) * 4096);
  const size_t o_err = take(sizeof(int));
  if (cudaMalloc(&pl->d_arena, off) != cudaSuccess) return SLICQ_ENOMEM;
  char* base = (char*)pl->d_arena;
  pl->d_bands = (BandDesc*)(base + o_bands);
  pl->d_groups = (GroupDesc*)(base + o_groups);
  pl->d_thread_band = (int16_t*)(base + o_tb);
  pl->d_slot_base = (int32_t*)(base + o_slot);
  pl->d_shared = (int4*)(base + o_shared);
  pl->d_half_chan = (int2*)(base + o_half);
  pl->d_jc = (int32_t*)(base + o_jc);
  pl->d_ga = (float*)(base + o_ga);
  pl->d_gs = (float*)(base + o_gs);
  pl->d_gadj = (float*)(base + o_gadj);
  pl->d_hw = (float*)(base + o_hw);
  pl->d_h0 = (float*)(base + o_h0);
  pl->d_cta_map_a = (int2*)(base + o_map_a);
  pl->d_lanes_a = (int*)(base + o_lanes_a);
  pl->d_cta_map_s = (int2*)(base + o_map_s);
  pl->d_lanes_s = (int*)(base + o_lanes_s);
  pl->d_tw_lo = (float2*)(base + o_twlo);
  pl->d_tw_hi = (float2*)(base + o_twhi);
  pl->d_twband = (float2*)(base + o_twband);
  pl->d_tw4 = (float2*)(base + o_tw4);
  pl->d_tw4096 = (float2*)(base + o_tw4096);
  pl->d_err = (int*)(base + o_err);

  slicq_status st = SLICQ_OK;
  cudaError_t e = cudaSuccess;
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) == cudaSuccess && sms > 0)
      pl->num_sms = sms;
  }
  e = cudaMemset(pl->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_bands, pl->bands.data(), sizeof(BandDesc) * nch, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_groups, pl->groups.data(), sizeof(GroupDesc) * pl->G, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_thread_band, pl->thread_band.data(),
                   sizeof(int16_t) * pl->thread_band.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_slot_base, pl->slot_base.data(), sizeof(int32_t) * pl->slot_base.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !pl->shared.empty())
    e = cudaMemcpy(pl->d_shared, pl->shared.data(), sizeof(int4) * pl->shared.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_jc, jc.data(), sizeof(int32_t) * nch, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !half.empty())
    e = cudaMemcpy(pl->d_half_chan, half.data(), sizeof(int2) * half.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = upload_lanes(pl, false, lanes_a);
  if (e == cudaSuccess) e = upload_lanes(pl, true, lanes_s);
  if (e != cudaSuccess) return SLICQ_ECUDA;

  // temporaries for the FP64 computation
  std::vector<WinJob> jobs(nch);
  for (int k = 0; k < nch; ++k) {
    const BandDesc& b = pl->bands[k];
    jobs[k] = WinJob{pl->jlo[k], pl->xi[k], pl->omega[k], b.len, b.win_off,
                     (k == 0 || k == pl->K + 1) ? 1 : 0, 1 << b.log2M, b.j0,
                     (k >= 1 && k <= pl->K) ? 1 : 0};
  }
  WinJob* d_jobs = nullptr;
  double* d_g64 = nullptr;
  double* d_d = nullptr;
  int* d_bad = nullptr;
  const int64_t wt = std::max<int64_t>(pl->win_total, 1);
  if (cudaMalloc(&d_jobs, sizeof(WinJob) * nch) != cudaSuccess ||
      cudaMalloc(&d_g64, sizeof(double) * wt) != cudaSuccess ||
      cudaMalloc(&d_d, sizeof(double) * L2) != cudaSuccess ||
      cudaMalloc(&d_bad, sizeof(int)) != cudaSuccess) {
    st = SLICQ_ENOMEM;
  }
  int bad = 0;
  if (st == SLICQ_OK) {
    e = cudaMemcpy(d_jobs, jobs.data(), sizeof(WinJob) * nch, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_bad, 0, sizeof(int));
    const int T = 256;
    if (e == cudaSuccess && pl->win_total > 0) {
      k_windows<<<(unsigned)((pl->win_total + T - 1) / T), T>>>(d_jobs, nch, pl->win_total, pl->params.fs,
                                                                (double)L2, pl->params.window, d_g64);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_diagonal<<<(unsigned)((L2 + T - 1) / T), T>>>(d_jobs, nch, d_g64, L2, d_d);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && pl->win_total > 0) {
      k_duals<<<(unsigned)((pl->win_total + T - 1) / T), T>>>(d_jobs, nch, pl->win_total, d_g64, d_d, L2,
                                                              pl->d_ga, pl->d_gs, pl->d_gadj, d_bad);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      const int64_t nt = std::max<int64_t>(std::max<int64_t>(int64_t(1) << pl->tw_lb, L2 >> pl->tw_lb),
                                           std::max<int64_t>(4096, pl->N));
      k_twiddles<<<(unsigned)((nt + T - 1) / T), T>>>(L2, pl->tw_lb, pl->logQ, pl->d_tw_lo, pl->d_tw_hi,
                                                      pl->d_twband, pl->d_tw4, pl->d_tw4096);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_tukey<<<(unsigned)((Mtr + 1 + T - 1) / T), T>>>(Mtr, pl->d_hw);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_slice_window<<<(unsigned)((L2 + T - 1) / T), T>>>(pl->N, Mtr, pl->d_h0);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = SLICQ_ECUDA;
    else if (bad) st = SLICQ_EINVAL;
  }
  cudaFree(d_jobs);
  cudaFree(d_g64);
  cudaFree(d_d);
  cudaFree(d_bad);
  if (st == SLICQ_OK) calibrate_lanes(pl);
  if (st == SLICQ_OK) tune_slice_cluster(pl);
  return st;
}

}  // namespace slicq
