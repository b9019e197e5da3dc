// Slice stage of the sliCQ: one thread-block cluster per slice.
//
// Forward (Algorithm 3, slicing, and Algorithm 1, line 2): the slice
// f^m[j] = f[j + (m-1)N] h_0[j - N] (j < 2N, circular, zero-padded) is
// transformed with a real-input DFT of length 2N, computed as an N-point
// complex DFT of z[n] = f^m[2n] + i f^m[2n+1] followed by the even/odd split.
// Bins 0..N go to the workspace for the band kernels.
//
// Inverse (Algorithm 2, last line, and Algorithm 4, overlap-add): bins 0..N
// of the synthesised slice spectrum are extended Hermitian, transformed back
// with an N-point complex DFT, multiplied by the dual slicing window
// (indicator of the support of h_0; h_0 itself for the adjoint) and
// overlap-added.  Samples where only this slice contributes are stored
// directly; the samples of each transition go to two patch rows (side 0:
// the earlier slice, side 1: the later one) that slice_ola_kernel adds, so
// the result is deterministic and needs no zero-filled output.
//
// The N-point DFT is a four-step transform N = P Q distributed over the C
// CTAs of the cluster: column DFTs (length P) over the CTA's Q/C columns,
// twiddle W_N^{q u}, one exchange through distributed shared memory, row DFTs
// (length Q) over the CTA's P/C rows; element (u, v) of the result is
// Z[u + P v].  Each DFT is a two-pass Stockham team transform in registers.
#include <cooperative_groups.h>

#include "fft_common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace slicq {
namespace {

struct SliceArgs {
  const float* __restrict__ f;    // forward input [batch][n]
  float* out;                     // inverse output [batch][n]
  float2* spec;                   // [slice][spec_stride]
  int64_t spec_stride;
  int64_t n, L;
  int S, N, Mtr;
  int C, logQc, logPc;
  const float* __restrict__ hw;   // Tukey transition, Mtr + 1 values
  const float2* __restrict__ h0;  // h_0 over the slice as pairs (h_0[2e], h_0[2e+1])
  TwiddleTables tw;               // global two-level tables (copied to shared memory)
  const float2* __restrict__ twband;  // pass-2 tables of lengths 16..1024, [r][j] per length
  const float2* __restrict__ tw4096;  // exp(-2 pi i t / 4096), t < 4096
  const float2* __restrict__ tw4; // four-step twiddles exp(-2 pi i q u / N) at [u Q + q]
  int tw_off;                     // shared-memory offset (float2) of the table copy
  float* ola_patch;               // [slice][2][ola_stride]: the two sides of each transition
  int ola_stride;                 // Mtr rounded up to a multiple of 4
  const RowDesc* __restrict__ rows;  // ragged batch: per-row clip description (or null)
  int adjoint;                    // multiply the output by h_0 instead of 1
};

// h_0 at slice sample j (reading of the Tukey window, Sec. 4.2).
__device__ __forceinline__ float slicing_window(const SliceArgs& a, int j) {
  const int d = abs(j - a.N);
  const int a0 = (a.N - a.Mtr) >> 1;
  const float ht = __ldg(a.hw + min(max(d - a0, 0), a.Mtr));
  return d <= a0 ? 1.f : (2 * d < a.N + a.Mtr ? ht : 0.f);
}

// Clip of slice row s: signal offset, length, padded length, slice index.
__device__ __forceinline__ void row_of(const SliceArgs& a, int64_t s, int64_t& sig_off, int& n,
                                       int& L, int& m) {
  if (a.rows) {
    const RowDesc r = a.rows[s];
    sig_off = r.sig_off;
    n = r.n;
    L = r.L;
    m = r.m;
  } else {
    const int64_t b = s / a.S;
    sig_off = b * a.n;
    n = (int)a.n;
    L = (int)a.L;
    m = (int)(s - b * a.S);
  }
}

template <int LOGP, int LOGQ>
struct Geo {
  static constexpr int P = 1 << LOGP, Q = 1 << LOGQ;
  using TP = Team<LOGP, kSlicePer>;
  using TQ = Team<LOGQ, kSlicePer>;
  static constexpr int CS1 = TP::BUF;      // odd column stride of pass buffers
  static constexpr int XS1 = P + 1;        // column stride of the exchange layout
  static constexpr int CS3 = TQ::BUF;
  static constexpr int ZS3 = Q + 1;
};

// Phase 1 + exchange + phase 3 of the distributed four-step DFT.  LOAD(e)
// returns input element e (0 <= e < N).  On return res[i * R2q + r] holds
// Z[u + P v] for u = rank * P/C + ul, v = (tt + TTq i) + r R1q, and the shared
// memory may be reused after a __syncthreads().
// Pass-2 twiddle exp(SIGN 2 pi i j r / 2^LOGL) of a team transform of length
// 2^LOGL (a column or row DFT) from its shared [r][j] table: one load.
template <int LOGL, int SIGN>
struct PassTw {
  const float2* t;
  __device__ __forceinline__ float2 operator()(int j, int r) const {
    const float2 w = t[r * Team<LOGL>::R1 + j];
    return SIGN < 0 ? w : c_conj(w);
  }
};

// Shared-memory copies: the two-level table exp(-2 pi i t / 2N) at tw_off,
// then the pass-2 tables of lengths P and Q and exp(-pi i v / Q), v < Q
// (caller synchronises).
struct SliceTables {
  SmemTwiddles tw;
  const float2* twP;
  const float2* twQ;
};

template <int LOGP, int LOGQ>
__device__ __forceinline__ SliceTables stage_twiddles(const SliceArgs& a, float2* sm) {
  constexpr int P = 1 << LOGP, Q = 1 << LOGQ;
  float2* lo = sm + a.tw_off;
  const int nlo = 1 << a.tw.lb;
  float2* hi = lo + nlo;
  const int nhi = (2 * a.N) >> a.tw.lb;
  float2* tp = hi + nhi;
  float2* tq = tp + P;
  float2* th = tq + Q;
  for (int i = threadIdx.x; i < nlo; i += blockDim.x) lo[i] = __ldg(a.tw.lo + i);
  for (int i = threadIdx.x; i < nhi; i += blockDim.x) hi[i] = __ldg(a.tw.hi + i);
  for (int i = threadIdx.x; i < P; i += blockDim.x) tp[i] = __ldg(a.twband + (P - 16) + i);
  for (int i = threadIdx.x; i < Q; i += blockDim.x) tq[i] = __ldg(a.twband + (Q - 16) + i);
  // e^{-pi i v / Q} = e^{-2 pi i (v 2048 / Q) / 4096}, v < Q (Q <= 2048)
  for (int i = threadIdx.x; i < Q; i += blockDim.x) th[i] = __ldg(a.tw4096 + i * (2048 / Q));
  return SliceTables{SmemTwiddles{lo, hi, a.tw.lb}, tp, tq};
}

// Row u of phase 3 held at local slot ul of CTA `rank` when rows are
// paired (PAIRED): the CTA holds rows rank H + w (w < H = Pc / 2) in slots
// w and their partners P - (rank H + w) in slots H + w; CTA 0's row 0 is
// its own partner, so its slot H holds the self-paired row P / 2.  The
// even/odd split of the forward then finds every partner row locally.
__device__ __forceinline__ int paired_row(int rank, int ul, int Pc, int P) {
  const int H = Pc >> 1;
  if (ul < H) return rank * H + ul;
  const int x = rank * H + ul - H;
  return x == 0 ? P / 2 : P - x;
}

// Local slot of the partner row (P - u, or u itself for u = 0, P / 2) of
// the row in slot ul, paired layout.
__device__ __forceinline__ int paired_partner_slot(int rank, int ul, int Pc) {
  const int H = Pc >> 1;
  if (rank == 0 && (ul == 0 || ul == H)) return ul;
  return ul < H ? ul + H : ul - H;
}

template <int LOGP, int LOGQ, int SIGN, bool PAIRED, class Load>
__device__ __forceinline__ void fourstep(const SliceArgs& a, cg::cluster_group& cluster,
                                         float2* sm, const SliceTables& tabs, Load load,
                                         float2* res, int& ul_out, int& tt_out) {
  using G = Geo<LOGP, LOGQ>;
  using TP = typename G::TP;
  using TQ = typename G::TQ;
  const int t = threadIdx.x;
  const int rank = (int)cluster.block_rank();

  // ---- phase 1: column DFTs over p for the CTA's columns q
  {
    const int Qc = 1 << a.logQc;
    const int ql = t & (Qc - 1);
    const int tt = t >> a.logQc;
    const int q = rank * Qc + ql;
    float2* buf = sm + ql * G::CS1;
    team_pass1<LOGP, SIGN, kSlicePer>(tt, buf, [&](int p) { return load(p * G::Q + q); });
    __syncthreads();
    float2 col[TP::HELD];
    team_pass2<LOGP, SIGN, kSlicePer>(tt, buf, PassTw<LOGP, SIGN>{tabs.twP}, col);
    __syncthreads();
    // four-step twiddle W_N^{q u} = W_2N^{2 q u}, then the exchange layout [ql][u]
#pragma unroll
    for (int i = 0; i < TP::J2; ++i)
#pragma unroll
      for (int r = 0; r < TP::R2; ++r) {
        const int u = team_out_index<LOGP, kSlicePer>(tt, i, r);
        float2 w = __ldg(a.tw4 + u * G::Q + q);
        if (SIGN > 0) w.y = -w.y;
        sm[ql * G::XS1 + u] = c_mul(col[i * TP::R2 + r], w);
      }
  }
  cluster.sync();

  // ---- phase 3: row DFTs over q for the CTA's rows u
  const int Pc = 1 << a.logPc;
  const int ul = t & (Pc - 1);
  const int tt = t >> a.logPc;
  const int u = PAIRED ? paired_row(rank, ul, Pc, G::P) : rank * Pc + ul;
  {
    float2 v1[TQ::J1 * TQ::R1];
#pragma unroll
    for (int i = 0; i < TQ::J1; ++i) {
      const int j = tt + TQ::TT * i;
#pragma unroll
      for (int r = 0; r < TQ::R1; ++r) {
        const int q = j + r * TQ::R2;
        const int src = q >> a.logQc;
        const int ql = q & ((1 << a.logQc) - 1);
        const float2* rsm = cluster.map_shared_rank(sm, src);
        v1[i * TQ::R1 + r] = rsm[ql * G::XS1 + u];
      }
    }
    cluster.sync();  // every CTA has read its rows; the exchange buffer is free
    float2* buf = sm + ul * G::CS3;
#pragma unroll
    for (int i = 0; i < TQ::J1; ++i) {
      const int j = tt + TQ::TT * i;
      float2 v[TQ::R1];
#pragma unroll
      for (int r = 0; r < TQ::R1; ++r) v[r] = v1[i * TQ::R1 + r];
      dft_reg<TQ::R1, SIGN>(v);
#pragma unroll
      for (int r = 0; r < TQ::R1; ++r) buf[TQ::pad1(j, r)] = v[r];
    }
    __syncthreads();
    team_pass2<LOGQ, SIGN, kSlicePer>(tt, buf, PassTw<LOGQ, SIGN>{tabs.twQ}, res);
  }
  ul_out = ul;
  tt_out = tt;
}

// ------------------------------------------------------------- forward ---

template <int LOGP, int LOGQ>
__global__ void __launch_bounds__(kSliceMaxThreads, kSlicePer == 16 ? 3 : 2) slice_forward_kernel(SliceArgs a) {
  using G = Geo<LOGP, LOGQ>;
  using TQ = typename G::TQ;
  extern __shared__ float2 sm[];
  pdl_launch_dependents();
  cg::cluster_group cluster = cg::this_cluster();
  const int64_t s = blockIdx.x / a.C;
  int64_t sig_off;
  int n32, L32, m;                            // the entry points keep L < 2^31
  row_of(a, s, sig_off, n32, L32, m);
  const float* f = a.f + sig_off;
  const int base = (m - 1) * a.N;             // position of slice sample 0 (slice 0: -N)
  const bool vec = (sig_off & 1) == 0;        // f is 8-byte aligned (uniform per CTA)

  // Element e of the packed slice is (x[2e], x[2e+1]); x[j] = f[j + (m-1)N] h_0[j-N].
  // Branch-free: every load is issued with a clamped index and weighted by 0
  // outside the support of h_0 and past the end of the signal.
  auto load = [&](int e) -> float2 {
    const int j = 2 * e;
    const float2 w = __ldg(a.h0 + e);
    const float w0 = w.x, w1 = w.y;
    int t = base + j;
    if (t < 0) t += L32; else if (t >= L32) t -= L32;   // t even, t + 1 < L
    const bool in0 = t < n32, in1 = t + 1 < n32;
    float2 x;
    if (vec && in1) {
      x = __ldg(reinterpret_cast<const float2*>(f + t));
    } else {
      x.x = __ldg(f + (in0 ? t : 0));
      x.y = __ldg(f + (in1 ? t + 1 : 0));
    }
    x.x = in0 ? x.x * w0 : 0.f;
    x.y = in1 ? x.y * w1 : 0.f;
    return x;
  };

  // the tables are first read in pass 2 of the column DFTs: the barrier after
  // pass 1 covers the staging, so the input loads start right away
  const SliceTables tabs = stage_twiddles<LOGP, LOGQ>(a, sm);
  const SmemTwiddles& tws = tabs.tw;
  pdl_wait();  // the input (and the previous kernel's use of the workspace)
  const int Pc = 1 << a.logPc;
  {
    float2 res[TQ::HELD];
    int ul, tt;
    fourstep<LOGP, LOGQ, -1, true>(a, cluster, sm, tabs, load, res, ul, tt);
    __syncthreads();
    // Z to shared memory, column-major [v][ul], for the even/odd split (needs
    // Z[N - k] from the partner row, held by this CTA): local reads, partner
    // reads and the stores of X are then all contiguous across a warp
#pragma unroll
    for (int i = 0; i < TQ::J2; ++i)
#pragma unroll
      for (int r = 0; r < TQ::R2; ++r)
        sm[team_out_index<LOGQ, kSlicePer>(tt, i, r) * Pc + ul] = res[i * TQ::R2 + r];  // [v][ul]
  }
  __syncthreads();

  // X[k], k = u + P v for this CTA's rows u; X[N] from k = 0.  A thread keeps
  // one row u (fixed: idx & (Pc - 1) with blockDim a multiple of Pc), so its
  // partner row P - u (row 0 for u = 0), that row's local slot and
  // e^{-2 pi i u / 2N} are computed once; e^{-2 pi i k / 2N} =
  // e^{-2 pi i u / 2N} e^{-pi i v / Q}.
  const int rank = (int)cluster.block_rank();
  float2* X = a.spec + s * a.spec_stride;
  const int ul = threadIdx.x & (Pc - 1);
  const int u = paired_row(rank, ul, Pc, G::P);
  const float2* psm = sm + paired_partner_slot(rank, ul, Pc);
  const float2 wu = tws((uint32_t)u);
  const float2* thalf = tabs.twQ + G::Q;  // e^{-pi i v / Q}, v < Q (staged after the Q table)
  const int vstep = (int)blockDim.x >> a.logPc;
#pragma unroll 8
  for (int v = (int)threadIdx.x >> a.logPc; v < G::Q; v += vstep) {
    const int vp = u == 0 ? ((G::Q - v) & (G::Q - 1)) : G::Q - 1 - v;
    const float2 zp = c_conj(psm[vp * Pc]);
    const float2 z = sm[v * Pc + ul];
    // even part E = (Z[k] + conj Z[N-k]) / 2, odd part O = (Z[k] - conj Z[N-k]) / 2i
    const float2 E = c_scale(c_add(z, zp), 0.5f);
    const float2 D = c_sub(z, zp);
    const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
    const int k = u + G::P * v;
    X[k] = c_add(E, c_mul(c_mul(wu, thalf[v]), O));
    if (k == 0) X[a.N] = c_sub(E, O);
  }
}

// ------------------------------------------------------------- inverse ---

template <int LOGP, int LOGQ>
__global__ void __launch_bounds__(kSliceMaxThreads, kSlicePer == 16 ? 3 : 2) slice_inverse_kernel(SliceArgs a) {
  using G = Geo<LOGP, LOGQ>;
  using TQ = typename G::TQ;
  extern __shared__ float2 sm[];
  pdl_launch_dependents();
  cg::cluster_group cluster = cg::this_cluster();
  const int64_t s = blockIdx.x / a.C;
  int64_t sig_off;
  int n32, L32, m;
  row_of(a, s, sig_off, n32, L32, m);
  const int Sc = L32 / a.N;                   // slices of this row's clip
  const int64_t tr0 = a.rows ? a.rows[s].tr_base : s - m;  // slot of the clip's transition 0
  const float2* H = a.spec + s * a.spec_stride;
  const int N = a.N;

  const SliceTables tabs = stage_twiddles<LOGP, LOGQ>(a, sm);
  const SmemTwiddles& tws = tabs.tw;
  pdl_wait();  // the synthesised spectra
  __syncthreads();
  // Z[k] = (H[k] + conj H[N-k]) + i e^{+2 pi i k / 2N} (H[k] - conj H[N-k])
  auto load = [&](int k) -> float2 {
    const float2 h = H[k];
    const float2 hc = c_conj(H[N - k]);
    const float2 sum = c_add(h, hc);
    const float2 dif = c_mul(c_sub(h, hc), c_conj(tws((uint32_t)k)));
    return make_float2(sum.x - dif.y, sum.y + dif.x);
  };

  {
    float2 res[TQ::HELD];
    int ul, tt;
    fourstep<LOGP, LOGQ, +1, false>(a, cluster, sm, tabs, load, res, ul, tt);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TQ::J2; ++i)
#pragma unroll
      for (int r = 0; r < TQ::R2; ++r) sm[ul * G::ZS3 + team_out_index<LOGQ, kSlicePer>(tt, i, r)] = res[i * TQ::R2 + r];
  }
  __syncthreads();

  // Time samples j = 2n, 2n+1 of z[n], n = u + P v; this CTA holds u in
  // [rank Pc, (rank+1) Pc), a thread one u and every v it visits.  With
  // d = j - N: |d| <= a0 only this slice contributes (stored directly);
  // a0 < d < a0 + M is the right transition (shared with slice m+1, this
  // slice is side 0, offset d - a0) and -(a0 + M) < d < -a0 the left one
  // (shared with slice m-1, side 1, offset j - a0).
  const int Pc = 1 << a.logPc;
  const int rank = (int)cluster.block_rank();
  const int Mtr = a.Mtr;
  const int a0 = (N - Mtr) >> 1;
  const int base = (m - 1) * N;
  float* out = a.out + sig_off;
  float* pr = a.ola_patch + ((tr0 + m) * 2 + 0) * (int64_t)a.ola_stride;
  float* pl = a.ola_patch + ((tr0 + (m + Sc - 1) % Sc) * 2 + 1) * (int64_t)a.ola_stride;
  const bool vec = (sig_off & 1) == 0 && (a0 & 1) == 0;  // 8-byte pair stores
  // one sample: direct, a transition side, or outside the support
  auto put = [&](int j, float x) {
    const int d = j - N;
    if (d >= -a0 && d <= a0) {
      int t = base + j;
      if (t < 0) t += L32; else if (t >= L32) t -= L32;
      if (t < n32) out[t] = x;
    } else if (d > a0 && d < a0 + Mtr) {
      pr[d - a0] = a.adjoint ? x * slicing_window(a, j) : x;
    } else if (d < -a0 && d > -a0 - Mtr) {
      pl[j - a0] = a.adjoint ? x * slicing_window(a, j) : x;
    }
  };
  // rows v whose samples can lie in the support |d| < a0 + M
  const int n_lo = max(0, (N - a0 - Mtr) >> 1), n_hi = min(N - 1, (N + a0 + Mtr) >> 1);
  const int v_lo = n_lo >> LOGP, v_hi = n_hi >> LOGP;
  const int ul = threadIdx.x & (Pc - 1);
  const int u = rank * Pc + ul;
  for (int v = v_lo + ((int)threadIdx.x >> a.logPc); v <= v_hi; v += (int)blockDim.x >> a.logPc) {
    const float2 z = sm[ul * G::ZS3 + v];
    const int j = 2 * (u + (v << LOGP));
    const int d = j - N;
    if (vec && d >= -a0 && d + 1 <= a0) {  // both samples direct
      int t = base + j;
      if (t < 0) t += L32; else if (t >= L32) t -= L32;
      if (t + 1 < n32) *reinterpret_cast<float2*>(out + t) = z;
      else if (t < n32) out[t] = z.x;
    } else if (vec && !a.adjoint && d > a0 && d + 1 < a0 + Mtr) {  // both in the right transition
      *reinterpret_cast<float2*>(pr + (d - a0)) = z;
    } else if (vec && !a.adjoint && d < -a0 - 1 && d > -a0 - Mtr) {  // both in the left transition
      *reinterpret_cast<float2*>(pl + (j - a0)) = z;
    } else {
      put(j, z.x);
      put(j + 1, z.y);
    }
  }
  // no remote shared-memory access after the exchange inside fourstep()
}

// Overlap-add of the transitions: output sample t = mN + a0 + o (o = 1..M-1,
// t < L) of row s's clip is side 0 (slice m) + side 1 (slice m + 1).  A
// thread takes offsets 4i .. 4i + 3 (16-byte patch loads; o = 0 is not a
// transition sample).
__global__ void __launch_bounds__(256) slice_ola_kernel(SliceArgs a, int64_t slice_base) {
  pdl_launch_dependents();
  pdl_wait();
  const int o0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int64_t s = slice_base + blockIdx.y;
  if (o0 >= a.Mtr) return;
  int64_t sig_off;
  int n32, L32, m;
  row_of(a, s, sig_off, n32, L32, m);
  const int64_t slot = a.rows ? a.rows[s].tr_base + m : s;
  const float* p = a.ola_patch + slot * 2 * (int64_t)a.ola_stride;  // 16-byte aligned rows
  const float4 x0 = __ldcs(reinterpret_cast<const float4*>(p + o0));
  const float4 x1 = __ldcs(reinterpret_cast<const float4*>(p + a.ola_stride + o0));
  const float v[4] = {x0.x + x1.x, x0.y + x1.y, x0.z + x1.z, x0.w + x1.w};
  const int t0 = m * a.N + ((a.N - a.Mtr) >> 1) + o0;  // < L: the transition ends before the clip
  float* out = a.out + sig_off;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = o0 + q;
    if (o >= 1 && o < a.Mtr && t0 + q < n32) out[t0 + q] = v[q];
  }
}

template <int LOGP, int LOGQ>
cudaError_t launch_slice(bool forward, const slicq_plan* pl, const SliceArgs& a, int64_t slices,
                         cudaStream_t st) {
  void (*kern)(SliceArgs) = forward ? slice_forward_kernel<LOGP, LOGQ> : slice_inverse_kernel<LOGP, LOGQ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->slice_smem);
  if (e != cudaSuccess) return e;
  const int threads = (1 << (LOGP + LOGQ)) / (kSlicePer * pl->C);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(slices * pl->C));
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = pl->slice_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl->C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // see pdl_wait
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t dispatch(bool forward, const slicq_plan* pl, const SliceArgs& a, int64_t slices,
                     cudaStream_t st) {
  switch (pl->logP * 16 + pl->logQ) {
    case 5 * 16 + 5: return launch_slice<5, 5>(forward, pl, a, slices, st);
    case 5 * 16 + 6: return launch_slice<5, 6>(forward, pl, a, slices, st);
    case 6 * 16 + 6: return launch_slice<6, 6>(forward, pl, a, slices, st);
    case 6 * 16 + 7: return launch_slice<6, 7>(forward, pl, a, slices, st);
    case 7 * 16 + 7: return launch_slice<7, 7>(forward, pl, a, slices, st);
    case 7 * 16 + 8: return launch_slice<7, 8>(forward, pl, a, slices, st);
    case 8 * 16 + 8: return launch_slice<8, 8>(forward, pl, a, slices, st);
    default: return cudaErrorInvalidValue;
  }
}

SliceArgs make_args(const slicq_plan* pl, const Workspace& ws, int64_t n) {
  SliceArgs a{};
  a.spec = ws.spec;
  a.spec_stride = ws.spec_stride;
  a.n = n;
  a.L = ws.L;
  a.S = (int)ws.S;
  a.N = (int)pl->N;
  a.Mtr = (int)pl->params.trans_len;
  a.C = pl->C;
  a.logQc = pl->logQ - ilog2c(pl->C);
  a.logPc = pl->logP - ilog2c(pl->C);
  a.hw = pl->d_hw;
  a.h0 = reinterpret_cast<const float2*>(pl->d_h0);
  a.tw = TwiddleTables{pl->d_tw_lo, pl->d_tw_hi, pl->tw_lb};
  a.tw_off = pl->slice_tw_off;
  a.twband = pl->d_twband;
  a.tw4096 = pl->d_tw4096;
  a.tw4 = pl->d_tw4;
  a.ola_patch = ws.ola_patch;
  a.ola_stride = (a.Mtr + 3) & ~3;
  return a;
}

}  // namespace

cudaError_t launch_slice_forward(const slicq_plan* pl, const float* f, int64_t n, int64_t batch,
                                 const Workspace& ws, cudaStream_t st, const RowDesc* rows) {
  SliceArgs a = make_args(pl, ws, n);
  a.f = f;
  a.rows = rows;
  return dispatch(true, pl, a, batch * ws.S, st);
}

cudaError_t launch_slice_inverse(const slicq_plan* pl, int64_t n, int64_t batch, SynthKind kind,
                                 const Workspace& ws, float* out, cudaStream_t st, const RowDesc* rows) {
  SliceArgs a = make_args(pl, ws, n);
  a.out = out;
  a.rows = rows;
  a.adjoint = kind == kSynthAdjoint;
  return dispatch(false, pl, a, batch * ws.S, st);
}

cudaError_t launch_slice_ola(const slicq_plan* pl, int64_t n, int64_t batch, const Workspace& ws, float* out,
                             cudaStream_t st, const RowDesc* rows) {
  SliceArgs a = make_args(pl, ws, n);
  a.out = out;
  a.rows = rows;
  const int64_t total = batch * ws.S;
  const unsigned bx = (unsigned)((a.Mtr + 1023) / 1024);  // 4 offsets per thread
  for (int64_t s0 = 0; s0 < total; s0 += kMaxGridY) {
    dim3 grid(bx, (unsigned)(total - s0 < kMaxGridY ? total - s0 : kMaxGridY));
    const cudaError_t e = launch_pdl(slice_ola_kernel, grid, dim3(256), 0, st, a, s0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace slicq
