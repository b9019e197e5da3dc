// Device building blocks of the slice and band FFTs: complex arithmetic,
// table twiddles, in-register DFTs of length <= 32 and the two-pass Stockham
// team transform used by every kernel of the library.
//
// DFT convention (Sec. 2.1 of arXiv:1210.0084 without its 1/sqrt(L), which
// the plan folds into the window tables):
//   SIGN = -1:  X[k] = sum_n x[n] exp(-2 pi i n k / L)
//   SIGN = +1:  x[n] = sum_k X[k] exp(+2 pi i n k / L)
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace slicq {

// ------------------------------------------- programmatic dependent launch ---
// Every hot kernel is launched with programmatic stream serialisation: it
// lets the next kernel in the stream start launching (its CTAs fill SMs this
// grid's tail leaves idle and stage their plan tables), and waits for the
// previous kernel to finish (its writes visible) before it touches any
// workspace, input or output memory.  Without the launch attribute both are
// no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// ---------------------------------------------------------------- complex ---
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (SIGN i)
template <int SIGN>
__device__ __forceinline__ float2 c_mul_i(float2 a) {
  return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------- twiddle tables ---
// exp(-2 pi i t / 2N) = lo[t mod 2^lb] * hi[t >> lb]; both tables hold the
// FP64-computed value rounded to float32 (built once per plan).
struct TwiddleTables {
  const float2* __restrict__ lo;
  const float2* __restrict__ hi;
  int lb;
};

__device__ __forceinline__ float2 twiddle(const TwiddleTables& tw, uint32_t t) {
  const float2 a = __ldg(tw.lo + (t & ((1u << tw.lb) - 1u)));
  const float2 b = __ldg(tw.hi + (t >> tw.lb));
  return c_mul(a, b);
}
// exp(SIGN 2 pi i t / 2N)
template <int SIGN>
__device__ __forceinline__ float2 twiddle_s(const TwiddleTables& tw, uint32_t t) {
  const float2 w = twiddle(tw, t);
  return SIGN < 0 ? w : c_conj(w);
}

// ------------------------------------------------ in-register DFT <= 32 ---
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }
__host__ __device__ constexpr int brev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
  return r;
}

// cos(2 pi e / 32) from the first-quadrant values (decimal expansions of
// cos(pi m / 16), m = 0..8).
__host__ __device__ constexpr float cos32q(int m) {
  return m == 0 ? 1.0f
       : m == 1 ? 0.98078528040323044913f
       : m == 2 ? 0.92387953251128675613f
       : m == 3 ? 0.83146961230254523708f
       : m == 4 ? 0.70710678118654752440f
       : m == 5 ? 0.55557023301960222474f
       : m == 6 ? 0.38268343236508977173f
       : m == 7 ? 0.19509032201612826785f
       : 0.0f;
}
__host__ __device__ constexpr float cos32(int e) {
  return (e & 31) <= 8 ? cos32q(e & 31)
       : (e & 31) <= 16 ? -cos32q(16 - (e & 31))
       : (e & 31) <= 24 ? -cos32q((e & 31) - 16)
       : cos32q(32 - (e & 31));
}
__host__ __device__ constexpr float sin32(int e) { return cos32(e - 8); }

// b * exp(SIGN 2 pi i e / 32) with e a compile-time constant after unrolling.
template <int SIGN>
__device__ __forceinline__ float2 rot32(float2 b, int e) {
  e &= 31;
  if (e == 0) return b;
  if (e == 16) return make_float2(-b.x, -b.y);
  if (e == 8) return c_mul_i<SIGN>(b);
  if (e == 24) return c_mul_i<-SIGN>(b);
  const float c = cos32(e), s = SIGN * sin32(e);
  return make_float2(fmaf(b.x, c, -b.y * s), fmaf(b.x, s, b.y * c));
}

// Natural-order in, natural-order out DFT of length R (R | 32) in registers:
// bit-reversal by renaming, then log2(R) radix-2 decimation-in-time stages.
template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
  constexpr int LOG = ilog2c(R);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = brev(i, LOG);
    if (j > i) {
      const float2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int s = 1; s <= LOG; ++s) {
    const int m = 1 << s, h = m >> 1;
#pragma unroll
    for (int k = 0; k < R; k += m) {
#pragma unroll
      for (int jj = 0; jj < h; ++jj) {
        const float2 b = rot32<SIGN>(v[k + jj + h], jj * (32 / m));
        const float2 a = v[k + jj];
        v[k + jj] = c_add(a, b);
        v[k + jj + h] = c_sub(a, b);
      }
    }
  }
}

// ------------------------------------------- two-pass Stockham (team) ---
// A DFT of length Lf = R1 * R2 (R1 = 2^ceil(log/2), R2 = 2^floor(log/2))
// done by a team of TT = max(1, Lf/PER) threads holding PER (or Lf) values
// each (PER = 32, or 16 where R1, R2 <= 16).  Pass 1: for j < R2, DFT_R1 over in[j + r R2], written to
// tmp[j R1 + r].  Pass 2: for j < R1, twiddle tmp[j + r R1] by
// W_Lf^{j r}, DFT_R2, result is element j + r R1.  The shared buffer pads one
// value per R1 (index x -> x + x / R1) so both passes are bank-conflict free.
template <int LOGL, int PER = 32>
struct Team {
  static constexpr int L = 1 << LOGL;
  static constexpr int R1 = 1 << ((LOGL + 1) / 2);
  static constexpr int R2 = L / R1;
  static constexpr int TT = L >= PER ? L / PER : 1;
  static constexpr int J1 = R2 / TT;    // pass-1 sub-transforms per thread
  static constexpr int J2 = R1 / TT;    // pass-2 sub-transforms per thread
  static constexpr int HELD = J2 * R2;  // values held after pass 2
  static constexpr int BUF = L + R2 + 1;  // padded buffer length (complex), odd
  __device__ __forceinline__ static int pad1(int j, int r) { return j * (R1 + 1) + r; }
  __device__ __forceinline__ static int pad2(int j, int r) { return j + r * (R1 + 1); }
};

// Pass 1 on values already in registers: v[i][r] is input element
// tt + TT i + r R2 (overwritten by the transform).
template <int LOGL, int SIGN, int PER = 32>
__device__ __forceinline__ void team_pass1_regs(int tt, float2* __restrict__ buf,
                                                float2 (&v)[Team<LOGL, PER>::J1][Team<LOGL, PER>::R1]) {
  using T = Team<LOGL, PER>;
#pragma unroll
  for (int i = 0; i < T::J1; ++i) {
    const int j = tt + T::TT * i;
    dft_reg<T::R1, SIGN>(v[i]);
#pragma unroll
    for (int r = 0; r < T::R1; ++r) buf[T::pad1(j, r)] = v[i][r];
  }
}

// Pass 1: LOAD(idx) gives input element idx (0 <= idx < L).  All of the
// thread's loads are issued before the first DFT so that they are in flight
// together.
template <int LOGL, int SIGN, int PER = 32, class Load>
__device__ __forceinline__ void team_pass1(int tt, float2* __restrict__ buf, Load load) {
  using T = Team<LOGL, PER>;
  float2 v[T::J1][T::R1];
#pragma unroll
  for (int i = 0; i < T::J1; ++i)
#pragma unroll
    for (int r = 0; r < T::R1; ++r) v[i][r] = load(tt + T::TT * i + r * T::R2);
  team_pass1_regs<LOGL, SIGN, PER>(tt, buf, v);
}

// Pass 2 (read half): twiddled, transformed values into res[i * R2 + r] for
// element (tt + TT i) + r R1.  TW(j, r) returns exp(SIGN 2 pi i j r / Lf).
template <int LOGL, int SIGN, int PER = 32, class Tw>
__device__ __forceinline__ void team_pass2(int tt, const float2* __restrict__ buf, Tw tw,
                                           float2* __restrict__ res) {
  using T = Team<LOGL, PER>;
#pragma unroll
  for (int i = 0; i < T::J2; ++i) {
    const int j = tt + T::TT * i;
    float2 v[T::R2];
#pragma unroll
    for (int r = 0; r < T::R2; ++r) {
      float2 x = buf[T::pad2(j, r)];
      if (r > 0) x = c_mul(x, tw(j, r));
      v[r] = x;
    }
    dft_reg<T::R2, SIGN>(v);
#pragma unroll
    for (int r = 0; r < T::R2; ++r) res[i * T::R2 + r] = v[r];
  }
}

// Shared-memory copy of the two-level table exp(-2 pi i t / 2N).
struct SmemTwiddles {
  const float2* lo;
  const float2* hi;
  int lb;
  __device__ __forceinline__ float2 operator()(uint32_t t) const {
    return c_mul(lo[t & ((1u << lb) - 1u)], hi[t >> lb]);
  }
};

// ------------------------------------------- three-pass Stockham (team) ---
// Lengths 2^11 and 2^12 (radices 16, 16, 8 or 16): a team of L/32 threads,
// 32 values each, spanning several warps.  Pass p reads in(j + r L/R) for
// its j values, twiddles by W_{Ns R}^{(j mod Ns) r} (Ns = product of the
// earlier radices), transforms and writes out((j/Ns) Ns R + (j mod Ns) + r Ns).
// `sync()` runs between the reads and the writes of a pass so that a pass can
// read and write the same buffer.
template <int LOGL>
struct Team3 {
  static constexpr int L = 1 << LOGL;
  static constexpr int R0 = 16, R1 = 16, R2 = L / 256;
  static constexpr int TT = L / 32;
  static constexpr int BUF = L + 1;  // odd length (bank spread between channels)
};

template <int L, int R, int NS, int SIGN, int TT, class In, class Tw, class Sync, class Out>
__device__ __forceinline__ void stockham_pass(int tt, In in, Tw tw, Sync sync, Out out) {
  constexpr int J = (L / R) / TT;
  float2 v[J][R];
#pragma unroll
  for (int i = 0; i < J; ++i)
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = in(tt + TT * i + r * (L / R));
  sync();
#pragma unroll
  for (int i = 0; i < J; ++i) {
    const int j = tt + TT * i;
    const int jm = j % NS;
    if (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[i][r] = c_mul(v[i][r], tw(jm * r, NS * R));
    }
    dft_reg<R, SIGN>(v[i]);
    const int o = (j / NS) * NS * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) out(o + r * NS, v[i][r]);
  }
}

// Element index of res[i * R2 + r] after team_pass2.
template <int LOGL, int PER = 32>
__device__ __forceinline__ int team_out_index(int tt, int i, int r) {
  using T = Team<LOGL, PER>;
  return tt + T::TT * i + r * T::R1;
}

}  // namespace slicq
