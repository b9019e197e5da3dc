// Split-precision tensor-core DFT stages (tcgen05, sm_103a).
//
// A radix-R stage of a band transform (Algorithms 1 and 2, the DFT_{M_k} of
// each channel) maps every sub-vector x (R complex values) to
// y_q = sum_p x_p exp(SIGN 2 pi i p q / R).  With x and y written as real
// rows [Re x_0, Im x_0, Re x_1, ...] this is the product y = x B of a row
// with the real 2R x 2R matrix
//   B[2p][2q] = C,  B[2p+1][2q] = -S,  B[2p][2q+1] = S,  B[2p+1][2q+1] = C,
//   C + iS = exp(SIGN 2 pi i p q / R).
// The 128 threads of a band CTA each hold J sub-vectors (J R = 32), so one
// stage is J products D_i = A_i B of 128 rows by 2R columns: one tcgen05.mma
// tile (M = 128) per sub-vector index i, FP32 accumulators in tensor memory.
//
// Split precision: each row is first scaled by a power of two (exact) so
// that its largest component lies in [1/2, 1), then written as hi + lo with
// hi = round16(x), lo = round16(x - hi) in FP16 or BF16; B likewise.  The
// product keeps the three terms A_hi B_hi + A_hi B_lo + A_lo B_hi (the
// fourth is below the others' rounding), accumulated in FP32.  FP16 pairs
// carry 22 significant bits (about FP32's accuracy); BF16 pairs 16 bits.
// Stages of radix <= 4 multiply only by +-1, +-i and stay in registers.
//
// Operands live in shared memory in the canonical no-swizzle K-major layout:
// 8-row x 16-byte core matrices of 128 contiguous bytes, core matrices
// adjacent along K 128 bytes apart (leading byte offset), 8-row groups
// (K/8) x 128 bytes apart (stride byte offset).
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_common.cuh"

namespace slicq {

enum TcPrecision { kPrecFP32 = 0, kPrecSplitFP16 = 1, kPrecSplitBF16 = 2 };

constexpr int kTcRows = 128;        // MMA M: one row per thread of a band CTA
constexpr int kTcCols = 64;         // TMEM columns: J sub-vectors x 2R fp32 accumulators per row
constexpr int kTcAElems = kTcRows * kTcCols;  // 16-bit elements of one A operand (hi or lo)
// Clock cycles a thread waits for the tensor cores before it gives up (about 1 s).
constexpr long long kTcWaitCycles = 2000000000LL;

// Bytes of the B tables for radix R (hi and lo): 0 for register radices.
__host__ __device__ constexpr int tc_b_bytes(int R) { return R <= 4 ? 0 : 2 * (2 * R) * (2 * R) * 2; }

// Bytes of a band CTA's tensor-core region for band length 2^logM (two-pass
// lengths): A hi and lo, B of both radices (shared when equal), the
// mbarrier and the TMEM address.
__host__ __device__ constexpr int tc_region_bytes(int logM) {
  return 2 * kTcAElems * 2 + tc_b_bytes(1 << ((logM + 1) / 2)) +
         (((logM + 1) / 2) == (logM / 2) ? 0 : tc_b_bytes(1 << (logM / 2))) + 16;
}

// 16-bit element offset of (row, k) in a tile of K columns (canonical layout).
__device__ __forceinline__ int tc_off(int row, int k, int K) {
  return ((row >> 3) * (K >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (no swizzle): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1 in bits 46-48.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B FP16 or
// BF16, both K-major, N = n, M = 128.
template <int PREC>
__device__ __forceinline__ uint32_t tc_idesc(int n) {
  const uint32_t ab = PREC == kPrecSplitBF16 ? 1u : 0u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// true once the mbarrier at `addr` has completed the phase with `parity`,
// false after `limit` SM clocks
__device__ __forceinline__ bool tc_wait(uint32_t addr, uint32_t parity, long long limit = kTcWaitCycles) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];\n"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
        "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
      : "r"(taddr)
      : "memory");
}

// Two values rounded to the 16-bit type, packed (first at the lower address),
// and the two rounded values back in FP32.
template <int PREC>
__device__ __forceinline__ uint32_t tc_pack(float a, float b, float& ra, float& rb) {
  if constexpr (PREC == kPrecSplitBF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 f = __bfloat1622float2(h);
    ra = f.x;
    rb = f.y;
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    ra = f.x;
    rb = f.y;
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}

// The CTA's tensor-core state: shared-memory operands, TMEM columns, the
// mbarrier the MMAs complete and its phase.
struct TcCtx {
  uint16_t* a_hi;
  uint16_t* a_lo;
  const uint16_t* b1;  // radix R1 (pass 1): hi, then lo at + (2 R1)^2
  const uint16_t* b2;  // radix R2 (pass 2)
  uint32_t mbar;       // shared address
  uint32_t tmem;       // TMEM address of column 0, lane 0
  uint32_t phase;
  bool ok;             // false once a wait gave up (the same in every thread)
};

// B (hi at b, lo at b + (2R)^2) of the radix-R DFT with sign SIGN, written
// by the CTA's threads.  cos32/sin32 are the float32 values of cos(2 pi e/32).
template <int R, int SIGN, int PREC>
__device__ __forceinline__ void tc_build_b(uint16_t* b) {
  if constexpr (R > 4) {
    constexpr int K = 2 * R;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
      const int n = e / K, k = e % K;  // B stored K-major: row n (output column), column k (input)
      const int q = n >> 1, p = k >> 1;
      const int ex = (p * q * (32 / R)) & 31;
      const float C = cos32(ex), S = SIGN * sin32(ex);
      const float val = (n & 1) == 0 ? ((k & 1) == 0 ? C : -S) : ((k & 1) == 0 ? S : C);
      float h, dummy;
      const uint32_t hp = tc_pack<PREC>(val, 0.f, h, dummy);
      float l;
      const uint32_t lp = tc_pack<PREC>(val - h, 0.f, l, dummy);
      b[tc_off(n, k, K)] = (uint16_t)(hp & 0xFFFFu);
      b[K * K + tc_off(n, k, K)] = (uint16_t)(lp & 0xFFFFu);
    }
  }
}

// Set-up at kernel start (every thread): carve the region, build B for the
// two radices, initialise the mbarrier, allocate the TMEM columns (warp 0).
// `region` is 16-byte aligned and holds tc_region_bytes(LOGM) bytes.
template <int LOGM, int SIGN, int PREC>
__device__ __forceinline__ TcCtx tc_setup(unsigned char* region) {
  constexpr int R1 = 1 << ((LOGM + 1) / 2), R2 = 1 << (LOGM / 2);
  TcCtx c;
  c.a_hi = reinterpret_cast<uint16_t*>(region);
  c.a_lo = c.a_hi + kTcAElems;
  uint16_t* b1 = c.a_lo + kTcAElems;
  uint16_t* b2 = R1 == R2 ? b1 : b1 + tc_b_bytes(R1) / 2;
  c.b1 = b1;
  c.b2 = b2;
  unsigned char* tail = region + tc_region_bytes(LOGM) - 16;
  c.mbar = smem_addr(tail);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(tail + 8);
  tc_build_b<R1, SIGN, PREC>(b1);
  if (R2 != R1) tc_build_b<R2, SIGN, PREC>(b2);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(c.mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(s_tmem)),
                 "n"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = *s_tmem;
  c.phase = 0;
  c.ok = true;
  return c;
}

// Tear-down at kernel end (every thread): after a failed wait, give the
// MMAs in flight a second bounded wait; then free the TMEM columns.
__device__ __forceinline__ void tc_teardown(TcCtx& c, int* err) {
  if (!c.ok && threadIdx.x == 0) {
    tc_wait(c.mbar, c.phase);
    if (err) atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(c.tmem), "n"(kTcCols) : "memory");
}

// One radix-R stage over the CTA: v[i] (R complex values) <- DFT_R(v[i]) for
// every thread's J sub-vectors.  Collective for R > 4: every thread of the
// CTA calls it (threads without data pass zeros).  Returns false (in every
// thread) if the tensor cores did not finish within the wait limit.
template <int R, int J, int SIGN, int PREC>
__device__ __forceinline__ bool tc_dft(float2 (&v)[J][R], TcCtx& c, const uint16_t* b) {
  if constexpr (R <= 4) {
#pragma unroll
    for (int i = 0; i < J; ++i) dft_reg<R, SIGN>(v[i]);
    return true;
  } else {
    constexpr int K = 2 * R;          // real inputs (and outputs) per sub-vector
    constexpr int TILE = kTcRows * K; // 16-bit elements of one sub-vector's A tile
    static_assert(J * K == kTcCols, "J sub-vectors of radix R fill the TMEM columns");
    const int row = threadIdx.x;
    float unscale[J];
    // 1. scaled hi / lo rows to shared memory, 16 bytes (8 values) at a time
#pragma unroll
    for (int i = 0; i < J; ++i) {
      float m = 0.f;
#pragma unroll
      for (int p = 0; p < R; ++p) m = fmaxf(m, fmaxf(fabsf(v[i][p].x), fabsf(v[i][p].y)));
      int e = ((__float_as_int(m) >> 23) & 0xFF) - 127;  // m in [2^e, 2^(e+1)); zero/subnormal: -127
      e = e < -125 ? -125 : (e > 125 ? 125 : e);
      const float sc = __int_as_float((127 - e - 1) << 23);  // 2^(-e-1)
      unscale[i] = __int_as_float((127 + e + 1) << 23);      // 2^(e+1)
#pragma unroll
      for (int kb = 0; kb < K / 8; ++kb) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const float2 x = v[i][kb * 4 + w];
          const float a = x.x * sc, bb = x.y * sc;
          float ha, hb, la, lb;
          hw[w] = tc_pack<PREC>(a, bb, ha, hb);
          lw[w] = tc_pack<PREC>(a - ha, bb - hb, la, lb);
        }
        const int o = i * TILE + tc_off(row, kb * 8, K);
        *reinterpret_cast<uint4*>(c.a_hi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(c.a_lo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // 2. one thread issues the J x (K/16) x 3 products and commits them
    if (threadIdx.x == 0) {
      const uint32_t idesc = tc_idesc<PREC>(K);
      const uint32_t sbo = (K / 8) * 128;
      const uint32_t ah = smem_addr(c.a_hi), al = smem_addr(c.a_lo);
      const uint32_t bh = smem_addr(b), bl = smem_addr(b + K * K);
#pragma unroll
      for (int i = 0; i < J; ++i) {
        const uint32_t d = c.tmem + (uint32_t)(i * K);
#pragma unroll
        for (int kk = 0; kk < K / 16; ++kk) {
          const uint32_t ao = (uint32_t)(i * TILE * 2 + kk * 256), bo = (uint32_t)(kk * 256);
          tc_mma(d, tc_desc(ah + ao, 128, sbo), tc_desc(bh + bo, 128, sbo), idesc, kk > 0 ? 1u : 0u);
          tc_mma(d, tc_desc(ah + ao, 128, sbo), tc_desc(bl + bo, 128, sbo), idesc, 1u);
          tc_mma(d, tc_desc(al + ao, 128, sbo), tc_desc(bh + bo, 128, sbo), idesc, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(c.mbar)
                   : "memory");
    }
    // 3. thread 0 waits for the products; the barrier hands completion (or
    // failure) to every thread
    const bool failed = threadIdx.x == 0 && !tc_wait(c.mbar, c.phase);
    if (__syncthreads_or(failed)) {
      c.ok = false;
      return false;
    }
    c.phase ^= 1u;
    tc_fence_after();
    // 4. each thread reads its own row (TMEM lane = row) back
    const uint32_t lane_base = (uint32_t)((threadIdx.x & ~31) << 16);
#pragma unroll
    for (int i = 0; i < J; ++i) {
#pragma unroll
      for (int c16 = 0; c16 < K / 16; ++c16) {
        float r[16];
        tc_ld16(c.tmem + lane_base + (uint32_t)(i * K + c16 * 16), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int w = 0; w < 16; ++w) asm volatile("" : "+f"(r[w]));
#pragma unroll
        for (int w = 0; w < 8; ++w) v[i][c16 * 8 + w] = make_float2(r[2 * w] * unscale[i], r[2 * w + 1] * unscale[i]);
      }
    }
    tc_fence_before();
    return true;
  }
}

}  // namespace slicq
