// Internal plan representation and launcher declarations of libslicq.
// Host and device code of the library include this; it is not installed.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "slicq.h"

namespace slicq {

// Threads of one band-group CTA, and complex values each thread holds.
// 128 threads keep a group's shared memory and registers small enough for
// two CTAs per SM, whose barriers do not wait on each other.
constexpr int kBandThreads = 128;
constexpr int kPerThread = 32;
constexpr int kMaxTwoPassLog2 = 10;  // M_k <= 1024: two register passes of <= 32
constexpr int kMaxBandLog2 = 12;     // M_k <= 4096: three passes (16, 16, <= 16)
constexpr int kMinBandLog2 = 4;   // M_k >= 16
constexpr int kSliceMaxThreads = 256;  // slice kernels: N / (kSlicePer C) <= 256
constexpr int kSlicePer = 32;          // complex values a slice-kernel thread holds
constexpr int64_t kMaxGridY = 65535;
// shared memory (complex values) a band group's synthesis may use for its
// twiddles, team buffers and accumulator layers; a group closes before
// exceeding it
constexpr int kSynSmemBudget = 26624;

// One kept channel k = 0..K+1 on the slice circle Z_{2N} (Sec. 3).
struct BandDesc {
  int32_t j0;        // first support bin, 0 <= j0 < 2N (circular)
  int32_t len;       // |J_k|
  int32_t log2M;     // M_k = 1 << log2M
  int32_t coef_off;  // off_k inside one slice's coefficients
  int32_t win_off;   // offset into the window tables
  int32_t tofs;      // first thread of the band's team inside the group CTA
  int32_t smem_off;  // complex offset of the team's buffer in shared memory
  int32_t dlo, dhi;  // half-spectrum bins the support covers directly (dhi < 0: none)
  int32_t mlo, mhi;  // half-spectrum bins -j for j in the support (mlo > mhi: none)
  // synthesis accumulator layers: bits 0-15 the layer (colour) of the direct
  // bins, bits 16-31 the mirrored-bin layer among the group's mirrored ones
  // (kNoPhase: none).  Channels of one layer touch disjoint bins.
  int32_t phases;
};
constexpr int kNoPhase = 0xFFFF;

// A CTA's worth of consecutive channels for the band kernels.
struct GroupDesc {
  int32_t band_begin, band_end;  // channels [begin, end)
  int32_t acc_lo, acc_hi;        // half-spectrum bins the group touches
  int32_t ex_lo, ex_hi;          // bins only this group touches (the others: patch slots)
  int32_t pad0_, pad1_;
  int32_t log2M;                 // every channel of the group has M = 2^log2M
  int32_t fp_lo, fp_len;         // spectrum block the analysis stages (even bounds)
  int32_t nphases;               // direct layers (bits 0-15), mirrored layers (16-31)
};


// One slice row of a ragged batch: the clip it belongs to and where that
// clip's samples are (uniform batches compute the same from (row / S)).
struct RowDesc {
  int64_t sig_off;   // first sample of the clip in the signal buffer
  int32_t n, L;      // clip length, padded length (multiple of 2N)
  int32_t S, m;      // slices of the clip, this row's slice index
  int64_t tr_base;   // overlap-add slot of the clip's transition 0
};

// Which of the plan's window tables a synthesis launch uses.
enum SynthKind { kSynthInverse = 0, kSynthAdjoint = 1 };

// Launch with programmatic stream serialisation (see pdl_wait in the kernels).
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace slicq

struct slicq_plan {
  slicq_params params;
  int device = 0;
  int K = 0;
  int n_channels = 0;
  int64_t N = 0;          // half slice length
  int64_t coefs_per_slice = 0;
  int logP = 0, logQ = 0; // four-step split of the N-point complex FFT
  int C = 1;              // cluster size of the slice kernels
  int G = 0;              // band groups
  int ovl_total = 0;      // patch slots of one slice: sum over shared bins of their group count
  int band_smem_s = 0;    // dynamic shared memory of band synthesis (bytes)
  int num_sms = 152;      // SMs of the plan's device (grid sizing)
  int slots_a = 152;      // CTAs the persistent band analysis runs (SMs x CTAs per SM)
  int slots_s = 152;      // CTAs the persistent band synthesis runs
  int band_smem_p = 0;    // dynamic shared memory of the persistent band analysis (bytes)
  int n_cta_a = 0;        // CTAs of the persistent band analysis
  int n_cta_s = 0;        // CTAs of the persistent band synthesis
  std::vector<double> cost_a, cost_s;  // estimated cycles per slice of each group
  int slice_smem = 0;     // dynamic shared memory of the slice kernels (bytes)
  int slice_tw_off = 0;   // float2 offset of the twiddle tables in that memory
  int tw_lb = 0;          // log2 of the fine twiddle table length
  int64_t win_total = 0;  // sum_k |J_k|

  std::vector<slicq::BandDesc> bands;
  std::vector<slicq::GroupDesc> groups;
  std::vector<int32_t> slot_base;    // [N+1] patch slot of bin h for group g: slot_base[h] + g (-1: one group)
  std::vector<int4> shared;          // bins of several groups: (h, first slot, group count, 0)
  std::vector<int16_t> thread_band;  // [G][kBandThreads] channel or -1
  std::vector<double> xi, omega;     // Table 1, channels 0..K+1
  std::vector<int64_t> jlo;          // unwrapped first support sample

  // device arena (one allocation)
  void* d_arena = nullptr;
  slicq::BandDesc* d_bands = nullptr;
  slicq::GroupDesc* d_groups = nullptr;
  int32_t* d_slot_base = nullptr;  // slot_base on the device
  int4* d_shared = nullptr;        // shared on the device
  int2* d_half_chan = nullptr;     // [coefs_per_slice / 2]: (off_k, log2 M_k) of each half-coefficient
  int32_t* d_jc = nullptr;         // [K+2] centre bin round(xi_k 2N / xi_s) (transposition)
  int16_t* d_thread_band = nullptr;
  float* d_ga = nullptr;    // g_k / sqrt(2N)
  float* d_gs = nullptr;    // w_k g~_k / sqrt(2N)
  float* d_gadj = nullptr;  // g_k / (2 sqrt(2N))
  float* d_hw = nullptr;    // Tukey transition, M + 1 values
  float* d_h0 = nullptr;    // h_0 over one slice, 2N values
  int2* d_cta_map_a = nullptr;  // persistent band analysis: CTA -> (group, lane)
  int* d_lanes_a = nullptr;     // its lanes (CTAs) per group
  int2* d_cta_map_s = nullptr;  // persistent band synthesis: CTA -> (group, lane)
  int* d_lanes_s = nullptr;     // its lanes (CTAs) per group
  float2* d_tw_lo = nullptr;  // exp(-2 pi i t / 2N), t < 2^tw_lb
  float2* d_tw_hi = nullptr;  // exp(-2 pi i (t << tw_lb) / 2N)
  float2* d_twband = nullptr; // band pass-2 twiddles, per length, [r][j] layout
  float2* d_tw4 = nullptr;    // four-step twiddles exp(-2 pi i q u / N) at [u Q + q]
  float2* d_tw4096 = nullptr; // exp(-2 pi i t / 4096), t < 4096
  int* d_err = nullptr;       // 1 once a split-precision band kernel gave up a tensor-core wait

  // optional kernel timing trace (events around every launch)
  struct Trace {
    bool on = false;
    int n = 0;
    std::vector<cudaEvent_t> ev;  // 2 per slot
    std::vector<int32_t> kid;
  };
  mutable Trace trace;
};

namespace slicq {

// Host layout (no device): fills everything in `pl` above the arena.
slicq_status build_layout(const slicq_params* p, slicq_plan* pl);
// Slice-kernel geometry (cluster size, shared-memory layout) for C CTAs per slice.
void set_slice_cluster(slicq_plan* pl, int C);

// Workspace partition for `rows` slice rows of a ragged batch (S = rows, L unused).
size_t workspace_layout_rows(const slicq_plan* pl, int64_t rows, void* base, struct Workspace* ws);

// Workspace partition for (n_samples, batch).
struct Workspace {
  int64_t S = 0, L = 0;
  int64_t spec_stride = 0;         // complex values per slice spectrum row
  float2* spec = nullptr;          // [batch * S][spec_stride]
  float2* band_patch = nullptr;    // [batch * S][ovl_total]: partial sums of shared bins
  float* ola_patch = nullptr;      // [batch * S][2][M rounded up to 4]: the two sides of each transition
  size_t bytes = 0;
};
size_t workspace_layout(const slicq_plan* pl, int64_t n_samples, int64_t batch,
                        void* base, Workspace* ws);

// Kernel launchers (return cudaGetLastError() of the launch).
cudaError_t launch_slice_forward(const slicq_plan* pl, const float* f,
                                 int64_t n, int64_t batch, const Workspace& ws,
                                 cudaStream_t st, const RowDesc* rows = nullptr);
// Transposition and masking applied to the coefficients a synthesis reads
// (slicq_inverse_modified).
struct SynthModify {
  int shift;          // channel k = 1..K reads channel k - shift
  const float* mask;  // [batch * S][coefs_per_slice] gains, or null
};

// `cycles` (optional, one per CTA): SM clocks each CTA of the persistent
// band kernel took, for the plan's lane calibration.
cudaError_t launch_band_analysis(const slicq_plan* pl, const Workspace& ws,
                                 int64_t batch, float2* coef, cudaStream_t st,
                                 long long* cycles = nullptr);
cudaError_t launch_band_synthesis(const slicq_plan* pl, const float2* coef,
                                  int64_t batch, SynthKind kind,
                                  const Workspace& ws, cudaStream_t st,
                                  long long* cycles = nullptr,
                                  const SynthModify* mod = nullptr);
// CTAs of the persistent band analysis (synthesis) one SM holds at the
// plan's shared-memory sizes.
int band_ctas_per_sm(const slicq_plan* pl, bool synthesis);

// Adds the two partial sums of the bins shared by neighbouring band groups
// (after launch_band_synthesis, before launch_slice_inverse).
cudaError_t launch_band_boundaries(const slicq_plan* pl, int64_t batch, const Workspace& ws,
                                   cudaStream_t st);
cudaError_t launch_slice_inverse(const slicq_plan* pl, int64_t n,
                                 int64_t batch, SynthKind kind,
                                 const Workspace& ws, float* out,
                                 cudaStream_t st, const RowDesc* rows = nullptr);
// sliCQ spectrogram |s^0 + s^1|^2 of coefficients [batch][S][coefs_per_slice].
cudaError_t launch_spectrogram(const slicq_plan* pl, const float2* coef, int64_t S, int64_t batch,
                               float* out, cudaStream_t st);

// Adds the two sides of every transition into the output (after
// launch_slice_inverse).
cudaError_t launch_slice_ola(const slicq_plan* pl, int64_t n, int64_t batch,
                             const Workspace& ws, float* out, cudaStream_t st,
                             const RowDesc* rows = nullptr);

}  // namespace slicq
