// Persistent band kernels with the split-precision (BF16 hi + lo)
// tensor-core radix stages (SLICQ_PREC_SPLIT_BF16); see tc_dft.cuh.
#include "band_kernels.cuh"

namespace slicq {

BandKernels band_kernels_split_bf16() {
  return {band_analysis_persistent_kernel<kPrecSplitBF16>, band_synthesis_persistent_kernel<kPrecSplitBF16>};
}

}  // namespace slicq
