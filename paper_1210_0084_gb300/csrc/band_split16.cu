// Persistent band kernels with the split-precision (FP16 hi + lo)
// tensor-core radix stages (SLICQ_PREC_SPLIT_FP16); see tc_dft.cuh.
#include "band_kernels.cuh"

namespace slicq {

BandKernels band_kernels_split_fp16() {
  return {band_analysis_persistent_kernel<kPrecSplitFP16>, band_synthesis_persistent_kernel<kPrecSplitFP16>};
}

}  // namespace slicq
