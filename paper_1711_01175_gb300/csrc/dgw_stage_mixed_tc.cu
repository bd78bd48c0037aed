// Mixed-precision instantiations with the volume term's derivative contractions
// on the tensor cores: split FP16 (per-row power-of-two scale) or BF16 operands,
// hi*hi + hi*lo + lo*hi accumulated in FP32; the rest as the mixed path.
#include "dgw_stage.cuh"

namespace dgw {

cudaError_t launch_stage_mixed_tc(int N, int fmt, bool lsrk, const StageParams& p, cudaStream_t s) {
  if (fmt == DGW_PRECISION_MIXED_TC_FP16) return launch_stage_any<float, kVolTcFp16>(N, lsrk, p, s);
  if (fmt == DGW_PRECISION_MIXED_TC_BF16) return launch_stage_any<float, kVolTcBf16>(N, lsrk, p, s);
  return cudaErrorInvalidValue;
}

}  // namespace dgw
