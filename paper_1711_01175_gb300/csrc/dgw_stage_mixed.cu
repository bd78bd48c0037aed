// Mixed-precision instantiations: volume, flux, lift and Q^{-1} in FP32 on FP32
// geometry; the state is read and the Runge-Kutta registers updated in FP64.
#include "dgw_stage.cuh"

namespace dgw {

cudaError_t launch_stage_mixed(int N, bool lsrk, const StageParams& p, cudaStream_t s) {
  return launch_stage_any<float>(N, lsrk, p, s);
}

cudaError_t launch_stage_batch_mixed(int N, const BatchLaunch& L, const BatchSet& S, int grid, cudaStream_t s) {
  return launch_stage_batch_any<float>(N, L, S, grid, s);
}

cudaError_t prepare_stage_batch_mixed(int N) {
  return prepare_stage_batch_any<float>(N);
}

}  // namespace dgw
