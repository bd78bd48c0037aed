// FP64 instantiations of the fused stage kernel (every operation in FP64).
#include "dgw_stage.cuh"

namespace dgw {

cudaError_t launch_stage_fp64(int N, bool lsrk, const StageParams& p, cudaStream_t s) {
  return launch_stage_any<double>(N, lsrk, p, s);
}

void stage_shape(int N, int* epb, int* threads) {
  switch (N) {
#define DGW_SHAPE(NN)            \
  case NN:                       \
    *epb = Shape<NN>::EPB;       \
    *threads = Shape<NN>::NT;    \
    return;
    DGW_SHAPE(1) DGW_SHAPE(2) DGW_SHAPE(3) DGW_SHAPE(4) DGW_SHAPE(5) DGW_SHAPE(6) DGW_SHAPE(7)
#undef DGW_SHAPE
    default:
      *epb = 0;
      *threads = 0;
  }
}

cudaError_t launch_stage_adjoint(int N, int mode, const StageParams& p, cudaStream_t s) {
  return launch_stage_adjoint_any(N, mode, p, s);
}

cudaError_t launch_stage_adjgrad(int N, const StageParams& g, const StageParams& a, cudaStream_t s) {
  return launch_stage_adjgrad_any(N, g, a, s);
}

cudaError_t launch_stage_batch_fp64(int N, const BatchLaunch& L, const BatchSet& S, int grid, cudaStream_t s) {
  return launch_stage_batch_any<double>(N, L, S, grid, s);
}

cudaError_t prepare_stage_batch_fp64(int N) {
  return prepare_stage_batch_any<double>(N);
}

}  // namespace dgw
