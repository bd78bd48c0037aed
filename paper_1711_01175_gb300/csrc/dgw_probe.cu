// Measurement helper: the FP64 fused multiply-add rate of a device, the
// ceiling of the FP64 path (whose stage kernel keeps the FP64 pipe busy).
#include <string>

#include "dgw_internal.cuh"

namespace dgw {
namespace {

constexpr int kProbeChains = 8;       // independent DFMA chains per thread
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;

__global__ void __launch_bounds__(kProbeThreads) fp64_fma_probe(double* out, int iters, double m, double c) {
  double a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace dgw

extern "C" dgw_status dgw_probe_fp64_rate(int device, double* tflops) {
  if (!tflops) {
    dgw::set_no_context_error("dgw_probe_fp64_rate: null output");
    return DGW_ERR_ARG;
  }
  auto cuda_fail = [](const char* what, cudaError_t e) {
    dgw::set_no_context_error(std::string("dgw_probe_fp64_rate: ") + what + ": " + cudaGetErrorString(e));
    return DGW_ERR_CUDA;
  };
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return cuda_fail("multiprocessor count", e);
  const int blocks = sms * dgw::kProbeBlocksPerSm;
  const int iters = 4096;
  double* out = nullptr;
  e = cudaMalloc(&out, (size_t)blocks * dgw::kProbeThreads * sizeof(double));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? DGW_ERR_OOM : cuda_fail("cudaMalloc", e);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {    // a warm-up launch, then the best of three
    cudaEventRecord(t0, 0);
    dgw::fp64_fma_probe<<<blocks, dgw::kProbeThreads>>>(out, iters, 0.9999999, 1e-7);
    cudaEventRecord(t1, 0);
    e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail("probe kernel", e);
  const double fmas = (double)blocks * dgw::kProbeThreads * dgw::kProbeChains * iters;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return DGW_OK;
}
