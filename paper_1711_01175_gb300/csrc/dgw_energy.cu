// Discrete energy E = 1/2 sum_K sum_nodes w J u^T Q u, Q = diag(rho I, C_V^{-1}).
//
// The isotropic compliance in Voigt form gives
//   sigma^T C_V^{-1} sigma = (1/(2 mu)) [sum_i s_ii^2 - lam/(3 lam + 2 mu) (tr s)^2]
//                            + (1/mu) (s23^2 + s13^2 + s12^2),
// the energy of the local solvers' energy identities (the paper's Section 4
// proofs use the same quadratic form with the time weight).  FP64 throughout;
// fixed grid and fixed reduction order, so the value is bit-reproducible.
#include "dgw_internal.cuh"

namespace dgw {

namespace {

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  }
  return s;   // valid in thread 0
}

template <int Np>
__global__ void __launch_bounds__(kEnergyThreads)
energy_partial_kernel(const double* __restrict__ u, const double* __restrict__ wJ,
                      const double* __restrict__ ec, long long nel, double* partials) {
  __shared__ double red[32];
  const unsigned total = (unsigned)(nel * Np);   // nel * Np < 2^31 (checked at upload)
  double acc = 0.0;
  for (unsigned g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const unsigned e = g / Np;
    const double rho = ec[e], i2mu = ec[nel + e], lfac = ec[2 * nel + e], imu = ec[3 * nel + e];
    const size_t T = total;   // field stride; 9 * T may exceed 2^32
    const double v1 = u[g], v2 = u[T + g], v3 = u[2 * T + g];
    const double s1 = u[3 * T + g], s2 = u[4 * T + g], s3 = u[5 * T + g];
    const double s4 = u[6 * T + g], s5 = u[7 * T + g], s6 = u[8 * T + g];
    const double tr = s1 + s2 + s3;
    const double kin = rho * (v1 * v1 + v2 * v2 + v3 * v3);
    const double pot = i2mu * (s1 * s1 + s2 * s2 + s3 * s3 - lfac * tr * tr) +
                       imu * (s4 * s4 + s5 * s5 + s6 * s6);
    acc += wJ[g] * (kin + pot);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kEnergyThreads)
energy_final_kernel(const double* __restrict__ partials, int nparts, double* result) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partials[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) *result = 0.5 * s;
}

// Block b sums partials[b * chunk, min((b + 1) * chunk, n)) into out[b].
__global__ void __launch_bounds__(kEnergyThreads)
energy_chunk_kernel(const double* __restrict__ partials, int nparts, int chunk, double* out) {
  __shared__ double red[32];
  const long long lo = static_cast<long long>(blockIdx.x) * chunk;
  const long long hi = lo + chunk < nparts ? lo + chunk : nparts;
  double acc = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += partials[i];
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

}  // namespace

cudaError_t launch_energy(const double* u, const double* wJ, const double* ec, long long nel, int Np,
                          double* partials, double* result, cudaStream_t s) {
  switch (Np) {
#define DGW_EN(NP)                                                                         \
  case NP:                                                                                 \
    energy_partial_kernel<NP><<<kEnergyBlocks, kEnergyThreads, 0, s>>>(u, wJ, ec, nel, partials); \
    break;
    DGW_EN(8) DGW_EN(27) DGW_EN(64) DGW_EN(125) DGW_EN(216) DGW_EN(343) DGW_EN(512)
#undef DGW_EN
    default:
      return cudaErrorInvalidValue;
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  energy_final_kernel<<<1, kEnergyThreads, 0, s>>>(partials, kEnergyBlocks, result);
  return cudaGetLastError();
}

cudaError_t launch_energy_final(const double* partials, int nparts, double* scratch, double* result,
                                cudaStream_t s) {
  if (nparts <= 8 * kEnergyThreads) {
    energy_final_kernel<<<1, kEnergyThreads, 0, s>>>(partials, nparts, result);
    return cudaGetLastError();
  }
  // Two levels: contiguous chunks per block, then one block over the chunk sums
  // (fixed grid for a given nparts, so the order of the sum is fixed too).
  const int chunk = (nparts + kEnergyBlocks - 1) / kEnergyBlocks;
  const int blocks = (nparts + chunk - 1) / chunk;
  energy_chunk_kernel<<<blocks, kEnergyThreads, 0, s>>>(partials, nparts, chunk, scratch);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  energy_final_kernel<<<1, kEnergyThreads, 0, s>>>(scratch, blocks, result);
  return cudaGetLastError();
}

}  // namespace dgw
