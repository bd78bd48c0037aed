// dgw_energy_static: the discrete energy for callers that cannot allocate
// device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- a host framework that owns all device memory through its own
// pool allocator (calling cudaMalloc behind its back breaks its accounting
// and can fail under its memory cap), a solver loop that was set up once and
// must not allocate in its steady state, or a caller that only holds device
// pointers handed over by another library.  Such a caller passes every input
// and the output as its own device memory; the reduction's only scratch, one
// partial sum per thread block, lives in a fixed file-scope __device__ array
// that is part of the loaded module.
//
// Limits and sharing: the array holds kStaticPartials partial sums, one per
// block of kStaticChunk elements, so nel is capped at
// DGW_ENERGY_STATIC_MAX_ELEMENTS (checked before any launch).  Every call
// shares the one array and leaves its partial sums in it; each call writes
// every slot it later reads, so nothing needs clearing, but two calls whose
// kernels overlap on the GPU (different streams without ordering) race on it.
// The array costs 512 KB on every device that loads the library, until the
// process exits.
#include <cmath>
#include <mutex>
#include <string>

#include "dgw_internal.cuh"

namespace dgw {
namespace {

constexpr int kStaticChunk = 16;         // elements per block
constexpr int kStaticPartials = DGW_ENERGY_STATIC_MAX_ELEMENTS / kStaticChunk;
constexpr int kStaticThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_partials[kStaticPartials];

// Device address of g_static_partials per device, taken once with that
// device current (the host-side symbol is only a stand-in).
double* g_partials_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

struct StaticRef {
  double D[(kMaxN + 1) * (kMaxN + 1)];
  double w[kMaxN + 1];
};

__device__ __forceinline__ double block_sum_static(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  }
  return s;
}

// One block per kStaticChunk elements: J from the node coordinates (relative to
// the element's first node), then w J u^T Q u summed over the chunk.
template <int N>
__global__ void __launch_bounds__(kStaticThreads)
energy_static_partial(const double* __restrict__ x, const double* __restrict__ u,
                      const double* __restrict__ rho, const double* __restrict__ lam,
                      const double* __restrict__ mu, long long nel, const StaticRef ref,
                      double* __restrict__ partials) {
  constexpr int n = N + 1, Np = n * n * n, nf = n * n;
  __shared__ double Xs[3][Np];
  __shared__ double red[32];
  const size_t T = (size_t)nel * Np;
  double acc = 0.0;
  const long long e_begin = (long long)blockIdx.x * kStaticChunk;
  const long long e_end = e_begin + kStaticChunk < nel ? e_begin + kStaticChunk : nel;
  for (long long e = e_begin; e < e_end; ++e) {
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * Np; i += blockDim.x) Xs[i % 3][i / 3] = x[(size_t)e * Np * 3 + i];
    __syncthreads();
    const double x0 = Xs[0][0], y0 = Xs[1][0], z0 = Xs[2][0];
    const double r = rho[e], l = lam[e], m = mu[e];
    const double i2mu = 1.0 / (2.0 * m), lfac = l / (3.0 * l + 2.0 * m), imu = 1.0 / m;
    for (int node = threadIdx.x; node < Np; node += blockDim.x) {
      const int idx[3] = {node % n, (node / n) % n, node / nf};
      const int stride[3] = {1, n, nf};
      const double c0[3] = {x0, y0, z0};
      double G[3][3];   // G[c][ax] = d X_c / d xi_ax
      for (int ax = 0; ax < 3; ++ax) {
        const int base = node - idx[ax] * stride[ax];
        for (int c = 0; c < 3; ++c) {
          double s = 0.0;
          for (int b = 0; b < n; ++b) s += ref.D[idx[ax] * n + b] * (Xs[c][base + b * stride[ax]] - c0[c]);
          G[c][ax] = s;
        }
      }
      const double J = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                       G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                       G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
      const double wJ = ref.w[idx[0]] * ref.w[idx[1]] * ref.w[idx[2]] * J;
      const size_t g = (size_t)e * Np + node;
      const double v1 = u[g], v2 = u[T + g], v3 = u[2 * T + g];
      const double s1 = u[3 * T + g], s2 = u[4 * T + g], s3 = u[5 * T + g];
      const double s4 = u[6 * T + g], s5 = u[7 * T + g], s6 = u[8 * T + g];
      const double tr = s1 + s2 + s3;
      const double kin = r * (v1 * v1 + v2 * v2 + v3 * v3);
      const double pot = i2mu * (s1 * s1 + s2 * s2 + s3 * s3 - lfac * tr * tr) + imu * (s4 * s4 + s5 * s5 + s6 * s6);
      acc += wJ * (kin + pot);
    }
  }
  const double s = block_sum_static(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kStaticThreads)
energy_static_final(const double* __restrict__ partials, int nparts, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partials[i];
  const double s = block_sum_static(acc, red);
  if (threadIdx.x == 0) *out = 0.5 * s;
}

// Where p lives: -1 not device memory, -2 managed memory (reachable from any
// device), otherwise the ordinal of the device that holds it.
int device_of(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (a.type == cudaMemoryTypeManaged) return -2;
  return a.type == cudaMemoryTypeDevice ? a.device : -1;
}

dgw_status static_fail(dgw_status st, const std::string& msg) {
  set_no_context_error(msg);
  return st;
}

}  // namespace

}  // namespace dgw

extern "C" dgw_status dgw_energy_static(int N, int64_t nel, const double* x, const double* u,
                                        const double* rho, const double* lam, const double* mu,
                                        double* energy_out, void* stream) {
  using namespace dgw;
  if (N < 1 || N > kMaxN) return static_fail(DGW_ERR_ARG, "dgw_energy_static: N outside 1..7");
  if (nel < 1) return static_fail(DGW_ERR_ARG, "dgw_energy_static: nel must be positive");
  if (nel > DGW_ENERGY_STATIC_MAX_ELEMENTS)
    return static_fail(DGW_ERR_ARG, "dgw_energy_static: nel " + std::to_string(nel) +
                                        " exceeds the static scratch limit of " +
                                        std::to_string(DGW_ENERGY_STATIC_MAX_ELEMENTS) + " elements");
  const int Np = (N + 1) * (N + 1) * (N + 1);
  if ((double)nel * Np >= 2147483647.0) return static_fail(DGW_ERR_ARG, "dgw_energy_static: nel*Np must be below 2^31");
  const void* ptrs[] = {x, u, rho, lam, mu, energy_out};
  int where[6];
  for (int i = 0; i < 6; ++i) {
    where[i] = ptrs[i] ? device_of(ptrs[i]) : -1;
    if (where[i] == -1) return static_fail(DGW_ERR_ARG, "dgw_energy_static: every array must be device memory");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return static_fail(DGW_ERR_CUDA, "dgw_energy_static: no current CUDA device");
  for (int i = 0; i < 6; ++i)
    if (where[i] >= 0 && where[i] != dev)
      return static_fail(DGW_ERR_ARG, "dgw_energy_static: an array is on device " + std::to_string(where[i]) +
                                          " but device " + std::to_string(dev) + " is current");
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
      if (e != cudaSuccess)
        return static_fail(DGW_ERR_CUDA, std::string("dgw_energy_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_partials_addr[dev] = static_cast<double*>(p);
    }
    partials = g_partials_addr[dev];
  }
  RefElem R;
  build_ref_elem(N, &R);
  StaticRef ref{};
  for (int i = 0; i < (N + 1) * (N + 1); ++i) ref.D[i] = R.D[i];
  for (int i = 0; i <= N; ++i) ref.w[i] = R.w[i];
  const int blocks = (int)((nel + kStaticChunk - 1) / kStaticChunk);
  cudaStream_t s = (cudaStream_t)stream;
  switch (N) {
#define DGW_ES(NN)                                                                                   \
  case NN:                                                                                           \
    energy_static_partial<NN><<<blocks, kStaticThreads, 0, s>>>(x, u, rho, lam, mu, nel, ref, partials); \
    break;
    DGW_ES(1) DGW_ES(2) DGW_ES(3) DGW_ES(4) DGW_ES(5) DGW_ES(6) DGW_ES(7)
#undef DGW_ES
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    energy_static_final<<<1, kStaticThreads, 0, s>>>(partials, blocks, energy_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return static_fail(DGW_ERR_CUDA, std::string("dgw_energy_static: launch: ") + cudaGetErrorString(e));
  return DGW_OK;
}
