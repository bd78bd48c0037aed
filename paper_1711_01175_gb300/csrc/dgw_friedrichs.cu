// DG stage kernel for the generic Friedrichs systems (FP64): scalar transport
// and the linearized shallow-water system (Phi = 1), Q = I.
//
// Same discretisation as the elastic stage kernel (GLL collocation, split-form
// volume term with curl-form metrics, upwind HDG flux with the trace
// eliminated, diagonal lift, LSRK(5,4) update), with m fields and the
// system's A(m) and stabilisation S(m) = sJ |A(n)| (m = n sJ):
//   transport      A(m) = beta.m,                S(m) = |beta.m|
//   shallow water  A(m)(phi, qx, qy) = (m1 qx + m2 qy, m1 phi, m2 phi),
//                  S(m)(phi, qx, qy) = (nu phi, m1 t, m2 t), nu = |(m1, m2)|,
//                  t = (m1 qx + m2 qy) / nu  (|A(n)| of eigenvalues 0, +-|n_xy|).
// One CTA holds EPB elements; thread t owns node t % Np of element t / Np.
// The state tile stays in FP64 shared memory, so the Runge-Kutta update reads
// u_in from there.
#include <type_traits>

#include "dgw_internal.cuh"

namespace dgw {

namespace {

template <int SYS>
struct FSys;
template <>
struct FSys<DGW_SYSTEM_TRANSPORT> {
  static constexpr int M = 1;
  static __device__ __forceinline__ void A(const double* beta, double m1, double m2, double m3, const double* w,
                                           double* out) {
    out[0] = (beta[0] * m1 + beta[1] * m2 + beta[2] * m3) * w[0];
  }
  static __device__ __forceinline__ void S(const double* beta, double m1, double m2, double m3, const double* d,
                                           double* out) {
    out[0] = fabs(beta[0] * m1 + beta[1] * m2 + beta[2] * m3) * d[0];
  }
};
template <>
struct FSys<DGW_SYSTEM_SHALLOW_WATER> {
  static constexpr int M = 3;
  static __device__ __forceinline__ void A(const double*, double m1, double m2, double, const double* w, double* out) {
    out[0] = m1 * w[1] + m2 * w[2];
    out[1] = m1 * w[0];
    out[2] = m2 * w[0];
  }
  static __device__ __forceinline__ void S(const double*, double m1, double m2, double, const double* d, double* out) {
    const double mm = m1 * m1 + m2 * m2;
    const double inu = mm > 0.0 ? rsqrt(mm) : 0.0;
    const double tq = (m1 * d[1] + m2 * d[2]) * inu;
    out[0] = mm * inu * d[0];
    out[1] = m1 * tq;
    out[2] = m2 * tq;
  }
};

template <int N, int SYS>
struct FSmem {
  using S = Shape<N>;
  static constexpr int M = FSys<SYS>::M;
  static constexpr size_t u_off = 0;                                        // double [M][NTILE]
  static constexpr size_t f_off = u_off + 8 * M * S::NTILE;                 // double [M][NTILE]
  static constexpr size_t g_off = f_off + 8 * M * S::NTILE;                 // double [10][NTILE]
  static constexpr size_t x_off = g_off + 8 * 10 * S::NTILE;                // double [M][NFI]
  static constexpr size_t d_off = x_off + 8 * M * S::NFACE_ITEMS;           // double [n*n]
  static constexpr size_t e_off = d_off + 8 * S::n * S::n;                  // double [32]
  static constexpr size_t bytes = e_off + 8 * 32;
};

template <int N, int SYS, bool LSRK>
__global__ void __launch_bounds__(Shape<N>::NT) friedrichs_stage_kernel(const StageParams p) {
  using S = Shape<N>;
  using L = FSmem<N, SYS>;
  using Y = FSys<SYS>;
  constexpr int M = Y::M;
  constexpr int n = S::n, Np = S::Np, nf = S::nf, EPB = S::EPB, NT = S::NT, NTILE = S::NTILE, NFI = S::NFACE_ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* u_s = reinterpret_cast<double*>(smem_raw + L::u_off);
  double* f_s = reinterpret_cast<double*>(smem_raw + L::f_off);
  double* g_s = reinterpret_cast<double*>(smem_raw + L::g_off);
  double* x_s = reinterpret_cast<double*>(smem_raw + L::x_off);
  double* D_s = reinterpret_cast<double*>(smem_raw + L::d_off);
  double* red_s = reinterpret_cast<double*>(smem_raw + L::e_off);

  const int t = threadIdx.x;
  const long long e0 = static_cast<long long>(blockIdx.x) * EPB;
  const int el = t / Np;
  const int node = t - el * Np;
  const long long e = e0 + el;
  const bool in_tile = t < NTILE;
  const bool active = in_tile && (e < p.nel);
  const size_t fstride = static_cast<size_t>(p.nel) * Np;
  const size_t gidx = active ? static_cast<size_t>(e) * Np + node : 0;
  const double* geo = static_cast<const double*>(p.geo);

  for (int i = t; i < n * n; i += NT) D_s[i] = p.D[i];
  if (in_tile) {
#pragma unroll
    for (int q = 0; q < M; ++q) u_s[q * NTILE + t] = active ? p.u_in[q * fstride + gidx] : 0.0;
#pragma unroll
    for (int c = 0; c < 10; ++c) g_s[c * NTILE + t] = active ? geo[c * fstride + gidx] : 0.0;
  }
  __syncthreads();

  const int ix = node % n;
  const int iy = (node / n) % n;
  const int iz = node / nf;
  double acc[M];
#pragma unroll
  for (int q = 0; q < M; ++q) acc[q] = 0.0;

  // Volume term: acc = sum_i [ D_i (A(Ja^i) u) + A(Ja^i) (D_i u) ];  vol = -1/2 (1/J) acc.
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    double m1 = 0, m2 = 0, m3 = 0;
    if (in_tile) {
      m1 = g_s[(3 * dir + 0) * NTILE + t];
      m2 = g_s[(3 * dir + 1) * NTILE + t];
      m3 = g_s[(3 * dir + 2) * NTILE + t];
      double w[M], F[M];
#pragma unroll
      for (int q = 0; q < M; ++q) w[q] = u_s[q * NTILE + t];
      Y::A(p.beta, m1, m2, m3, w, F);
#pragma unroll
      for (int q = 0; q < M; ++q) f_s[q * NTILE + t] = F[q];
    }
    __syncthreads();
    if (in_tile) {
      const int stride = dir == 0 ? 1 : (dir == 1 ? n : nf);
      const int a = dir == 0 ? ix : (dir == 1 ? iy : iz);
      const int base = t - a * stride;
      double ds[M];
#pragma unroll
      for (int q = 0; q < M; ++q) ds[q] = 0.0;
#pragma unroll
      for (int b = 0; b < n; ++b) {
        const double Dab = D_s[a * n + b];
#pragma unroll
        for (int q = 0; q < M; ++q) {
          acc[q] += Dab * f_s[q * NTILE + base + b * stride];
          ds[q] += Dab * u_s[q * NTILE + base + b * stride];
        }
      }
      double G[M];
      Y::A(p.beta, m1, m2, m3, ds, G);
#pragma unroll
      for (int q = 0; q < M; ++q) acc[q] += G[q];
    }
    __syncthreads();
  }

  // Face items: (1/(w_0 J)) 1/2 (A(m) - tau S(m)) (u^- - u^+),  m = n sJ outward.
  for (int it = t; it < NFI; it += NT) {
    const int eli = it / (6 * nf);
    const int r = it - eli * (6 * nf);
    const long long ei = e0 + eli;
    if (ei >= p.nel) continue;
    const int f = r / nf;
    const int pf = r - f * nf;
    const int d = f >> 1;
    const bool hi = (f & 1) != 0;
    const int fa = pf % n, fb = pf / n;
    const int cd = hi ? N : 0;
    const int c0 = d == 0 ? cd : fa;
    const int c1 = d == 0 ? fa : (d == 1 ? cd : fb);
    const int c2 = d == 2 ? cd : fb;
    const int sidx = eli * Np + c0 + n * (c1 + n * c2);
    const double sgn = hi ? 1.0 : -1.0;
    const double m1 = sgn * g_s[(3 * d + 0) * NTILE + sidx];
    const double m2 = sgn * g_s[(3 * d + 1) * NTILE + sidx];
    const double m3 = sgn * g_s[(3 * d + 2) * NTILE + sidx];
    const double jv = g_s[9 * NTILE + sidx];
    double du[M];
    const int g = p.vmapP[static_cast<size_t>(ei) * 6 * nf + r];
    if (g >= 0) {
#pragma unroll
      for (int q = 0; q < M; ++q) du[q] = u_s[q * NTILE + sidx] - (p.self_only ? 0.0 : p.u_in[q * fstride + g]);
    } else if (g == kGhostFreeSurface) {
      // shallow-water wall: exterior (phi, q - 2 (q.n) n), jump (0, 2 (q.n) n) with n
      // the horizontal part of the normal (the mesh upload refuses this tag for transport)
#pragma unroll
      for (int q = 0; q < M; ++q) du[q] = 0.0;
      if constexpr (M == 3) {
        const double mm = m1 * m1 + m2 * m2;
        const double qn = mm > 0.0 ? 2.0 * (m1 * u_s[NTILE + sidx] + m2 * u_s[2 * NTILE + sidx]) / mm : 0.0;
        du[1] = qn * m1;
        du[2] = qn * m2;
      }
    } else {
#pragma unroll
      for (int q = 0; q < M; ++q) du[q] = u_s[q * NTILE + sidx];
    }
    double Ad[M], Sd[M];
    Y::A(p.beta, m1, m2, m3, du, Ad);
    Y::S(p.beta, m1, m2, m3, du, Sd);
    const double s = 0.5 * p.w_end_inv * jv * (LSRK ? p.dt : 1.0);   // LSRK: dt L(u) directly
#pragma unroll
    for (int q = 0; q < M; ++q) x_s[q * NFI + it] = s * (Ad[q] - p.tau * Sd[q]);
  }
  __syncthreads();

  double e_node = 0.0;
  if (active) {
    double r[M];
    const double hv = -0.5 * g_s[9 * NTILE + t] * (LSRK ? p.dt : 1.0);
#pragma unroll
    for (int q = 0; q < M; ++q) r[q] = hv * acc[q];
    const int fb0 = el * 6 * nf;
    auto add_face = [&](int f, int pidx) {
#pragma unroll
      for (int q = 0; q < M; ++q) r[q] += x_s[q * NFI + fb0 + f * nf + pidx];
    };
    if (ix == 0) add_face(0, iy + n * iz);
    if (ix == N) add_face(1, iy + n * iz);
    if (iy == 0) add_face(2, ix + n * iz);
    if (iy == N) add_face(3, ix + n * iz);
    if (iz == 0) add_face(4, ix + n * iy);
    if (iz == N) add_face(5, ix + n * iy);
    if constexpr (!LSRK) {
#pragma unroll
      for (int q = 0; q < M; ++q) p.out[q * fstride + gidx] = r[q];
    } else {
      const bool first = p.first != 0;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        const double dtr = r[q];                       // dt already applied
        const double rn = first ? dtr : fma(p.a, p.res[q * fstride + gidx], dtr);
        p.res[q * fstride + gidx] = rn;
        const double uo = fma(p.b, rn, u_s[q * NTILE + t]);
        p.out[q * fstride + gidx] = uo;
        e_node += uo * uo;
      }
      if (p.energy_partials != nullptr) e_node *= p.wJ[gidx];
    }
  }
  if constexpr (LSRK) {
    if (p.energy_partials != nullptr) {
      double v = e_node;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if ((t & 31) == 0) red_s[t >> 5] = v;
      __syncthreads();
      if (t < 32) {
        double w2 = t < NT / 32 ? red_s[t] : 0.0;
        for (int off = 16; off > 0; off >>= 1) w2 += __shfl_down_sync(0xffffffffu, w2, off);
        if (t == 0) p.energy_partials[blockIdx.x] = w2;
      }
    }
  }
}

template <int N, int SYS, bool LSRK>
cudaError_t launch_friedrichs_t(const StageParams& p, cudaStream_t s) {
  using S = Shape<N>;
  const size_t smem = FSmem<N, SYS>::bytes;
  cudaError_t err = cudaFuncSetAttribute(friedrichs_stage_kernel<N, SYS, LSRK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const long long blocks = (p.nel + S::EPB - 1) / S::EPB;
  if (blocks <= 0) return cudaSuccess;
  StageParams q = p;
  finish_stage_params(q);
  friedrichs_stage_kernel<N, SYS, LSRK><<<(unsigned)blocks, S::NT, smem, s>>>(q);
  return cudaGetLastError();
}

template <int SYS>
cudaError_t launch_friedrichs_sys(int N, bool lsrk, const StageParams& p, cudaStream_t s) {
  switch (N) {
#define DGW_FCASE(NN) \
  case NN:            \
    return lsrk ? launch_friedrichs_t<NN, SYS, true>(p, s) : launch_friedrichs_t<NN, SYS, false>(p, s);
    DGW_FCASE(1) DGW_FCASE(2) DGW_FCASE(3) DGW_FCASE(4) DGW_FCASE(5) DGW_FCASE(6) DGW_FCASE(7)
#undef DGW_FCASE
    default:
      return cudaErrorInvalidValue;
  }
}

// E partials of a plain (Q = I) m-field state: w J |u|^2 per CTA.
__global__ void __launch_bounds__(kEnergyThreads)
plain_energy_kernel(const double* __restrict__ u, const double* __restrict__ wJ, int m, long long total,
                    double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < m; ++q) {
      const double v = u[static_cast<size_t>(q) * total + g];
      s += v * v;
    }
    acc += wJ[g] * s;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w2 = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) w2 += __shfl_down_sync(0xffffffffu, w2, off);
    if (threadIdx.x == 0) partials[blockIdx.x] = w2;
  }
}

}  // namespace

cudaError_t launch_friedrichs(int system, int N, bool lsrk, const StageParams& p, cudaStream_t s) {
  if (system == DGW_SYSTEM_TRANSPORT) return launch_friedrichs_sys<DGW_SYSTEM_TRANSPORT>(N, lsrk, p, s);
  if (system == DGW_SYSTEM_SHALLOW_WATER) return launch_friedrichs_sys<DGW_SYSTEM_SHALLOW_WATER>(N, lsrk, p, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_plain_energy(const double* u, const double* wJ, int m, long long total, double* partials,
                                double* result, cudaStream_t s) {
  plain_energy_kernel<<<kEnergyBlocks, kEnergyThreads, 0, s>>>(u, wJ, m, total, partials);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_energy_final(partials, kEnergyBlocks, nullptr, result, s);
}

}  // namespace dgw
