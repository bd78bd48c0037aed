// Mesh geometry on the device (set-up, run once per mesh upload).
//
// Per element, from the node coordinates X(xi):
//   * dX/dxi by the 1-D derivative matrix along each reference axis;
//   * the contravariant metric terms J a^i_k = J d xi_i / d x_k in the
//     conservative curl form  J a^i_n = -[curl_xi (X_l grad_xi X_m)]_i,
//     (n, m, l) cyclic -- with the same D, so sum_i D_i (J a^i_k) = 0 holds
//     to round-off (free-stream preservation on curved elements);
//   * J = det(dX/dxi), 1/J and the mass weights w_i w_j w_k J.
// The scaled outward normal of a face node, m = n sJ = +-J a^d, is read from
// the same metric array by the stage kernel.
#include "dgw_internal.cuh"

namespace dgw {

namespace {

template <int N>
__global__ void geometry_kernel(const double* __restrict__ x, long long nel, GeometryOut out,
                                const double* __restrict__ Dg, const double* __restrict__ wg) {
  constexpr int n = N + 1, Np = n * n * n, nf = n * n;
  extern __shared__ __align__(16) unsigned char geo_smem[];
  double(*Xs)[Np] = reinterpret_cast<double(*)[Np]>(geo_smem);          // [3][Np]
  double(*Ws)[Np] = Xs + 3;                                               // [9][Np]: W^{(c)}_k at 3c+k
  double(*Jas)[Np] = Ws + 9;                                              // [9][Np]
  double* Js = reinterpret_cast<double*>(Jas + 9);                        // [Np]
  double* D = Js + Np;                                                    // [n*n]
  double* w = D + n * n;                                                  // [n]
  const long long e = blockIdx.x;
  const int t = threadIdx.x;
  for (int i = t; i < n * n; i += blockDim.x) D[i] = Dg[i];
  for (int i = t; i < n; i += blockDim.x) w[i] = wg[i];
  for (int i = t; i < 3 * Np; i += blockDim.x) Xs[i % 3][i / 3] = x[(size_t)e * Np * 3 + i];
  __syncthreads();
  // Coordinates relative to the element's first node: the discrete metrics are
  // translation invariant in exact arithmetic (D annihilates constants; the
  // discrete curl of c grad X_m vanishes), and rounding stops scaling with |x|/h.
  const double x0 = Xs[0][0], y0 = Xs[1][0], z0 = Xs[2][0];
  __syncthreads();
  for (int i = t; i < Np; i += blockDim.x) {
    Xs[0][i] -= x0;
    Xs[1][i] -= y0;
    Xs[2][i] -= z0;
  }
  __syncthreads();

  const int ix = t % n, iy = (t / n) % n, iz = t / nf;
  const int strides[3] = {1, n, nf};
  const int idx[3] = {ix, iy, iz};
  auto dref = [&](const double* f, int axis) {
    const int base = t - idx[axis] * strides[axis];
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += D[idx[axis] * n + b] * f[base + b * strides[axis]];
    return s;
  };

  double dX[3][3] = {};   // dX[axis][coord]
  if (t < Np) {
    for (int ax = 0; ax < 3; ++ax)
      for (int c = 0; c < 3; ++c) dX[ax][c] = dref(Xs[c], ax);
    for (int c = 0; c < 3; ++c) {
      const int m = (c + 1) % 3, l = (c + 2) % 3;
      for (int k = 0; k < 3; ++k) Ws[3 * c + k][t] = Xs[l][t] * dX[k][m];
    }
  }
  __syncthreads();
  if (t < Np) {
    for (int c = 0; c < 3; ++c) {
      const double* W0 = Ws[3 * c + 0];
      const double* W1 = Ws[3 * c + 1];
      const double* W2 = Ws[3 * c + 2];
      Jas[0 * 3 + c][t] = -(dref(W2, 1) - dref(W1, 2));
      Jas[1 * 3 + c][t] = -(dref(W0, 2) - dref(W2, 0));
      Jas[2 * 3 + c][t] = -(dref(W1, 0) - dref(W0, 1));
    }
    // J = det G, G[c][ax] = dX[ax][c]
    const double g00 = dX[0][0], g01 = dX[1][0], g02 = dX[2][0];
    const double g10 = dX[0][1], g11 = dX[1][1], g12 = dX[2][1];
    const double g20 = dX[0][2], g21 = dX[1][2], g22 = dX[2][2];
    const double J = g00 * (g11 * g22 - g12 * g21) - g01 * (g10 * g22 - g12 * g20) +
                     g02 * (g10 * g21 - g11 * g20);
    Js[t] = J;
    const size_t fstride = (size_t)nel * Np;
    const size_t gi = (size_t)e * Np + t;
    for (int c = 0; c < 9; ++c) out.geo[c * fstride + gi] = Jas[c][t];
    out.geo[9 * fstride + gi] = 1.0 / J;
    out.wJ[gi] = w[ix] * w[iy] * w[iz] * J;
  }
  __syncthreads();
  if (t == 0) {
    double mn = Js[0];
    for (int i = 1; i < Np; ++i) mn = fmin(mn, Js[i]);
    out.minJ[e] = mn;
  }

}

__global__ void to_float_kernel(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

}  // namespace

cudaError_t launch_geometry(int N, const double* x, long long nel, const double* D, const double* w,
                            const GeometryOut& out, cudaStream_t s) {
  if (nel <= 0) return cudaSuccess;
  const int n = N + 1, Np = n * n * n;
  const int threads = ((Np + 31) / 32) * 32;
  const size_t smem = sizeof(double) * (22 * (size_t)Np + n * n + n);
  cudaError_t err = cudaSuccess;
  switch (N) {
#define DGW_GEO(NN)                                                                        \
  case NN:                                                                                 \
    err = cudaFuncSetAttribute(geometry_kernel<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)smem);                                                 \
    if (err != cudaSuccess) return err;                                                    \
    geometry_kernel<NN><<<(unsigned)nel, threads, smem, s>>>(x, nel, out, D, w);           \
    break;
    DGW_GEO(1) DGW_GEO(2) DGW_GEO(3) DGW_GEO(4) DGW_GEO(5) DGW_GEO(6) DGW_GEO(7)
#undef DGW_GEO
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_float(const double* src, float* dst, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  to_float_kernel<<<152 * 8, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace dgw
