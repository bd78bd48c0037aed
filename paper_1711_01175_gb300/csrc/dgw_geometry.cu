// Mesh geometry on the device (set-up, run once per mesh upload).
//
// Per element, from the node coordinates X(xi):
//   * dX/dxi by the 1-D derivative matrix along each reference axis;
//   * the contravariant metric terms J a^i_k = J d xi_i / d x_k in the
//     conservative curl form  J a^i_n = -[curl_xi (X_l grad_xi X_m)]_i,
//     (n, m, l) cyclic -- with the same D, so sum_i D_i (J a^i_k) = 0 holds
//     to round-off (free-stream preservation on curved elements);
//   * J = det(dX/dxi), 1/J and the mass weights w_i w_j w_k J;
//   * on every face node the scaled outward normal m = n sJ = +-J a^d and the
//     stabilisation blocks P = (B(m)^T B(m))^{1/2} and P^{-1}, where B(m) is
//     the 6x3 strain map of the normal: |A(m)| = diag(P, B P^{-1} B^T).
#include <cmath>

#include "dgw_internal.cuh"

namespace dgw {

namespace {

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (FP64).
__device__ void sym3_eig(double a[3][3], double V[3][3], double lam[3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 32; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-34 * dia) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(tt * tt + 1.0);
        const double s = tt * c;
        for (int k = 0; k < 3; ++k) {           // A <- A J  (columns p, q)
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {           // A <- J^T A (rows p, q)
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {           // V <- V J
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < 3; ++i) lam[i] = a[i][i];
}

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

  // Face stabilisation blocks.
  const size_t ffstride = (size_t)nel * 6 * nf;
  for (int it = t; it < 6 * nf; it += blockDim.x) {
    const int f = it / nf, pf = it % nf;
    const int d = f >> 1;
    const bool hi = f & 1;
    const int fa = pf % n, fb = pf / n, cd = hi ? N : 0;
    const int c0 = d == 0 ? cd : fa;
    const int c1 = d == 0 ? fa : (d == 1 ? cd : fb);
    const int c2 = d == 2 ? cd : fb;
    const int vn = c0 + n * (c1 + n * c2);
    const double sgn = hi ? 1.0 : -1.0;
    const double m0 = sgn * Jas[3 * d + 0][vn], m1 = sgn * Jas[3 * d + 1][vn],
                 m2 = sgn * Jas[3 * d + 2][vn];
    const double mm = m0 * m0 + m1 * m1 + m2 * m2;
    // B^T B = |m|^2 I + m m^T - diag(m^2)
    double C[3][3] = {{mm, m0 * m1, m0 * m2}, {m0 * m1, mm, m1 * m2}, {m0 * m2, m1 * m2, mm}};
    double V[3][3], lam[3];
    sym3_eig(C, V, lam);
    double sq[3], isq[3];
    for (int k = 0; k < 3; ++k) {
      sq[k] = sqrt(fmax(lam[k], 0.0));
      isq[k] = sq[k] > 0.0 ? 1.0 / sq[k] : 0.0;
    }
    auto entry = [&](const double* s, int i, int j) {
      return V[i][0] * s[0] * V[j][0] + V[i][1] * s[1] * V[j][1] + V[i][2] * s[2] * V[j][2];
    };
    const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
    const size_t fi = (size_t)e * 6 * nf + it;
    for (int c = 0; c < 6; ++c) {
      out.face[c * ffstride + fi] = entry(sq, pairs[c][0], pairs[c][1]);
      out.face[(6 + c) * ffstride + fi] = entry(isq, pairs[c][0], pairs[c][1]);
    }
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
