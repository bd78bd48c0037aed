// iHDG-II (the paper's Section 3, Algorithm "The iHDG-II approach") for the
// transport and shallow-water systems: solve sigma u - L(u) = b by
// element-local solves,
//     (sigma I - L_K^self) u_K^{k+1} = b_K + L_K^nbr(u^k),
// where the weighted trace of eq. iHDGtrace takes the element's own unknowns
// at k+1 and its neighbours' at k.  With the upwind flux the neighbour
// coupling of a face node is the m x m matrix
//     C = -(1/(w_0 J)) 1/2 (A(m) - tau S(m)),   m = n sJ outward,
// applied to (u^+)^k: for transport the scalar -(1/(w_0 J)) 1/2 (beta.m -
// tau |beta.m|), non-zero on inflow faces only.
//
// Set-up (dgw_ihdg_setup): L_K^self column by column from the transport stage
// kernel in its self-only mode (neighbour states zero) applied to the unit
// vector of node j in every element; sigma I - L_K^self is inverted per
// element by Gauss-Jordan elimination with partial pivoting in shared memory
// (one CTA per element) and stored transposed, so that the matrix-vector
// product of an iteration reads it coalesced.  Iteration (dgw_ihdg_solve): one
// CTA per element gathers the neighbour terms, applies the inverse, writes
// u^{k+1} and a partial sum of w J (u^{k+1} - u^k)^2; the host stops on the
// paper's criterion ||u^k - u^{k-1}||_{L2} < tol (eq. tolerancecriteriarelerror).
#include <cmath>
#include <string>
#include <vector>

#include "dgw_internal.cuh"

namespace dgw {
namespace {

// Degrees built: transport N <= 4, shallow water N <= 3.  A local block of
// m Np rows is inverted in shared memory up to 125 x 125 (122 KB) and in its
// own global-memory block beyond (shallow water N = 3: 192 rows, 295 KB; the
// blocks of the CTAs in flight stay in L2).  Shallow water at N = 4 (375 rows,
// 1.1 MB per block) would stream every block through HBM once per pivot.
constexpr int kIhdgMaxNTransport = 4;
constexpr int kIhdgMaxNShallow = 3;
constexpr int kIhdgMaxNElastic = 3;     // 9 Np = 576 rows at N = 3 (2.65 MB per block)
constexpr int kIhdgSmemRows = 125;

// Unit vector of (field q, node j) in every element of an [m][nel][Np] state
// (color == nullptr), or in the elements whose colour is `colour`.
__global__ void unit_column_kernel(double* u, long long nodes, int Np, int m, int q, int j, const int* color,
                                   int colour) {
  const long long total = nodes * m;
  for (long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long rem = g % nodes;
    const bool mine = color == nullptr || color[rem / Np] == colour;
    u[g] = (g / nodes == q && rem % Np == j && mine) ? 1.0 : 0.0;
  }
}

// Column (q, j) of every block (color == nullptr) or of the blocks of colour
// `colour`: A[e][(p, i)][(q, j)] = sigma delta - col[p][e][i] (row-major
// blocks of n = m Np, rows and columns field-major).
__global__ void scatter_column_kernel(const double* col, double* A, long long nodes, int Np, int m, int qj,
                                      double sigma, const int* color, int colour) {
  const int n = m * Np;
  const long long total = nodes * m;
  for (long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int p = static_cast<int>(g / nodes);
    const long long rem = g - static_cast<long long>(p) * nodes;
    const long long e = rem / Np;
    if (color != nullptr && color[e] != colour) continue;
    const int row = p * Np + static_cast<int>(rem - e * Np);
    A[(e * n + row) * n + qj] = (row == qj ? sigma : 0.0) - col[g];
  }
}

// In-place Gauss-Jordan inversion of each n x n block of A (partial pivoting;
// row exchanges recorded and undone as column exchanges at the end), written
// back transposed.  SMEM: the block is worked on in shared memory, else in
// place in global memory.  A zero pivot sets *singular.
template <bool SMEM>
__global__ void __launch_bounds__(256) gj_invert_kernel(double* A, int n, long long nel, int* singular) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long e = blockIdx.x;
  if (e >= nel) return;
  double* Ae = A + static_cast<size_t>(e) * n * n;
  double* a = SMEM ? reinterpret_cast<double*>(smem_raw) : Ae;                  // [n][n]
  double* fcol = reinterpret_cast<double*>(smem_raw) + (SMEM ? n * n : 0);     // [n]
  int* perm = reinterpret_cast<int*>(fcol + n);                                 // [n]
  __shared__ int piv_row;
  __shared__ double pinv;
  const int t = threadIdx.x, NT = blockDim.x;
  if constexpr (SMEM) {
    for (int q = t; q < n * n; q += NT) a[q] = Ae[q];
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t < 32) {
      // pivot: the largest |a[i][k]|, i >= k (lowest index on ties)
      double best = -1.0;
      int bi = k;
      for (int i = k + t; i < n; i += 32) {
        const double v = fabs(a[i * n + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (t == 0) {
        piv_row = bi;
        perm[k] = bi;
        if (!(best > 0.0)) atomicExch(singular, 1);
      }
    }
    __syncthreads();
    const int p = piv_row;
    if (p != k) {
      for (int j = t; j < n; j += NT) {
        const double tmp = a[k * n + j];
        a[k * n + j] = a[p * n + j];
        a[p * n + j] = tmp;
      }
    }
    __syncthreads();
    if (t == 0) pinv = 1.0 / a[k * n + k];
    __syncthreads();
    for (int j = t; j < n; j += NT) a[k * n + j] = (j == k ? 1.0 : a[k * n + j]) * pinv;
    for (int i = t; i < n; i += NT) fcol[i] = i == k ? 0.0 : a[i * n + k];
    __syncthreads();
    for (int q = t; q < n * n; q += NT) {
      const int i = q / n, j = q - (q / n) * n;
      if (i != k) a[q] = (j == k ? 0.0 : a[q]) - fcol[i] * a[k * n + j];
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      for (int i = t; i < n; i += NT) {
        const double tmp = a[i * n + k];
        a[i * n + k] = a[i * n + p];
        a[i * n + p] = tmp;
      }
    }
    __syncthreads();
  }
  if constexpr (SMEM) {
    for (int q = t; q < n * n; q += NT) {
      const int i = q / n, j = q - (q / n) * n;
      Ae[j * n + i] = a[q];
    }
  } else {
    for (int q = t; q < n * n; q += NT) {            // transpose in place, each pair once
      const int i = q / n, j = q - (q / n) * n;
      if (i < j) {
        const double tmp = a[i * n + j];
        a[i * n + j] = a[j * n + i];
        a[j * n + i] = tmp;
      }
    }
  }
}

// C of every face node of every element (zero on boundary faces), m x m row-major.
template <int N, int M>
__global__ void face_coef_kernel(const double* geo, const int* vmapP, long long nel, double beta0, double beta1,
                                 double beta2, double tau, double w_end_inv, double* cf) {
  constexpr int n = N + 1, Np = n * n * n, nf = n * n;
  const long long total = nel * 6 * nf;
  const size_t fstride = static_cast<size_t>(nel) * Np;
  for (long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long e = g / (6 * nf);
    const int r = static_cast<int>(g - e * 6 * nf);
    double C[M * M];
#pragma unroll
    for (int q = 0; q < M * M; ++q) C[q] = 0.0;
    if (vmapP[g] >= 0) {
      const int f = r / nf, pf = r - (r / nf) * nf, d = f >> 1;
      const bool hi = (f & 1) != 0;
      const int fa = pf % n, fb = pf / n, cd = hi ? N : 0;
      const int c0 = d == 0 ? cd : fa;
      const int c1 = d == 0 ? fa : (d == 1 ? cd : fb);
      const int c2 = d == 2 ? cd : fb;
      const size_t gi = static_cast<size_t>(e) * Np + c0 + n * (c1 + n * c2);
      const double sgn = hi ? 1.0 : -1.0;
      const double m1 = sgn * geo[(3 * d + 0) * fstride + gi];
      const double m2 = sgn * geo[(3 * d + 1) * fstride + gi];
      const double m3 = sgn * geo[(3 * d + 2) * fstride + gi];
      const double s = -0.5 * w_end_inv * geo[9 * fstride + gi];
      if constexpr (M == 1) {
        const double bm = beta0 * m1 + beta1 * m2 + beta2 * m3;
        C[0] = s * (bm - tau * fabs(bm));
      } else {
        // A(m) = [[0, m1, m2], [m1, 0, 0], [m2, 0, 0]];
        // S(m) = [[nu, 0, 0], [0, m1^2/nu, m1 m2/nu], [0, m1 m2/nu, m2^2/nu]], nu = |(m1, m2)|
        const double nu = sqrt(m1 * m1 + m2 * m2);
        const double inu = nu > 0.0 ? 1.0 / nu : 0.0;
        C[0] = -s * tau * nu;
        C[1] = s * m1;
        C[2] = s * m2;
        C[3] = s * m1;
        C[4] = -s * tau * m1 * m1 * inu;
        C[5] = -s * tau * m1 * m2 * inu;
        C[6] = s * m2;
        C[7] = -s * tau * m1 * m2 * inu;
        C[8] = -s * tau * m2 * m2 * inu;
      }
    }
#pragma unroll
    for (int q = 0; q < M * M; ++q) cf[g * M * M + q] = C[q];
  }
}

// One iHDG-II iteration: u_next_K = inv_K (sigma u_prev_K + f_K + sum_faces C u_k^+),
// and part[e] = sum_(p,i) w J (u_next - u_k)^2 over the element.
template <int N, int M>
__global__ void __launch_bounds__((M * (N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
    ihdg_iter_kernel(const double* __restrict__ invT, const double* __restrict__ cf, const int* __restrict__ vmapP,
                     const double* __restrict__ wJ, const double* u_prev, const double* f, double sigma,
                     const double* __restrict__ uk, double* __restrict__ unext, long long nel, double* part) {
  constexpr int n = N + 1, Np = n * n * n, nf = n * n, NB = M * Np, NT = (NB + 31) / 32 * 32;
  __shared__ double rhs_s[NB];
  __shared__ double x_s[6 * nf * M];
  __shared__ double red[32];
  const long long e = blockIdx.x;
  const int t = threadIdx.x;
  const size_t fstride = static_cast<size_t>(nel) * Np;
  for (int r = t; r < 6 * nf; r += NT) {
    const size_t gr = static_cast<size_t>(e) * 6 * nf + r;
    const int g = vmapP[gr];
#pragma unroll
    for (int p = 0; p < M; ++p) {
      double x = 0.0;
      if (g >= 0) {
#pragma unroll
        for (int q = 0; q < M; ++q) x += cf[gr * M * M + p * M + q] * uk[q * fstride + g];
      }
      x_s[r * M + p] = x;
    }
  }
  __syncthreads();
  const int p = t / Np, i = t - (t / Np) * Np;
  const size_t gi = p * fstride + static_cast<size_t>(e) * Np + i;
  if (t < NB) {
    double rhs = (u_prev ? sigma * u_prev[gi] : 0.0) + (f ? f[gi] : 0.0);
    const int ix = i % n, iy = (i / n) % n, iz = i / nf;
    if (ix == 0) rhs += x_s[(0 * nf + iy + n * iz) * M + p];
    if (ix == N) rhs += x_s[(1 * nf + iy + n * iz) * M + p];
    if (iy == 0) rhs += x_s[(2 * nf + ix + n * iz) * M + p];
    if (iy == N) rhs += x_s[(3 * nf + ix + n * iz) * M + p];
    if (iz == 0) rhs += x_s[(4 * nf + ix + n * iy) * M + p];
    if (iz == N) rhs += x_s[(5 * nf + ix + n * iy) * M + p];
    rhs_s[t] = rhs;
  }
  __syncthreads();
  double v = 0.0;
  if (t < NB) {
    const double* Mt = invT + static_cast<size_t>(e) * NB * NB + t;
    double acc = 0.0;
#pragma unroll 3
    for (int j = 0; j < NB; ++j) acc = fma(Mt[static_cast<size_t>(j) * NB], rhs_s[j], acc);
    unext[gi] = acc;
    const double d = acc - uk[gi];
    v = wJ[static_cast<size_t>(e) * Np + i] * d * d;
  }
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    double sum = 0.0;
    for (int w = 0; w < NT / 32; ++w) sum += red[w];
    part[e] = sum;
  }
}

template <int N, int M>
cudaError_t launch_iter(const dgw_ctx* c, const double* u_prev, const double* f, const double* uk, double* unext,
                        cudaStream_t s) {
  constexpr int NB = M * (N + 1) * (N + 1) * (N + 1), NT = (NB + 31) / 32 * 32;
  ihdg_iter_kernel<N, M><<<(unsigned)c->nel, NT, 0, s>>>(c->ihdg_inv, c->ihdg_cf, c->vmapP, c->wJ, u_prev, f,
                                                          c->ihdg_sigma, uk, unext, c->nel, c->ihdg_part);
  return cudaGetLastError();
}

cudaError_t launch_iter_any(const dgw_ctx* c, const double* u_prev, const double* f, const double* uk, double* unext,
                            cudaStream_t s) {
  if (c->cfg.system == DGW_SYSTEM_SHALLOW_WATER) {
    switch (c->cfg.N) {
      case 1: return launch_iter<1, 3>(c, u_prev, f, uk, unext, s);
      case 2: return launch_iter<2, 3>(c, u_prev, f, uk, unext, s);
      case 3: return launch_iter<3, 3>(c, u_prev, f, uk, unext, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (c->cfg.N) {
    case 1: return launch_iter<1, 1>(c, u_prev, f, uk, unext, s);
    case 2: return launch_iter<2, 1>(c, u_prev, f, uk, unext, s);
    case 3: return launch_iter<3, 1>(c, u_prev, f, uk, unext, s);
    case 4: return launch_iter<4, 1>(c, u_prev, f, uk, unext, s);
    default: return cudaErrorInvalidValue;
  }
}

// One iHDG-II iteration in residual form (the elastic system): with
// r = sigma u_prev + f + L(u^k) - sigma u^k, u^{k+1}_K = u^k_K + inv_K r_K.  As
// L(u)_K = L_K^self u^k_K + L_K^nbr(u^k), r_K = b_K + L_K^nbr(u^k) - (sigma I -
// L_K^self) u^k_K, so this is the local solve of eq. iHDGlocal; the neighbour
// terms come from the full operator (Lu = L(u^k)) instead of per-face
// coefficients.  part[e] = sum_(p,i) w J (u^{k+1} - u^k)^2 over the element.
template <int N, int M>
__global__ void __launch_bounds__((M * (N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
    ihdg_resid_kernel(const double* __restrict__ invT, const double* __restrict__ Lu, const double* __restrict__ wJ,
                      const double* u_prev, const double* f, double sigma, const double* __restrict__ uk,
                      double* __restrict__ unext, long long nel, double* part) {
  constexpr int n = N + 1, Np = n * n * n, NB = M * Np, NT = (NB + 31) / 32 * 32;
  __shared__ double r_s[NB];
  __shared__ double red[32];
  const long long e = blockIdx.x;
  const int t = threadIdx.x;
  const size_t fstride = static_cast<size_t>(nel) * Np;
  const int p = t / Np, i = t - (t / Np) * Np;
  const size_t gi = p * fstride + static_cast<size_t>(e) * Np + i;
  double ukv = 0.0;
  if (t < NB) {
    ukv = uk[gi];
    r_s[t] = (u_prev ? sigma * u_prev[gi] : 0.0) + (f ? f[gi] : 0.0) + Lu[gi] - sigma * ukv;
  }
  __syncthreads();
  double v = 0.0;
  if (t < NB) {
    const double* Mt = invT + static_cast<size_t>(e) * NB * NB + t;
    double acc = 0.0;
#pragma unroll 3
    for (int j = 0; j < NB; ++j) acc = fma(Mt[static_cast<size_t>(j) * NB], r_s[j], acc);
    const double un = ukv + acc;
    unext[gi] = un;
    const double d = un - ukv;
    v = wJ[static_cast<size_t>(e) * Np + i] * d * d;
  }
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    double sum = 0.0;
    for (int w = 0; w < NT / 32; ++w) sum += red[w];
    part[e] = sum;
  }
}

cudaError_t launch_resid_any(const dgw_ctx* c, const double* u_prev, const double* f, const double* uk,
                             const double* Lu, double* unext, cudaStream_t s) {
  switch (c->cfg.N) {
#define DGW_RCASE(NN)                                                                                          \
  case NN: {                                                                                                   \
    constexpr int NT = (9 * (NN + 1) * (NN + 1) * (NN + 1) + 31) / 32 * 32;                                    \
    ihdg_resid_kernel<NN, 9><<<(unsigned)c->nel, NT, 0, s>>>(c->ihdg_inv, Lu, c->wJ, u_prev, f, c->ihdg_sigma, uk, \
                                                              unext, c->nel, c->ihdg_part);                    \
    return cudaGetLastError();                                                                                 \
  }
    DGW_RCASE(1) DGW_RCASE(2) DGW_RCASE(3)
#undef DGW_RCASE
    default:
      return cudaErrorInvalidValue;
  }
}

// L(u) of an FP64 elastic context without the point force (the operator of
// sigma u - L(u) = b; a source enters through f).
cudaError_t launch_elastic_operator(const dgw_ctx* c, const double* u, double* out, cudaStream_t s) {
  StageParams p{};
  int epb = 0, nthreads = 0;
  stage_shape(c->cfg.N, &epb, &nthreads);
  p.pf_elems = 1LL * c->sm_count * epb;
  p.src_elem = -1;
  p.u_in = u;
  p.out = out;
  p.geo = c->geo;
  p.fz = c->fz;
  p.vmapP = c->vmapP;
  p.mat = c->mat;
  p.nel = c->nel;
  p.tau = c->cfg.flux_tau ? 1.0 : 0.0;
  p.w_end_inv = 1.0 / c->ref.w[0];
  for (int i = 0; i < (c->cfg.N + 1) * (c->cfg.N + 1); ++i) p.D[i] = c->ref.D[i];
  return launch_stage_fp64(c->cfg.N, false, p, s);
}

// Greedy colouring of the element graph (elements sharing an interior face get
// different colours).  Returns the number of colours, or -1 if an element is its
// own neighbour (no colouring then separates its own values from its neighbour's).
int color_elements(const dgw_ctx* c, std::vector<int>& color) {
  const long long nel = c->nel;
  color.assign(static_cast<size_t>(nel), -1);
  int ncol = 0;
  for (long long e = 0; e < nel; ++e) {
    unsigned long long used = 0;
    for (int f = 0; f < 6; ++f) {
      const size_t k = static_cast<size_t>(e) * 6 + f;
      const long long nb = c->etoe[k];
      if (nb < 0 || c->bc[k] != DGW_BC_INTERIOR) continue;
      if (nb == e) return -1;
      if (color[nb] >= 0 && color[nb] < 64) used |= 1ull << color[nb];
    }
    int col = 0;
    while (col < 64 && ((used >> col) & 1ull)) ++col;
    color[e] = col;
    if (col + 1 > ncol) ncol = col + 1;
  }
  return ncol;
}

cudaError_t launch_face_coef(const dgw_ctx* c, cudaStream_t s) {
  const double* geo = static_cast<const double*>(c->geo);
  const double tau = c->cfg.flux_tau ? 1.0 : 0.0;
  const double wi = 1.0 / c->ref.w[0];
  const double* b = c->cfg.beta;
  const int blocks = 4 * c->sm_count;
  const bool sw = c->cfg.system == DGW_SYSTEM_SHALLOW_WATER;
  switch (c->cfg.N * 2 + (sw ? 1 : 0)) {
#define DGW_FC(NN, MM, KEY)                                                                                     \
  case KEY:                                                                                                     \
    face_coef_kernel<NN, MM><<<blocks, 256, 0, s>>>(geo, c->vmapP, c->nel, b[0], b[1], b[2], tau, wi, c->ihdg_cf); \
    break;
    DGW_FC(1, 1, 2) DGW_FC(2, 1, 4) DGW_FC(3, 1, 6) DGW_FC(4, 1, 8) DGW_FC(1, 3, 3) DGW_FC(2, 3, 5)
    DGW_FC(3, 3, 7)
#undef DGW_FC
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

dgw_status ifail(dgw_ctx* c, dgw_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    set_no_context_error(msg);
  return st;
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void ihdg_free(dgw_ctx* c) {
  if (c->ihdg_inv) cudaFree(c->ihdg_inv);
  if (c->ihdg_cf) cudaFree(c->ihdg_cf);
  if (c->ihdg_part) cudaFree(c->ihdg_part);
  if (c->ihdg_u2) cudaFree(c->ihdg_u2);
  c->ihdg_inv = c->ihdg_cf = c->ihdg_part = c->ihdg_u2 = nullptr;
  c->ihdg_ready = false;
}

}  // namespace

void ihdg_release(dgw_ctx* c) { ihdg_free(c); }

}  // namespace dgw

#define ICUDA(call, what)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return dgw::ifail(c, DGW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" {

dgw_status dgw_ihdg_setup(dgw_ctx* c, double sigma, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_ihdg_setup");
  if (!c) return dgw::ifail(nullptr, DGW_ERR_ARG, "null context");
  const bool elastic = c->cfg.system == DGW_SYSTEM_ELASTIC;
  if (elastic && c->cfg.precision != DGW_PRECISION_FP64)
    return dgw::ifail(c, DGW_ERR_UNSUPPORTED, "iHDG-II for the elastic system is built in FP64 only");
  if (elastic && c->cfg.N > dgw::kIhdgMaxNElastic)
    return dgw::ifail(c, DGW_ERR_UNSUPPORTED, "iHDG-II for the elastic system is built for N <= 3");
  if (c->cfg.system == DGW_SYSTEM_TRANSPORT && c->cfg.N > dgw::kIhdgMaxNTransport)
    return dgw::ifail(c, DGW_ERR_UNSUPPORTED, "iHDG-II for transport is built for N <= 4");
  if (c->cfg.system == DGW_SYSTEM_SHALLOW_WATER && c->cfg.N > dgw::kIhdgMaxNShallow)
    return dgw::ifail(c, DGW_ERR_UNSUPPORTED, "iHDG-II for shallow water is built for N <= 3");
  if (!c->has_mesh) return dgw::ifail(c, DGW_ERR_STATE, "iHDG-II set-up before the mesh");
  if (elastic && !c->has_material) return dgw::ifail(c, DGW_ERR_STATE, "iHDG-II set-up before the material");
  std::vector<int> color;
  int ncolors = 0;
  if (elastic) {
    ncolors = dgw::color_elements(c, color);
    if (ncolors < 0)
      return dgw::ifail(c, DGW_ERR_UNSUPPORTED, "iHDG-II for the elastic system: an element is its own neighbour");
  }
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) return dgw::ifail(c, DGW_ERR_ARG, "sigma must be finite and >= 0");
  if (cudaSetDevice(c->device) != cudaSuccess) return dgw::ifail(c, DGW_ERR_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = c->cfg.N, n = N + 1, Np = n * n * n, nf = n * n, m = c->m, nb = m * Np;
  const long long nel = c->nel;
  const size_t nodes = static_cast<size_t>(nel) * Np;
  dgw::ihdg_free(c);
  const size_t inv_bytes = static_cast<size_t>(nel) * nb * nb * sizeof(double);
  if (cudaMalloc(&c->ihdg_inv, inv_bytes) != cudaSuccess ||
      (!elastic &&
       cudaMalloc(&c->ihdg_cf, static_cast<size_t>(nel) * 6 * nf * m * m * sizeof(double)) != cudaSuccess) ||
      cudaMalloc(&c->ihdg_part, (static_cast<size_t>(nel) + 1 + dgw::kEnergyBlocks) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->ihdg_u2, nodes * m * sizeof(double)) != cudaSuccess) {
    dgw::ihdg_free(c);
    return dgw::ifail(c, DGW_ERR_OOM, "iHDG-II buffers (" + std::to_string(inv_bytes >> 20) + " MB of inverses)");
  }
  int* singular = nullptr;
  ICUDA(cudaMalloc(&singular, sizeof(int)), "alloc flag");
  ICUDA(cudaMemsetAsync(singular, 0, sizeof(int), s), "clear flag");
  // Columns of L_K^self: unit vector of node j in every element -> self-only operator.
  dgw::StageParams p{};
  p.u_in = c->ihdg_u2;
  p.out = c->u2;
  p.geo = c->geo;
  p.vmapP = c->vmapP;
  p.nel = nel;
  p.tau = c->cfg.flux_tau ? 1.0 : 0.0;
  p.w_end_inv = 1.0 / c->ref.w[0];
  p.src_elem = -1;
  p.self_only = 1;
  for (int k = 0; k < 3; ++k) p.beta[k] = c->cfg.beta[k];
  for (int i = 0; i < n * n; ++i) p.D[i] = c->ref.D[i];
  const int blocks = 4 * c->sm_count;
  cudaError_t e = cudaSuccess;
  if (elastic) {
    // The elastic operator has no self-only mode: apply it to the unit vector of
    // (field, node) in the elements of one colour at a time.  Their interior
    // neighbours are of other colours, hence zero, and L(u)_K = L_K^self u_K there.
    int* color_d = nullptr;
    e = cudaMalloc(&color_d, color.size() * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(color_d, color.data(), color.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    for (int col = 0; col < ncolors && e == cudaSuccess; ++col) {
      for (int qj = 0; qj < nb && e == cudaSuccess; ++qj) {
        dgw::unit_column_kernel<<<blocks, 256, 0, s>>>(c->ihdg_u2, static_cast<long long>(nodes), Np, m, qj / Np,
                                                        qj % Np, color_d, col);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = dgw::launch_elastic_operator(c, c->ihdg_u2, c->u2, s);
        if (e == cudaSuccess) {
          dgw::scatter_column_kernel<<<blocks, 256, 0, s>>>(c->u2, c->ihdg_inv, static_cast<long long>(nodes), Np, m,
                                                             qj, sigma, color_d, col);
          e = cudaGetLastError();
        }
      }
    }
    if (color_d) {
      const cudaError_t e2 = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = e2;
      cudaFree(color_d);
    }
  }
  for (int qj = 0; qj < nb && e == cudaSuccess && !elastic; ++qj) {
    dgw::unit_column_kernel<<<blocks, 256, 0, s>>>(c->ihdg_u2, static_cast<long long>(nodes), Np, m, qj / Np, qj % Np,
                                                    nullptr, 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = dgw::launch_friedrichs(c->cfg.system, N, false, p, s);
    if (e == cudaSuccess) {
      dgw::scatter_column_kernel<<<blocks, 256, 0, s>>>(c->u2, c->ihdg_inv, static_cast<long long>(nodes), Np, m, qj,
                                                         sigma, nullptr, 0);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) {
    cudaFree(singular);
    return dgw::ifail(c, DGW_ERR_CUDA, std::string("local matrices: ") + cudaGetErrorString(e));
  }
  if (nb <= dgw::kIhdgSmemRows) {
    const size_t smem = static_cast<size_t>(nb) * nb * 8 + nb * 8 + nb * 4;
    e = cudaFuncSetAttribute(dgw::gj_invert_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      dgw::gj_invert_kernel<true><<<(unsigned)nel, 256, smem, s>>>(c->ihdg_inv, nb, nel, singular);
      e = cudaGetLastError();
    }
  } else {
    dgw::gj_invert_kernel<false><<<(unsigned)nel, 256, nb * 8 + nb * 4, s>>>(c->ihdg_inv, nb, nel, singular);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !elastic) e = dgw::launch_face_coef(c, s);
  int sing = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sing, singular, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(singular);
  if (e != cudaSuccess) return dgw::ifail(c, DGW_ERR_CUDA, std::string("local inverses: ") + cudaGetErrorString(e));
  if (sing) {
    dgw::ihdg_free(c);
    return dgw::ifail(c, DGW_ERR_ARG, "a local matrix sigma I - L_K^self is singular");
  }
  c->ihdg_sigma = sigma;
  c->ihdg_ready = true;
  return DGW_OK;
}

dgw_status dgw_ihdg_solve(dgw_ctx* c, const double* u_prev, const double* f, double* u, double tol, int max_iter,
                          int* iterations, double* last_change, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_ihdg_solve");
  if (!c) return dgw::ifail(nullptr, DGW_ERR_ARG, "null context");
  if (!c->ihdg_ready) return dgw::ifail(c, DGW_ERR_STATE, "dgw_ihdg_setup first");
  if (!u || !iterations || max_iter < 1 || !(tol >= 0.0)) return dgw::ifail(c, DGW_ERR_ARG, "bad arguments");
  if (!dgw::dev_ptr(u) || (u_prev && !dgw::dev_ptr(u_prev)) || (f && !dgw::dev_ptr(f)))
    return dgw::ifail(c, DGW_ERR_ARG, "u, u_prev and f must be device buffers");
  if (u_prev == u || f == u) return dgw::ifail(c, DGW_ERR_ARG, "u must not alias u_prev or f");
  if (cudaSetDevice(c->device) != cudaSuccess) return dgw::ifail(c, DGW_ERR_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes =
      static_cast<size_t>(c->nel) * (c->cfg.N + 1) * (c->cfg.N + 1) * (c->cfg.N + 1) * c->m * sizeof(double);
  double* cur = u;
  double* nxt = c->ihdg_u2;
  double* result = c->ihdg_part + c->nel;
  double change = INFINITY;
  int k = 0;
  while (k < max_iter) {
    if (c->cfg.system == DGW_SYSTEM_ELASTIC) {
      ICUDA(dgw::launch_elastic_operator(c, cur, c->u2, s), "operator");
      ICUDA(dgw::launch_resid_any(c, u_prev, f, cur, c->u2, nxt, s), "iteration kernel");
    } else {
      ICUDA(dgw::launch_iter_any(c, u_prev, f, cur, nxt, s), "iteration kernel");
    }
    ICUDA(dgw::launch_energy_final(c->ihdg_part, static_cast<int>(c->nel), result + 1, result, s), "change norm");
    double half_sq = 0.0;
    ICUDA(cudaMemcpyAsync(&half_sq, result, sizeof(double), cudaMemcpyDeviceToHost, s), "copy change");
    ICUDA(cudaStreamSynchronize(s), "iteration");
    ++k;
    double* tmp = cur;
    cur = nxt;
    nxt = tmp;
    change = std::sqrt(2.0 * half_sq);           // the reduction returns half the sum
    if (!std::isfinite(change)) return dgw::ifail(c, DGW_ERR_UNSTABLE, "iHDG-II iterate is not finite");
    if (change < tol) break;
  }
  if (cur != u) ICUDA(cudaMemcpyAsync(u, cur, bytes, cudaMemcpyDeviceToDevice, s), "copy result");
  ICUDA(cudaStreamSynchronize(s), "result");
  *iterations = k;
  if (last_change) *last_change = change;
  return DGW_OK;
}

}  // extern "C"
