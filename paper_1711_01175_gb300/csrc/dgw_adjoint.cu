// Discrete adjoint of the LSRK(5,4) steps, material gradients, receivers.
//
// The stage map of the 2N-storage scheme, (u, res) -> (u + b_s res', res')
// with res' = a_s res + dt L u, has the transpose
//   w = b_s lu + lr;   lu <- lu + dt L^T w;   lr <- a_s w.
// L^T comes from the forward operator: M Q L splits into a part that is skew
// and linear in A_k (split-form volume term, central flux) and a symmetric
// part independent of the sign of A_k (the upwind stabilisation), so
// L^T = (M Q) L_rev (M Q)^{-1} with L_rev the operator for -A_k.  One adjoint
// stage is two launches: the weight preparation (w, z = (M Q)^{-1} w,
// lr <- a_s w), then one kernel that on each tile computes the gradient terms
// dt w^T (dL/dm) u_{s-1} on the recomputed stage input (GRAD mode) and adds
// dt M Q L_rev z (ADJ mode).
// The material enters L through Q^{-1} (per element) and through the face
// impedances of the stabilisation (face-averaged medium); the second part is
// accumulated per face node and chained to (rho, lambda, mu) at the end.
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "dgw_internal.cuh"

namespace dgw {
namespace {

// w = b lu + lr;  z = (M Q)^{-1} w;  lr <- a w.  mat = [1/rho, lam, mu] (FP64).
__global__ void adjoint_prep_kernel(const double* __restrict__ lu, double* __restrict__ lr, double* __restrict__ W,
                                    double* __restrict__ Z, const double* __restrict__ mat,
                                    const double* __restrict__ wJ, long long nel, int Np, double a, double b) {
  const size_t total = (size_t)nel * Np;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const long long e = (long long)(g / Np);
    const double irho = mat[e], lam = mat[nel + e], mu = mat[2 * nel + e];
    const double iwj = 1.0 / wJ[g];
    double w[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      w[q] = b * lu[q * total + g] + lr[q * total + g];
      W[q * total + g] = w[q];
      lr[q * total + g] = a * w[q];
    }
    const double tr = w[3] + w[4] + w[5];
    Z[g] = irho * w[0] * iwj;
    Z[total + g] = irho * w[1] * iwj;
    Z[2 * total + g] = irho * w[2] * iwj;
    Z[3 * total + g] = (lam * tr + 2.0 * mu * w[3]) * iwj;
    Z[4 * total + g] = (lam * tr + 2.0 * mu * w[4]) * iwj;
    Z[5 * total + g] = (lam * tr + 2.0 * mu * w[5]) * iwj;
    Z[6 * total + g] = mu * w[6] * iwj;
    Z[7 * total + g] = mu * w[7] * iwj;
    Z[8 * total + g] = mu * w[8] * iwj;
  }
}

// Face impedance terms -> (rho, lambda, mu).  Each face's impedances use the
// average of the two sides' medium (the element's own on boundary faces), so
// both sides' face-node terms contribute, with weight 1/2, to each side.
__global__ void adjoint_chain_kernel(const double* __restrict__ gface, const long long* __restrict__ etoe,
                                     const signed char* __restrict__ etof, const double* __restrict__ mat,
                                     long long nel, int nf, double* __restrict__ grad) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const size_t fs = (size_t)nel * 6 * nf;
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int f = 0; f < 6; ++f) {
    const long long e2 = etoe[e * 6 + f];
    const bool interior = e2 >= 0;
    double gzs = 0.0, gzp = 0.0;
    for (int k = 0; k < nf; ++k) {
      gzs += gface[((size_t)e * 6 + f) * nf + k];
      gzp += gface[fs + ((size_t)e * 6 + f) * nf + k];
    }
    const long long o = interior ? e2 : e;
    if (interior) {
      const int f2 = etof[e * 6 + f];
      for (int k = 0; k < nf; ++k) {
        gzs += gface[((size_t)e2 * 6 + f2) * nf + k];
        gzp += gface[fs + ((size_t)e2 * 6 + f2) * nf + k];
      }
    }
    const double wgt = interior ? 0.5 : 1.0;
    const double rb = 0.5 * (1.0 / mat[e] + 1.0 / mat[o]);
    const double lb = 0.5 * (mat[nel + e] + mat[nel + o]);
    const double mb = 0.5 * (mat[2 * nel + e] + mat[2 * nel + o]);
    const double zp = sqrt(rb * (lb + 2.0 * mb)), zs = sqrt(rb * mb);
    g0 += wgt * (gzp * (lb + 2.0 * mb) / (2.0 * zp) + gzs * mb / (2.0 * zs));
    g1 += wgt * (gzp * rb / (2.0 * zp));
    g2 += wgt * (gzp * rb / zp + gzs * rb / (2.0 * zs));
  }
  grad[e] += g0;
  grad[nel + e] += g1;
  grad[2 * nel + e] += g2;
}

__global__ void receivers_sample_kernel(const double* __restrict__ u, const long long* __restrict__ relem,
                                        const double* __restrict__ rw, long long nel, int Np, double* out) {
  __shared__ double red[3][128];
  const int r = blockIdx.x;
  const size_t total = (size_t)nel * Np;
  const long long e = relem[r];
  double s[3] = {0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < Np; j += blockDim.x) {
    const double w = rw[(size_t)r * Np + j];
    for (int c = 0; c < 3; ++c) s[c] += w * u[c * total + (size_t)e * Np + j];
  }
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
  __syncthreads();
  if (threadIdx.x < 3) {
    double acc = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) acc += red[threadIdx.x][k];
    out[r * 3 + threadIdx.x] = acc;
  }
}

// Receivers one after another (several may share an element): deterministic.
__global__ void receivers_adjoint_kernel(double* __restrict__ lu, const long long* __restrict__ relem,
                                         const double* __restrict__ rw, const double* __restrict__ gv, int nrec,
                                         long long nel, int Np) {
  const size_t total = (size_t)nel * Np;
  for (int r = 0; r < nrec; ++r) {
    const long long e = relem[r];
    for (int j = threadIdx.x; j < Np; j += blockDim.x) {
      const double w = rw[(size_t)r * Np + j];
      for (int c = 0; c < 3; ++c) lu[c * total + (size_t)e * Np + j] += gv[r * 3 + c] * w;
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace dgw

namespace {

dgw_status afail(dgw_ctx* c, dgw_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    dgw::set_no_context_error(msg);
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

const double kA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                      -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                      1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                      2277821191437.0 / 14882151754819.0};
const double kC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                      2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

double ricker_h(double t, double f0, double t0) {
  const double a = M_PI * f0 * (t - t0);
  return (1.0 - 2.0 * a * a) * std::exp(-a * a);
}

#define ACUDA(call, what)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return afail(c, DGW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

dgw_status ensure(dgw_ctx* c, double** p, size_t& cap, size_t need) {
  if (*p && cap >= need) return DGW_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  cap = 0;
  if (cudaMalloc((void**)p, need) != cudaSuccess) return afail(c, DGW_ERR_OOM, "adjoint scratch");
  cap = need;
  return DGW_OK;
}

dgw::StageParams base_params(dgw_ctx* c) {
  dgw::StageParams p{};
  p.geo = c->geo;
  p.fz = c->fz;
  p.vmapP = c->vmapP;
  p.mat = c->mat;
  p.nel = c->nel;
  p.tau = c->cfg.flux_tau ? 1.0 : 0.0;
  p.w_end_inv = 1.0 / c->ref.w[0];
  p.wJ = c->wJ;
  p.ec = c->ec;
  p.src_elem = c->src_elem;
  p.src_w = c->src_w;
  for (int i = 0; i < (c->cfg.N + 1) * (c->cfg.N + 1); ++i) p.D[i] = c->ref.D[i];
  return p;
}

}  // namespace

extern "C" {

dgw_status dgw_receivers_set(dgw_ctx* c, int n, const int64_t* elements, const double* xi) {
  if (!c) return afail(nullptr, DGW_ERR_ARG, "null context");
  if (c->cfg.system != DGW_SYSTEM_ELASTIC) return afail(c, DGW_ERR_UNSUPPORTED, "receivers are elastic only");
  if (!c->has_mesh) return afail(c, DGW_ERR_STATE, "receivers before mesh");
  if (n < 0 || (n > 0 && (!elements || !xi))) return afail(c, DGW_ERR_ARG, "bad receiver arrays");
  const int N = c->cfg.N, nn = N + 1, Np = nn * nn * nn;
  std::vector<double> w((size_t)n * Np);
  std::vector<long long> el(n);
  for (int r = 0; r < n; ++r) {
    if (elements[r] < 0 || elements[r] >= c->nel) return afail(c, DGW_ERR_ARG, "receiver element out of range");
    el[r] = elements[r];
    double l[3][dgw::kMaxN + 1];
    for (int a = 0; a < 3; ++a) {
      const double x = xi[3 * r + a];
      if (!(x >= -1.0 && x <= 1.0)) return afail(c, DGW_ERR_ARG, "receiver xi must lie in [-1, 1]^3");
      for (int j = 0; j < nn; ++j) {
        double v = 1.0;
        for (int k = 0; k < nn; ++k)
          if (k != j) v *= (x - c->ref.r[k]) / (c->ref.r[j] - c->ref.r[k]);
        l[a][j] = v;
      }
    }
    for (int kk = 0; kk < nn; ++kk)
      for (int jj = 0; jj < nn; ++jj)
        for (int ii = 0; ii < nn; ++ii) w[(size_t)r * Np + ii + nn * (jj + nn * kk)] = l[0][ii] * l[1][jj] * l[2][kk];
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return afail(c, DGW_ERR_CUDA, "cudaSetDevice");
  if (c->rec_elem) cudaFree(c->rec_elem);
  if (c->rec_w) cudaFree(c->rec_w);
  c->rec_elem = nullptr;
  c->rec_w = nullptr;
  c->rec_n = 0;
  if (n == 0) return DGW_OK;
  ACUDA(cudaMalloc(&c->rec_elem, n * sizeof(long long)), "alloc receivers");
  ACUDA(cudaMalloc(&c->rec_w, w.size() * sizeof(double)), "alloc receivers");
  ACUDA(cudaMemcpyAsync(c->rec_elem, el.data(), n * sizeof(long long), cudaMemcpyHostToDevice, c->setup), "copy receivers");
  ACUDA(cudaMemcpyAsync(c->rec_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, c->setup), "copy receivers");
  ACUDA(cudaStreamSynchronize(c->setup), "copy receivers");
  c->rec_n = n;
  return DGW_OK;
}

dgw_status dgw_receivers_sample(dgw_ctx* c, const double* u, double* out, void* stream) {
  if (!c) return afail(nullptr, DGW_ERR_ARG, "null context");
  if (!c->has_mesh || c->rec_n == 0) return afail(c, DGW_ERR_STATE, "no receivers");
  if (!u || !out || !dev_ptr(u) || !dev_ptr(out)) return afail(c, DGW_ERR_ARG, "u and out must be device buffers");
  if (cudaSetDevice(c->device) != cudaSuccess) return afail(c, DGW_ERR_CUDA, "cudaSetDevice");
  const int Np = (c->cfg.N + 1) * (c->cfg.N + 1) * (c->cfg.N + 1);
  dgw::receivers_sample_kernel<<<c->rec_n, 128, 0, (cudaStream_t)stream>>>(u, c->rec_elem, c->rec_w, c->nel, Np, out);
  ACUDA(cudaGetLastError(), "receiver sampling");
  return DGW_OK;
}

dgw_status dgw_receivers_adjoint(dgw_ctx* c, double* lam_u, const double* gv, void* stream) {
  if (!c) return afail(nullptr, DGW_ERR_ARG, "null context");
  if (!c->has_mesh || c->rec_n == 0) return afail(c, DGW_ERR_STATE, "no receivers");
  if (!lam_u || !gv || !dev_ptr(lam_u) || !dev_ptr(gv)) return afail(c, DGW_ERR_ARG, "device buffers required");
  if (cudaSetDevice(c->device) != cudaSuccess) return afail(c, DGW_ERR_CUDA, "cudaSetDevice");
  const int Np = (c->cfg.N + 1) * (c->cfg.N + 1) * (c->cfg.N + 1);
  dgw::receivers_adjoint_kernel<<<1, 128, 0, (cudaStream_t)stream>>>(lam_u, c->rec_elem, c->rec_w, gv, c->rec_n,
                                                                     c->nel, Np);
  ACUDA(cudaGetLastError(), "receiver adjoint");
  return DGW_OK;
}

// The adjoint of nsteps steps from the checkpoint u_ckpt (with receiver-trace
// sources g_traces[k] injected before the transpose of step k when g_traces is
// not NULL).  The forward states are recomputed once, keeping every stage
// input and, when the scratch fits, every stage's operator output dt (K u + f)
// (10 nsteps states; else 5 nsteps and the gradient terms recompute the
// operator); the reverse sweep then runs, per stage, the weight preparation
// and the fused GRAD + ADJ kernel.
static dgw_status adjoint_segment(dgw_ctx* c, double* lam_u, double* lam_res, double* grad_mat, const double* u_ckpt,
                                  const double* g_traces, double t0, double dt, int nsteps, cudaStream_t s) {
  if (!c) return afail(nullptr, DGW_ERR_ARG, "null context");
  if (c->cfg.system != DGW_SYSTEM_ELASTIC) return afail(c, DGW_ERR_UNSUPPORTED, "the adjoint is elastic only");
  if (!c->has_mesh || !c->has_material) return afail(c, DGW_ERR_STATE, "adjoint before mesh and material");
  if (c->cfg.precision != DGW_PRECISION_FP64)
    return afail(c, DGW_ERR_UNSUPPORTED, "the adjoint is built for FP64 contexts only");
  if (nsteps < 1) return afail(c, DGW_ERR_ARG, "nsteps must be >= 1");
  if (!(dt > 0.0) || !std::isfinite(t0)) return afail(c, DGW_ERR_ARG, "need dt > 0 and finite t0");
  const void* ptrs[] = {lam_u, lam_res, grad_mat, u_ckpt};
  for (const void* q : ptrs)
    if (!q || !dev_ptr(q)) return afail(c, DGW_ERR_ARG, "lam_u, lam_res, grad_mat and u_ckpt must be device buffers");
  if (lam_u == lam_res) return afail(c, DGW_ERR_ARG, "lam_u and lam_res must be distinct");
  if (g_traces) {
    if (c->rec_n == 0) return afail(c, DGW_ERR_STATE, "trace sources without receivers");
    if (!dev_ptr(g_traces)) return afail(c, DGW_ERR_ARG, "g_traces must be a device buffer");
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return afail(c, DGW_ERR_CUDA, "cudaSetDevice");
  const int N = c->cfg.N, n = N + 1, Np = n * n * n, nf = n * n;
  const size_t state = (size_t)c->nel * Np * 9 * sizeof(double);
  const size_t nodes = (size_t)c->nel * Np;
  // scratch: W, Z, forward register, the 5 stage inputs of every step, then
  // (when it fits) the 5 stage outputs dt (K u + f) of every step
  dgw_status st;
  const char* low = std::getenv("DGW_ADJOINT_LOW_MEMORY");
  bool keep_out = !(low && low[0] == '1');
  if (!keep_out ||
      ensure(c, &c->adj_scratch, c->adj_scratch_bytes, state * (3 + 10 * (size_t)nsteps)) != DGW_OK) {
    cudaGetLastError();
    keep_out = false;
    if ((st = ensure(c, &c->adj_scratch, c->adj_scratch_bytes, state * (3 + 5 * (size_t)nsteps))) != DGW_OK)
      return st;
  }
  if ((st = ensure(c, &c->adj_gface, c->adj_gface_bytes, 2 * (size_t)c->nel * 6 * nf * sizeof(double))) != DGW_OK)
    return st;
  if (!c->etoe_d) {
    ACUDA(cudaMalloc(&c->etoe_d, c->nel * 6 * sizeof(long long)), "alloc connectivity");
    ACUDA(cudaMalloc(&c->etof_d, c->nel * 6), "alloc connectivity");
    std::vector<signed char> f8(c->nel * 6);
    for (long long k = 0; k < c->nel * 6; ++k) f8[k] = (signed char)c->etof[k];
    ACUDA(cudaMemcpyAsync(c->etoe_d, c->etoe.data(), c->nel * 6 * sizeof(long long), cudaMemcpyHostToDevice, c->setup), "copy");
    ACUDA(cudaMemcpyAsync(c->etof_d, f8.data(), c->nel * 6, cudaMemcpyHostToDevice, c->setup), "copy");
    ACUDA(cudaStreamSynchronize(c->setup), "copy connectivity");
  }
  double* base = c->adj_scratch;
  double* W = base;
  double* Z = base + 9 * nodes;
  double* fres = base + 2 * 9 * nodes;
  double* ins = base + 3 * 9 * nodes;
  // input of stage st of step k: the checkpoint for (0, 0), else slot 5 k + st
  auto input = [&](int k, int st_) -> double* {
    return (k == 0 && st_ == 0) ? const_cast<double*>(u_ckpt) : ins + (size_t)(5 * k + st_) * 9 * nodes;
  };
  double* outs = ins + (size_t)5 * nsteps * 9 * nodes;
  auto output = [&](int k, int st_) -> double* {
    return keep_out ? outs + (size_t)(5 * k + st_) * 9 * nodes : nullptr;
  };
  ACUDA(cudaMemsetAsync(c->adj_gface, 0, 2 * (size_t)c->nel * 6 * nf * sizeof(double), s), "clear face terms");

  // forward recompute of the segment (the first stage of a step does not read
  // the register, a_0 = 0); the last step's final state is not needed (its
  // last stage runs only for its operator output, into W)
  for (int k = 0; k < nsteps; ++k) {
    for (int st_ = 0; st_ < 5; ++st_) {
      const bool last = k == nsteps - 1 && st_ == 4;
      if (last && !keep_out) break;
      dgw::StageParams p = base_params(c);
      p.u_in = input(k, st_);
      p.out = last ? W : (st_ < 4 ? input(k, st_ + 1) : input(k + 1, 0));
      p.rout = output(k, st_);
      p.res = fres;
      p.a = kA[st_];
      p.b = kB[st_];
      p.dt = dt;
      p.src_amp = c->src_elem >= 0 ? ricker_h(t0 + k * dt + kC[st_] * dt, c->src_f0, c->src_t0) : 0.0;
      ACUDA(dgw::launch_stage_fp64(N, true, p, s), "forward recompute");
    }
  }
  const int pblocks = c->sm_count * 8;
  const int Np_ = Np;
  for (int k = nsteps - 1; k >= 0; --k) {
    const double tk = t0 + k * dt;
    if (g_traces) {
      dgw::receivers_adjoint_kernel<<<1, 128, 0, s>>>(lam_u, c->rec_elem, c->rec_w, g_traces + (size_t)k * c->rec_n * 3,
                                                      c->rec_n, c->nel, Np_);
      ACUDA(cudaGetLastError(), "receiver adjoint");
    }
    for (int st_ = 4; st_ >= 0; --st_) {
      dgw::adjoint_prep_kernel<<<pblocks, 256, 0, s>>>(lam_u, lam_res, W, Z, static_cast<const double*>(c->mat),
                                                       c->wJ, c->nel, Np, kA[st_], kB[st_]);
      ACUDA(cudaGetLastError(), "adjoint preparation");
      dgw::StageParams g = base_params(c);
      g.u_in = input(k, st_);
      g.res = W;
      g.out = nullptr;
      g.dt = dt;
      g.grad_el = grad_mat;
      g.grad_face = c->adj_gface;
      g.rout = output(k, st_);
      g.src_amp = c->src_elem >= 0 ? ricker_h(tk + kC[st_] * dt, c->src_f0, c->src_t0) : 0.0;
      dgw::StageParams a = base_params(c);
      a.u_in = Z;
      a.res = lam_u;
      a.out = lam_u;
      a.dt = dt;
      a.src_elem = -1;
      ACUDA(dgw::launch_stage_adjgrad(N, g, a, s), "adjoint stage");
    }
  }
  dgw::adjoint_chain_kernel<<<(unsigned)((c->nel + 127) / 128), 128, 0, s>>>(
      c->adj_gface, c->etoe_d, c->etof_d, static_cast<const double*>(c->mat), c->nel, nf, grad_mat);
  ACUDA(cudaGetLastError(), "gradient chain");
  return DGW_OK;
}

dgw_status dgw_adjoint_step(dgw_ctx* c, double* lam_u, double* lam_res, double* grad_mat, const double* u_ckpt,
                            double t0, double dt, int nsteps, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_adjoint_step");
  return adjoint_segment(c, lam_u, lam_res, grad_mat, u_ckpt, nullptr, t0, dt, nsteps, (cudaStream_t)stream);
}

dgw_status dgw_adjoint_traces(dgw_ctx* c, double* lam_u, double* lam_res, double* grad_mat, const double* u_ckpt,
                              const double* g_traces, double t0, double dt, int nsteps, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_adjoint_traces");
  if (c && !g_traces) return afail(c, DGW_ERR_ARG, "g_traces must be given (dgw_adjoint_step runs without)");
  return adjoint_segment(c, lam_u, lam_res, grad_mat, u_ckpt, g_traces, t0, dt, nsteps, (cudaStream_t)stream);
}

}  // extern "C"
