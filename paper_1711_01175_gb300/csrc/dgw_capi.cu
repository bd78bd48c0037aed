// C ABI entry points (declared in include/dgw.h): context, mesh and material
// upload with validation, and the compute calls that enqueue the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "dgw_internal.cuh"

namespace {

thread_local std::string g_error;   // errors of calls without a usable context

dgw_status fail(dgw_ctx* ctx, dgw_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_error = buf;
  return st;
}

dgw_status cuda_fail(dgw_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? DGW_ERR_OOM : DGW_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define DGW_CUDA(ctx, call, what)                       \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

// LSRK(5,4) of Carpenter & Kennedy (1994), 2N-storage, five stages, fourth order.
const double kLsrkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                          -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kLsrkC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                          2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};
const double kLsrkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                          1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                          2277821191437.0 / 14882151754819.0};

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

void free_mesh(dgw_ctx* c) {
  dfree(c->geo);
  dfree(c->fz);
  dfree(c->vmapP);
  dfree(c->wJ);
  dfree(c->u2);
  dfree(c->partials);
  dfree(c->stage_partials);
  c->stage_ctas = 0;
  dfree(c->stage_u);
  dfree(c->stage_res);
  dfree(c->mat);
  dfree(c->ec);
  dfree(c->src_w);
  c->src_elem = -1;
  dfree(c->rec_elem);
  dfree(c->rec_w);
  c->rec_n = 0;
  dfree(c->adj_scratch);
  c->adj_scratch_bytes = 0;
  dfree(c->adj_gface);
  c->adj_gface_bytes = 0;
  dfree(c->etoe_d);
  dfree(c->etof_d);
  dgw::ihdg_release(c);
  c->has_mesh = c->has_material = false;
  c->nel = 0;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int Np_of(int N) { return (N + 1) * (N + 1) * (N + 1); }

// Ricker wavelet (1 - 2 (pi f0 (t - t0))^2) exp(-(pi f0 (t - t0))^2).
double ricker(double t, double f0, double t0) {
  const double a = M_PI * f0 * (t - t0);
  return (1.0 - 2.0 * a * a) * std::exp(-a * a);
}

dgw_status launch_stage(dgw_ctx* c, const double* u_in, double* out, double* res, bool lsrk,
                        double a, double b, double dt, cudaStream_t s, double* energy_partials = nullptr,
                        double t_stage = 0.0) {
  dgw::StageParams p{};
  {
    int epb = 0, nthreads = 0;
    dgw::stage_shape(c->cfg.N, &epb, &nthreads);
    p.pf_elems = 1LL * c->sm_count * epb * dgw::stage_pf_tenths(c->cfg.N, c->cfg.precision) / 10;
  }
  p.src_elem = c->src_elem;
  p.src_w = c->src_w;
  p.fault = c->fault;
  p.src_amp = c->src_elem >= 0 ? ricker(t_stage, c->src_f0, c->src_t0) : 0.0;
  p.energy_partials = energy_partials;
  p.wJ = c->wJ;
  p.ec = c->ec;
  p.u_in = u_in;
  p.out = out;
  p.res = res;
  p.geo = c->geo;
  p.fz = c->fz;
  p.vmapP = c->vmapP;
  p.mat = c->mat;
  p.nel = c->nel;
  p.a = a;
  p.b = b;
  p.dt = dt;
  p.tau = c->cfg.flux_tau ? 1.0 : 0.0;
  p.w_end_inv = 1.0 / c->ref.w[0];
  std::memcpy(p.D, c->ref.D, sizeof(p.D));
  for (int k = 0; k < 3; ++k) p.beta[k] = c->cfg.beta[k];
  cudaError_t e = c->cfg.system != DGW_SYSTEM_ELASTIC ? dgw::launch_friedrichs(c->cfg.system, c->cfg.N, lsrk, p, s)
                  : c->cfg.precision == DGW_PRECISION_MIXED ? dgw::launch_stage_mixed(c->cfg.N, lsrk, p, s)
                  : c->cfg.precision == DGW_PRECISION_FP64  ? dgw::launch_stage_fp64(c->cfg.N, lsrk, p, s)
                                                            : dgw::launch_stage_mixed_tc(c->cfg.N, c->cfg.precision, lsrk, p, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel launch");
  return DGW_OK;
}

dgw_status ready(dgw_ctx* c) {
  if (!c) return fail(nullptr, DGW_ERR_ARG, "null context");
  if (!c->has_mesh) return fail(c, DGW_ERR_STATE, "no mesh uploaded");
  if (!c->has_material) return fail(c, DGW_ERR_STATE, "no material uploaded");
  return DGW_OK;
}

dgw_status set_device(dgw_ctx* c) {
  DGW_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  return DGW_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// Reference element: GLL nodes (end points and roots of P_N'), weights
// 2 / (N (N+1) P_N(r)^2), and the Lagrange derivative matrix.
// ----------------------------------------------------------------------------
namespace dgw {

static void legendre_pd(int N, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 1; k < N; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    const double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

bool build_ref_elem(int N, RefElem* out) {
  if (N < 1 || N > kMaxN) return false;
  RefElem R;
  R.N = N;
  const int n = N + 1;
  for (int i = 0; i < n; ++i) {
    double x = -std::cos(M_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 100; ++it) {
        double P, dP;
        legendre_pd(N, x, &P, &dP);
        // root of (1 - x^2) P_N'(x): Newton with derivative -N(N+1) P_N(x)
        const double step = ((1.0 - x * x) * dP) / (-N * (N + 1.0) * P);
        x -= step;
        if (std::fabs(step) < 1e-16) break;
      }
    }
    R.r[i] = (i == 0) ? -1.0 : (i == N ? 1.0 : x);
  }
  for (int i = 0; i < n; ++i) {
    double P, dP;
    legendre_pd(N, R.r[i], &P, &dP);
    R.w[i] = 2.0 / (N * (N + 1.0) * P * P);
  }
  double bw[kMaxN + 1];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (R.r[j] - R.r[k]);
    bw[j] = 1.0 / prod;
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      R.D[i * n + j] = (bw[j] / bw[i]) / (R.r[i] - R.r[j]);
      diag -= R.D[i * n + j];   // rows of D sum to zero (derivative of a constant)
    }
    R.D[i * n + i] = diag;
  }
  *out = R;
  return true;
}

void set_no_context_error(const std::string& msg) { g_error = msg; }

}  // namespace dgw

// ----------------------------------------------------------------------------
extern "C" {

int dgw_abi_version(void) { return DGW_ABI_VERSION; }

dgw_status dgw_reference_nodes(int N, double* r, double* w) {
  if (!r || !w) return fail(nullptr, DGW_ERR_ARG, "null output pointer");
  dgw::RefElem R;
  if (!dgw::build_ref_elem(N, &R)) return fail(nullptr, DGW_ERR_ARG, "N=%d outside 1..%d", N, dgw::kMaxN);
  for (int i = 0; i <= N; ++i) {
    r[i] = R.r[i];
    w[i] = R.w[i];
  }
  return DGW_OK;
}

dgw_status dgw_create(dgw_ctx** out, int device, const dgw_config* cfg) {
  if (!out || !cfg) return fail(nullptr, DGW_ERR_ARG, "null argument");
  *out = nullptr;
  if (cfg->N < 1 || cfg->N > dgw::kMaxN) return fail(nullptr, DGW_ERR_ARG, "N=%d outside 1..7", cfg->N);
  if (cfg->flux_tau != 0 && cfg->flux_tau != 1) return fail(nullptr, DGW_ERR_ARG, "flux_tau must be 0 or 1");
  if (cfg->precision < DGW_PRECISION_FP64 || cfg->precision > DGW_PRECISION_MIXED_TC_BF16)
    return fail(nullptr, DGW_ERR_ARG, "unknown precision %d", cfg->precision);
  if (!(cfg->cfl > 0.0)) return fail(nullptr, DGW_ERR_ARG, "cfl must be positive");
  if (cfg->system != DGW_SYSTEM_ELASTIC && cfg->system != DGW_SYSTEM_TRANSPORT &&
      cfg->system != DGW_SYSTEM_SHALLOW_WATER)
    return fail(nullptr, DGW_ERR_ARG, "unknown system %d", cfg->system);
  if (cfg->system != DGW_SYSTEM_ELASTIC && cfg->precision != DGW_PRECISION_FP64)
    return fail(nullptr, DGW_ERR_UNSUPPORTED, "transport and shallow water are built in FP64 only");
  if (cfg->system == DGW_SYSTEM_TRANSPORT) {
    const double b2 = cfg->beta[0] * cfg->beta[0] + cfg->beta[1] * cfg->beta[1] + cfg->beta[2] * cfg->beta[2];
    if (!(b2 > 0.0) || !std::isfinite(b2)) return fail(nullptr, DGW_ERR_ARG, "transport needs a finite nonzero beta");
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev)
    return fail(nullptr, DGW_ERR_CUDA, "no CUDA device %d (%s)", device,
                e == cudaSuccess ? "out of range" : cudaGetErrorString(e));
  dgw_ctx* c = new dgw_ctx();
  c->device = device;
  c->cfg = *cfg;
  c->m = cfg->system == DGW_SYSTEM_ELASTIC ? 9 : (cfg->system == DGW_SYSTEM_TRANSPORT ? 1 : 3);
  dgw::build_ref_elem(cfg->N, &c->ref);
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return fail(nullptr, DGW_ERR_CUDA, "cudaSetDevice(%d) failed", device);
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaStreamCreateWithFlags(&c->setup, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return fail(nullptr, DGW_ERR_CUDA, "set-up stream");
  }
  if (cudaMalloc(&c->fault, 2 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(c->fault, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaStreamDestroy(c->setup);
    if (c->fault) cudaFree(c->fault);
    delete c;
    return fail(nullptr, DGW_ERR_CUDA, "fault word");
  }
  *out = c;
  return DGW_OK;
}

dgw_status dgw_destroy(dgw_ctx* c) {
  if (!c) return DGW_OK;
  cudaSetDevice(c->device);
  free_mesh(c);
  if (c->setup) cudaStreamDestroy(c->setup);
  if (c->fault) cudaFree(c->fault);
  delete c;
  return DGW_OK;
}

dgw_status dgw_debug_status(dgw_ctx* c, int* code, int64_t* element, int64_t* count) {
  if (!c) return fail(nullptr, DGW_ERR_ARG, "null context");
  if (!dgw::kDebugChecks) return fail(c, DGW_ERR_UNSUPPORTED, "library built without DGW_DEBUG_CHECKS");
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  unsigned long long f[2] = {0, 0};
  DGW_CUDA(c, cudaDeviceSynchronize(), "debug status");
  DGW_CUDA(c, cudaMemcpy(f, c->fault, sizeof f, cudaMemcpyDeviceToHost), "debug status");
  DGW_CUDA(c, cudaMemset(c->fault, 0, sizeof f), "debug status");
  if (code) *code = (int)(f[0] >> 56);
  if (element) *element = (int64_t)(f[0] & ((1ull << 56) - 1));
  if (count) *count = (int64_t)f[1];
  return DGW_OK;
}

dgw_status dgw_mesh_upload(dgw_ctx* c, int64_t nel, const double* x, const int64_t* etoe,
                           const int8_t* etof, const int8_t* orient, const int8_t* bc) {
  dgw::NvtxRange nvtx_range("dgw_mesh_upload");
  if (!c) return fail(nullptr, DGW_ERR_ARG, "null context");
  if (!x || !etoe || !etof || !orient || !bc) return fail(c, DGW_ERR_ARG, "null mesh array");
  const int N = c->cfg.N, n = N + 1, Np = Np_of(N), nf = n * n;
  if (nel <= 0) return fail(c, DGW_ERR_ARG, "nel must be positive");
  if ((double)nel * Np >= 2147483647.0) return fail(c, DGW_ERR_ARG, "nel*Np must be below 2^31");
  // Connectivity checks.
  for (int64_t e = 0; e < nel; ++e) {
    for (int f = 0; f < 6; ++f) {
      const int64_t k = e * 6 + f;
      const int64_t e2 = etoe[k];
      if (e2 >= 0) {
        if (e2 >= nel) return fail(c, DGW_ERR_ARG, "element %lld face %d: neighbour %lld out of range", (long long)e, f, (long long)e2);
        if (bc[k] != DGW_BC_INTERIOR) return fail(c, DGW_ERR_ARG, "element %lld face %d: neighbour given but bc tag %d", (long long)e, f, bc[k]);
        const int f2 = etof[k], o = orient[k];
        if (f2 < 0 || f2 >= 6 || o < 0 || o >= 8) return fail(c, DGW_ERR_ARG, "element %lld face %d: bad etof/orient", (long long)e, f);
        const int64_t k2 = e2 * 6 + f2;
        if (etoe[k2] != e || etof[k2] != f) return fail(c, DGW_ERR_ARG, "element %lld face %d: connectivity not symmetric", (long long)e, f);
        // The neighbour's permutation must be the inverse of ours: check the corners.
        const int o2 = orient[k2];
        const int cs[3][2] = {{0, 0}, {N, 0}, {0, N}};
        for (auto& cc : cs) {
          int a1 = (o & 1) ? cc[1] : cc[0], b1 = (o & 1) ? cc[0] : cc[1];
          int a2 = (o & 2) ? N - a1 : a1, b2 = (o & 4) ? N - b1 : b1;
          int a3 = (o2 & 1) ? b2 : a2, b3 = (o2 & 1) ? a2 : b2;
          int a4 = (o2 & 2) ? N - a3 : a3, b4 = (o2 & 4) ? N - b3 : b3;
          if (a4 != cc[0] || b4 != cc[1])
            return fail(c, DGW_ERR_ARG, "element %lld face %d: orientation codes %d/%d are not inverse", (long long)e, f, o, o2);
        }
      } else {
        if (bc[k] != DGW_BC_FREE_SURFACE && bc[k] != DGW_BC_ABSORBING)
          return fail(c, DGW_ERR_ARG, "element %lld face %d: boundary face without a boundary tag", (long long)e, f);
        if (bc[k] == DGW_BC_FREE_SURFACE && c->cfg.system == DGW_SYSTEM_TRANSPORT)
          return fail(c, DGW_ERR_ARG, "element %lld face %d: tag 1 (wall) is not defined for transport", (long long)e, f);
      }
    }
  }
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  free_mesh(c);
  // Neighbour map: flat e2*Np + node2 per face node, or the ghost sentinel.
  std::vector<int> vmap((size_t)nel * 6 * nf);
  const int tang[3][2] = {{1, 2}, {0, 2}, {0, 1}};
  auto vol_node = [&](int f, int a, int b) {
    int ijk[3];
    const int d = f / 2;
    ijk[d] = (f & 1) ? N : 0;
    ijk[tang[d][0]] = a;
    ijk[tang[d][1]] = b;
    return ijk[0] + n * (ijk[1] + n * ijk[2]);
  };
  for (int64_t e = 0; e < nel; ++e) {
    for (int f = 0; f < 6; ++f) {
      const int64_t k = e * 6 + f;
      for (int b = 0; b < n; ++b) {
        for (int a = 0; a < n; ++a) {
          int val;
          if (etoe[k] >= 0) {
            const int o = orient[k];
            int a1 = (o & 1) ? b : a, b1 = (o & 1) ? a : b;
            int a2 = (o & 2) ? N - a1 : a1, b2 = (o & 4) ? N - b1 : b1;
            val = (int)(etoe[k] * Np + vol_node(etof[k], a2, b2));
          } else {
            val = bc[k] == DGW_BC_FREE_SURFACE ? dgw::kGhostFreeSurface : dgw::kGhostAbsorbing;
          }
          vmap[(size_t)k * nf + a + n * b] = val;
        }
      }
    }
  }
  // Shortest element edge (corner to corner), for the CFL time step.
  double hmin = INFINITY;
  const int corner_edges[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                                   {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
  for (int64_t e = 0; e < nel; ++e) {
    const double* xe = x + (size_t)e * Np * 3;
    int cn[8];
    for (int cc = 0; cc < 8; ++cc)
      cn[cc] = ((cc & 1) ? N : 0) + n * (((cc & 2) ? N : 0) + n * ((cc & 4) ? N : 0));
    for (auto& ed : corner_edges) {
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double dd = xe[cn[ed[0]] * 3 + k] - xe[cn[ed[1]] * 3 + k];
        d2 += dd * dd;
      }
      hmin = std::fmin(hmin, std::sqrt(d2));
    }
  }

  const size_t nodes = (size_t)nel * Np, fnodes = (size_t)nel * 6 * nf;
  double *x_d = nullptr, *geo64 = nullptr, *minJ = nullptr, *D_d = nullptr, *w_d = nullptr;
  auto cleanup = [&]() {
    dfree(x_d);
    dfree(minJ);
    dfree(D_d);
    dfree(w_d);
    if (c->geo != (void*)geo64) dfree(geo64);
  };
#define DGW_TRY(call, what)                          \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) {                         \
      cleanup();                                     \
      free_mesh(c);                                  \
      return cuda_fail(c, e_, what);                 \
    }                                                \
  } while (0)
  DGW_TRY(cudaMalloc(&x_d, nodes * 3 * sizeof(double)), "alloc x");
  DGW_TRY(cudaMalloc(&geo64, nodes * 10 * sizeof(double)), "alloc geometry");
  DGW_TRY(cudaMalloc(&c->wJ, nodes * sizeof(double)), "alloc wJ");
  DGW_TRY(cudaMalloc(&minJ, (size_t)nel * sizeof(double)), "alloc minJ");
  DGW_TRY(cudaMalloc(&D_d, sizeof(c->ref.D)), "alloc D");
  DGW_TRY(cudaMalloc(&w_d, sizeof(c->ref.w)), "alloc w");
  DGW_TRY(cudaMalloc(&c->vmapP, fnodes * sizeof(int)), "alloc neighbour map");
  DGW_TRY(cudaMalloc(&c->u2, nodes * c->m * sizeof(double)), "alloc state buffer");
  DGW_TRY(cudaMalloc(&c->partials, (dgw::kEnergyBlocks + 1) * sizeof(double)), "alloc energy partials");
  {
    int epb = 0, nthreads = 0;
    dgw::stage_shape(N, &epb, &nthreads);
    c->stage_ctas = (int)((nel + epb - 1) / epb);
    DGW_TRY(cudaMalloc(&c->stage_partials, ((size_t)c->stage_ctas + 1 + dgw::kEnergyBlocks) * sizeof(double)),
            "alloc stage energy partials");
  }
  DGW_TRY(cudaMemcpyAsync(x_d, x, nodes * 3 * sizeof(double), cudaMemcpyHostToDevice, c->setup), "copy x");
  DGW_TRY(cudaMemcpyAsync(D_d, c->ref.D, sizeof(c->ref.D), cudaMemcpyHostToDevice, c->setup), "copy D");
  DGW_TRY(cudaMemcpyAsync(w_d, c->ref.w, sizeof(c->ref.w), cudaMemcpyHostToDevice, c->setup), "copy w");
  DGW_TRY(cudaMemcpyAsync(c->vmapP, vmap.data(), fnodes * sizeof(int), cudaMemcpyHostToDevice, c->setup), "copy neighbour map");
  dgw::GeometryOut go{geo64, c->wJ, minJ};
  DGW_TRY(dgw::launch_geometry(N, x_d, nel, D_d, w_d, go, c->setup), "geometry kernel");
  DGW_TRY(cudaStreamSynchronize(c->setup), "geometry kernel");
  std::vector<double> mj(nel);
  DGW_TRY(cudaMemcpyAsync(mj.data(), minJ, nel * sizeof(double), cudaMemcpyDeviceToHost, c->setup), "copy minJ");
  DGW_TRY(cudaStreamSynchronize(c->setup), "copy minJ");
  for (int64_t e = 0; e < nel; ++e) {
    if (!(mj[e] > 0.0)) {
      cleanup();
      free_mesh(c);
      return fail(c, DGW_ERR_ARG, "element %lld: Jacobian %.3e <= 0 at some node", (long long)e, mj[e]);
    }
  }
  if (dgw::fp32_arrays(c->cfg.precision)) {
    float* g32 = nullptr;
    DGW_TRY(cudaMalloc(&g32, nodes * 10 * sizeof(float)), "alloc geometry fp32");
    c->geo = g32;
    DGW_TRY(dgw::launch_to_float(geo64, g32, nodes * 10, c->setup), "geometry to fp32");
    DGW_TRY(cudaStreamSynchronize(c->setup), "geometry to fp32");
  } else {
    c->geo = geo64;
  }
  cleanup();
#undef DGW_TRY
  c->nel = nel;
  c->etoe.assign(etoe, etoe + nel * 6);
  c->etof.assign(etof, etof + nel * 6);
  c->bc.assign(bc, bc + nel * 6);
  c->h_min = hmin;
  c->has_mesh = true;
  c->has_material = false;
  if (c->cfg.system != DGW_SYSTEM_ELASTIC) {
    // Q = I: no medium to upload; the wave speed is |beta| (transport) or sqrt(Phi) = 1.
    const double* b = c->cfg.beta;
    c->c_max = c->cfg.system == DGW_SYSTEM_TRANSPORT ? std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]) : 1.0;
    c->has_material = true;
  }
  return DGW_OK;
}

dgw_status dgw_material_upload(dgw_ctx* c, const double* rho, const double* lam, const double* mu) {
  dgw::NvtxRange nvtx_range("dgw_material_upload");
  if (!c) return fail(nullptr, DGW_ERR_ARG, "null context");
  if (c->cfg.system != DGW_SYSTEM_ELASTIC)
    return fail(c, DGW_ERR_UNSUPPORTED, "transport and shallow water have no medium (Q = I)");
  if (!c->has_mesh) return fail(c, DGW_ERR_STATE, "material before mesh");
  if (!rho || !lam || !mu) return fail(c, DGW_ERR_ARG, "null material array");
  const long long nel = c->nel;
  std::vector<double> m64(3 * nel), ec(4 * nel);
  double cmax = 0.0;
  for (long long e = 0; e < nel; ++e) {
    if (!(rho[e] > 0.0) || !(mu[e] > 0.0) || !(lam[e] > -2.0 / 3.0 * mu[e]) || !std::isfinite(lam[e]))
      return fail(c, DGW_ERR_ARG, "element %lld: need rho > 0, mu > 0, lambda > -2/3 mu", e);
    m64[e] = 1.0 / rho[e];
    m64[nel + e] = lam[e];
    m64[2 * nel + e] = mu[e];
    ec[e] = rho[e];
    ec[nel + e] = 1.0 / (2.0 * mu[e]);
    ec[2 * nel + e] = lam[e] / (3.0 * lam[e] + 2.0 * mu[e]);
    ec[3 * nel + e] = 1.0 / mu[e];
    cmax = std::fmax(cmax, std::sqrt((lam[e] + 2.0 * mu[e]) / rho[e]));
  }
  // Face media: the average of the two sides' (rho, lam, mu) on interior faces,
  // the element's own on boundary faces; impedances Zp = sqrt(rho (lam + 2 mu)),
  // Zs = sqrt(rho mu) of that medium.
  std::vector<double> fz(4 * 6 * nel);
  const size_t fzs = 6 * (size_t)nel;
  for (long long e = 0; e < nel; ++e) {
    for (int f = 0; f < 6; ++f) {
      const long long k = e * 6 + f;
      const long long o = (c->etoe[k] >= 0 && c->bc[k] == DGW_BC_INTERIOR) ? c->etoe[k] : e;
      const double r = 0.5 * (rho[e] + rho[o]), l = 0.5 * (lam[e] + lam[o]), m = 0.5 * (mu[e] + mu[o]);
      const double zp = std::sqrt(r * (l + 2.0 * m)), zs = std::sqrt(r * m);
      fz[k] = zs;
      fz[fzs + k] = zp - zs;
      fz[2 * fzs + k] = 1.0 / zs;
      fz[3 * fzs + k] = 1.0 / zp - 1.0 / zs;
    }
  }
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  dfree(c->mat);
  dfree(c->ec);
  dfree(c->fz);
  dfree(c->src_w);          // the source weights depend on rho: set the source again
  c->src_elem = -1;
  c->has_material = false;
  DGW_CUDA(c, cudaMalloc(&c->ec, 4 * nel * sizeof(double)), "alloc energy constants");
  DGW_CUDA(c, cudaMemcpyAsync(c->ec, ec.data(), 4 * nel * sizeof(double), cudaMemcpyHostToDevice, c->setup), "copy energy constants");
  if (dgw::fp32_arrays(c->cfg.precision)) {
    std::vector<float> m32(m64.begin(), m64.end());
    std::vector<float> fz32(fz.begin(), fz.end());
    DGW_CUDA(c, cudaMalloc(&c->mat, 3 * nel * sizeof(float)), "alloc material");
    DGW_CUDA(c, cudaMemcpyAsync(c->mat, m32.data(), 3 * nel * sizeof(float), cudaMemcpyHostToDevice, c->setup), "copy material");
    DGW_CUDA(c, cudaMalloc(&c->fz, fz32.size() * sizeof(float)), "alloc face media");
    DGW_CUDA(c, cudaMemcpyAsync(c->fz, fz32.data(), fz32.size() * sizeof(float), cudaMemcpyHostToDevice, c->setup), "copy face media");
  } else {
    DGW_CUDA(c, cudaMalloc(&c->mat, 3 * nel * sizeof(double)), "alloc material");
    DGW_CUDA(c, cudaMemcpyAsync(c->mat, m64.data(), 3 * nel * sizeof(double), cudaMemcpyHostToDevice, c->setup), "copy material");
    DGW_CUDA(c, cudaMalloc(&c->fz, fz.size() * sizeof(double)), "alloc face media");
    DGW_CUDA(c, cudaMemcpyAsync(c->fz, fz.data(), fz.size() * sizeof(double), cudaMemcpyHostToDevice, c->setup), "copy face media");
  }
  DGW_CUDA(c, cudaStreamSynchronize(c->setup), "material upload");
  c->c_max = cmax;
  {
    uint64_t h = 1469598103934665603ull;       // FNV-1a over the three arrays' bytes
    for (const double* a : {rho, lam, mu}) {
      const unsigned char* b = reinterpret_cast<const unsigned char*>(a);
      for (size_t i = 0; i < (size_t)nel * sizeof(double); ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
      }
    }
    c->medium_hash = h;
  }
  c->has_material = true;
  return DGW_OK;
}

static dgw_status ensure_staging(dgw_ctx* c, bool need_res) {
  const size_t bytes = (size_t)c->nel * Np_of(c->cfg.N) * c->m * sizeof(double);
  if (!c->stage_u) DGW_CUDA(c, cudaMalloc(&c->stage_u, bytes), "alloc staging state");
  if (need_res && !c->stage_res) DGW_CUDA(c, cudaMalloc(&c->stage_res, bytes), "alloc staging register");
  return DGW_OK;
}

dgw_status dgw_rhs(dgw_ctx* c, const double* u, double* rhs, double t, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_rhs");
  dgw_status st = ready(c);
  if (st != DGW_OK) return st;
  if (!u || !rhs || (const void*)u == (void*)rhs) return fail(c, DGW_ERR_ARG, "u and rhs must be distinct non-null buffers");
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)c->nel * Np_of(c->cfg.N) * c->m * sizeof(double);
  const bool host = !is_device_ptr(u) || !is_device_ptr(rhs);
  if (!host) return launch_stage(c, u, rhs, nullptr, false, 0.0, 0.0, 0.0, s, nullptr, t);
  if ((st = ensure_staging(c, true)) != DGW_OK) return st;
  DGW_CUDA(c, cudaMemcpyAsync(c->stage_u, u, bytes, cudaMemcpyDefault, s), "copy u in");
  if ((st = launch_stage(c, c->stage_u, c->stage_res, nullptr, false, 0, 0, 0, s, nullptr, t)) != DGW_OK) return st;
  DGW_CUDA(c, cudaMemcpyAsync(rhs, c->stage_res, bytes, cudaMemcpyDefault, s), "copy rhs out");
  DGW_CUDA(c, cudaStreamSynchronize(s), "rhs");
  return DGW_OK;
}

dgw_status dgw_stage(dgw_ctx* c, const double* u_in, double* u_out, double* res, int stage, double t,
                     double dt, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_stage");
  dgw_status st = ready(c);
  if (st != DGW_OK) return st;
  if (stage < 0 || stage > 4) return fail(c, DGW_ERR_ARG, "stage %d outside 0..4", stage);
  if (!u_in || !u_out || !res || (const void*)u_in == (void*)u_out || (void*)u_out == (void*)res ||
      (const void*)u_in == (void*)res)
    return fail(c, DGW_ERR_ARG, "u_in, u_out and res must be distinct non-null buffers");
  if (!is_device_ptr(u_in) || !is_device_ptr(u_out) || !is_device_ptr(res))
    return fail(c, DGW_ERR_ARG, "dgw_stage takes device pointers");
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  return launch_stage(c, u_in, u_out, res, true, kLsrkA[stage], kLsrkB[stage], dt, (cudaStream_t)stream, nullptr,
                      t + kLsrkC[stage] * dt);
}

dgw_status dgw_stage_energy(dgw_ctx* c, const double* u_in, double* u_out, double* res, int stage, double t,
                            double dt, double* energy_out, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_stage_energy");
  dgw_status st = ready(c);
  if (st != DGW_OK) return st;
  if (stage < 0 || stage > 4) return fail(c, DGW_ERR_ARG, "stage %d outside 0..4", stage);
  if (!energy_out) return fail(c, DGW_ERR_ARG, "null energy_out");
  if (!u_in || !u_out || !res || (const void*)u_in == (void*)u_out || (void*)u_out == (void*)res ||
      (const void*)u_in == (void*)res)
    return fail(c, DGW_ERR_ARG, "u_in, u_out and res must be distinct non-null buffers");
  if (!is_device_ptr(u_in) || !is_device_ptr(u_out) || !is_device_ptr(res))
    return fail(c, DGW_ERR_ARG, "dgw_stage_energy takes device pointers");
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = launch_stage(c, u_in, u_out, res, true, kLsrkA[stage], kLsrkB[stage], dt, s, c->stage_partials,
                        t + kLsrkC[stage] * dt)) != DGW_OK)
    return st;
  double* result = c->stage_partials + c->stage_ctas;
  DGW_CUDA(c, dgw::launch_energy_final(c->stage_partials, c->stage_ctas, result + 1, result, s), "energy reduction");
  double value = 0.0;
  DGW_CUDA(c, cudaMemcpyAsync(&value, result, sizeof(double), cudaMemcpyDeviceToHost, s), "copy energy");
  DGW_CUDA(c, cudaStreamSynchronize(s), "stage energy");
  *energy_out = value;
  if (!std::isfinite(*energy_out)) return fail(c, DGW_ERR_UNSTABLE, "energy is not finite");
  return DGW_OK;
}

}  // extern "C"

namespace {

// nsteps LSRK(5,4) steps of u (res: the register, or NULL for the context's
// own); with energy_out, the last stage also accumulates the energy of the
// new state.  The first stage never reads the register (a_0 = 0), so host
// buffers copy only u in.
dgw_status step_impl(dgw_ctx* c, double* u, double* res, double t0, double dt, int nsteps, double* energy_out,
                     void* stream) {
  dgw_status st = ready(c);
  if (st != DGW_OK) return st;
  if (!u || u == res) return fail(c, DGW_ERR_ARG, "u must be non-null and distinct from res");
  if (nsteps < 0) return fail(c, DGW_ERR_ARG, "nsteps must be >= 0");
  if (energy_out && nsteps < 1) return fail(c, DGW_ERR_ARG, "the fused energy needs nsteps >= 1");
  if (!std::isfinite(dt)) return fail(c, DGW_ERR_ARG, "dt must be finite");
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)c->nel * Np_of(c->cfg.N) * c->m * sizeof(double);
  const bool host = !is_device_ptr(u) || (res && !is_device_ptr(res));
  double* ud = u;
  double* rd = res;
  if (host || !res) {
    if ((st = ensure_staging(c, true)) != DGW_OK) return st;
    rd = c->stage_res;
  }
  if (host) {
    ud = c->stage_u;
    DGW_CUDA(c, cudaMemcpyAsync(ud, u, bytes, cudaMemcpyDefault, s), "copy u in");
  }
  double* cur = ud;
  double* nxt = c->u2;
  for (int k = 0; k < nsteps; ++k) {
    const double tk = t0 + k * dt;
    for (int sidx = 0; sidx < 5; ++sidx) {
      double* partials = (energy_out && k == nsteps - 1 && sidx == 4) ? c->stage_partials : nullptr;
      if ((st = launch_stage(c, cur, nxt, rd, true, kLsrkA[sidx], kLsrkB[sidx], dt, s, partials,
                             tk + kLsrkC[sidx] * dt)) != DGW_OK)
        return st;
      double* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  }
  if (cur != ud) DGW_CUDA(c, cudaMemcpyAsync(ud, cur, bytes, cudaMemcpyDeviceToDevice, s), "copy state back");
  if (host) {
    DGW_CUDA(c, cudaMemcpyAsync(u, ud, bytes, cudaMemcpyDefault, s), "copy u out");
    if (res && nsteps > 0) DGW_CUDA(c, cudaMemcpyAsync(res, rd, bytes, cudaMemcpyDefault, s), "copy res out");
  }
  if (energy_out) {
    double* result = c->stage_partials + c->stage_ctas;
    DGW_CUDA(c, dgw::launch_energy_final(c->stage_partials, c->stage_ctas, result + 1, result, s), "energy reduction");
    double value = 0.0;
    DGW_CUDA(c, cudaMemcpyAsync(&value, result, sizeof(double), cudaMemcpyDeviceToHost, s), "copy energy");
    DGW_CUDA(c, cudaStreamSynchronize(s), "step energy");
    *energy_out = value;
    if (!std::isfinite(value)) return fail(c, DGW_ERR_UNSTABLE, "energy is not finite");
  } else if (host) {
    DGW_CUDA(c, cudaStreamSynchronize(s), "step");
  }
  return DGW_OK;
}

}  // namespace

extern "C" {

dgw_status dgw_step(dgw_ctx* c, double* u, double* res, double t0, double dt, int nsteps, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_step");
  return step_impl(c, u, res, t0, dt, nsteps, nullptr, stream);
}

dgw_status dgw_step_energy(dgw_ctx* c, double* u, double* res, double t0, double dt, int nsteps,
                           double* energy_out, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_step_energy");
  if (!energy_out) return fail(c, DGW_ERR_ARG, "null energy_out");
  return step_impl(c, u, res, t0, dt, nsteps, energy_out, stream);
}

dgw_status dgw_energy(dgw_ctx* c, const double* u, double* energy_out, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_energy");
  dgw_status st = ready(c);
  if (st != DGW_OK) return st;
  if (!u || !energy_out) return fail(c, DGW_ERR_ARG, "null argument");
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const double* ud = u;
  if (!is_device_ptr(u)) {
    if ((st = ensure_staging(c, false)) != DGW_OK) return st;
    const size_t bytes = (size_t)c->nel * Np_of(c->cfg.N) * c->m * sizeof(double);
    DGW_CUDA(c, cudaMemcpyAsync(c->stage_u, u, bytes, cudaMemcpyDefault, s), "copy u in");
    ud = c->stage_u;
  }
  double* result = c->partials + dgw::kEnergyBlocks;
  if (c->cfg.system == DGW_SYSTEM_ELASTIC) {
    DGW_CUDA(c, dgw::launch_energy(ud, c->wJ, c->ec, c->nel, Np_of(c->cfg.N), c->partials, result, s),
             "energy kernels");
  } else {
    DGW_CUDA(c, dgw::launch_plain_energy(ud, c->wJ, c->m, c->nel * Np_of(c->cfg.N), c->partials, result, s),
             "energy kernels");
  }
  double value = 0.0;
  DGW_CUDA(c, cudaMemcpyAsync(&value, result, sizeof(double), cudaMemcpyDeviceToHost, s), "copy energy");
  DGW_CUDA(c, cudaStreamSynchronize(s), "energy");
  *energy_out = value;
  if (!std::isfinite(*energy_out)) return fail(c, DGW_ERR_UNSTABLE, "energy is not finite");
  return DGW_OK;
}

dgw_status dgw_source_set(dgw_ctx* c, int64_t element, const double* xi, const double* force, double f0,
                          double t0) {
  if (!c) return fail(nullptr, DGW_ERR_ARG, "null context");
  if (c->cfg.system != DGW_SYSTEM_ELASTIC) return fail(c, DGW_ERR_UNSUPPORTED, "point forces are elastic only");
  if (!c->has_mesh || !c->has_material) return fail(c, DGW_ERR_STATE, "source before mesh and material");
  if (element < 0) {
    dfree(c->src_w);
    c->src_elem = -1;
    return DGW_OK;
  }
  if (element >= c->nel) return fail(c, DGW_ERR_ARG, "source element %lld out of range", (long long)element);
  if (!xi || !force) return fail(c, DGW_ERR_ARG, "null xi or force");
  for (int a = 0; a < 3; ++a)
    if (!(xi[a] >= -1.0 && xi[a] <= 1.0)) return fail(c, DGW_ERR_ARG, "xi must lie in [-1, 1]^3");
  if (!(f0 > 0.0) || !std::isfinite(t0)) return fail(c, DGW_ERR_ARG, "need f0 > 0 and finite t0");
  const int N = c->cfg.N, n = N + 1, Np = Np_of(N);
  if (set_device(c) != DGW_OK) return DGW_ERR_CUDA;
  std::vector<double> wj(Np), rho(1);
  DGW_CUDA(c, cudaMemcpyAsync(wj.data(), c->wJ + (size_t)element * Np, Np * sizeof(double), cudaMemcpyDeviceToHost,
                              c->setup), "copy mass weights");
  DGW_CUDA(c, cudaMemcpyAsync(rho.data(), c->ec + element, sizeof(double), cudaMemcpyDeviceToHost, c->setup),
           "copy density");
  DGW_CUDA(c, cudaStreamSynchronize(c->setup), "copy source data");
  // Lagrange basis values at xi along each axis (product formula).
  double l[3][dgw::kMaxN + 1];
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < n; ++j) {
      double v = 1.0;
      for (int k = 0; k < n; ++k)
        if (k != j) v *= (xi[a] - c->ref.r[k]) / (c->ref.r[j] - c->ref.r[k]);
      l[a][j] = v;
    }
  std::vector<double> w(3 * Np);
  for (int kk = 0; kk < n; ++kk)
    for (int jj = 0; jj < n; ++jj)
      for (int ii = 0; ii < n; ++ii) {
        const int node = ii + n * (jj + n * kk);
        const double phi = l[0][ii] * l[1][jj] * l[2][kk] / (wj[node] * rho[0]);
        for (int q = 0; q < 3; ++q) w[q * Np + node] = force[q] * phi;
      }
  if (!c->src_w) DGW_CUDA(c, cudaMalloc(&c->src_w, 3 * (size_t)dgw::kMaxNp() * sizeof(double)), "alloc source");
  DGW_CUDA(c, cudaMemcpyAsync(c->src_w, w.data(), 3 * Np * sizeof(double), cudaMemcpyHostToDevice, c->setup),
           "copy source");
  DGW_CUDA(c, cudaStreamSynchronize(c->setup), "copy source");
  c->src_elem = element;
  c->src_f0 = f0;
  c->src_t0 = t0;
  return DGW_OK;
}


dgw_status dgw_dt_cfl(dgw_ctx* c, double* dt_out) {
  dgw_status st = ready(c);
  if (st != DGW_OK) return st;
  if (!dt_out) return fail(c, DGW_ERR_ARG, "null argument");
  const double N = c->cfg.N;
  *dt_out = c->cfg.cfl * c->h_min / (c->c_max * N * N);
  return DGW_OK;
}

const char* dgw_last_error(const dgw_ctx* c) {
  if (c) return c->err.c_str();
  return g_error.c_str();
}

}  // extern "C"
