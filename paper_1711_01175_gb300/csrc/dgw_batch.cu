// Batches of solves advanced together (the serving path).
//
// A batch holds solves of one degree, precision and flux, each owned by its
// own context (mesh, medium, source) with caller-owned state and register.
// dgw_batch_create records a CUDA graph of two LSRK steps: ten launches of the
// persistent batched stage kernel (every launch covers the tiles of all
// solves; the state alternates between the caller's buffer and the context's
// second buffer and is back in the caller's buffer after ten stages) and one
// launch that advances each solve's device time by 2 dt.  The kernels read
// the batch composition (descriptors, count, tile total) from device memory,
// so dgw_batch_set only enqueues uploads on the caller's stream -- no new
// recording, no synchronisation -- and dgw_batch_run replays the graph.
#include <cmath>
#include <string>
#include <vector>

#include "dgw_internal.cuh"

namespace dgw {

cudaError_t launch_stage_batch_fp64(int N, const BatchLaunch& L, int grid, cudaStream_t s);
cudaError_t launch_stage_batch_mixed(int N, const BatchLaunch& L, int grid, cudaStream_t s);
cudaError_t prepare_stage_batch_fp64(int N, int sm_count, int* grid);
cudaError_t prepare_stage_batch_mixed(int N, int sm_count, int* grid);

cudaError_t launch_stage_batch(int N, bool mixed, const BatchLaunch& L, int grid, cudaStream_t s) {
  return mixed ? launch_stage_batch_mixed(N, L, grid, s) : launch_stage_batch_fp64(N, L, grid, s);
}

cudaError_t prepare_stage_batch(int N, bool mixed, int sm_count, int* grid) {
  return mixed ? prepare_stage_batch_mixed(N, sm_count, grid) : prepare_stage_batch_fp64(N, sm_count, grid);
}

namespace {

__global__ void batch_advance_kernel(const BatchSolve* solves, const BatchHeader* hdr, int nsteps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < hdr->nsolves) *solves[i].t += nsteps * solves[i].dt;
}

// LSRK(5,4) of Carpenter & Kennedy (1994), 2N-storage, five stages, fourth order.
const double kA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                      -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                      1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                      2277821191437.0 / 14882151754819.0};
const double kC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                      2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

}  // namespace
}  // namespace dgw

struct dgw_batch {
  int device = 0;
  int N = 0;
  int precision = 0;
  int tau = 1;
  int sm_count = 0;
  int grid = 0;
  int nsolves = 0;
  long long total_tiles = 0;
  dgw::BatchSolve* d_solves = nullptr;   // [capacity]
  dgw::BatchHeader* d_hdr = nullptr;
  double* d_times = nullptr;             // [capacity]
  int capacity = 0;
  std::vector<dgw::BatchSolve> h_solves;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;   // private stream the graph is recorded on
  std::string err;
};

namespace {

dgw_status bfail(dgw_batch* b, dgw_status st, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    dgw::set_no_context_error(msg);
  return st;
}

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void drop_graph(dgw_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

}  // namespace

extern "C" {

dgw_status dgw_batch_create(dgw_batch** out, int device, int N, int precision, int flux_tau, int max_solves) {
  if (!out) return bfail(nullptr, DGW_ERR_ARG, "null argument");
  *out = nullptr;
  if (N < 1 || N > dgw::kMaxN) return bfail(nullptr, DGW_ERR_ARG, "N outside 1..7");
  if (precision != DGW_PRECISION_FP64 && precision != DGW_PRECISION_MIXED)
    return bfail(nullptr, DGW_ERR_ARG, "unknown precision");
  if (flux_tau != 0 && flux_tau != 1) return bfail(nullptr, DGW_ERR_ARG, "flux_tau must be 0 or 1");
  if (max_solves < 1 || max_solves > (1 << 20)) return bfail(nullptr, DGW_ERR_ARG, "max_solves outside 1..2^20");
  if (cudaSetDevice(device) != cudaSuccess) return bfail(nullptr, DGW_ERR_CUDA, "cudaSetDevice failed");
  dgw_batch* b = new dgw_batch();
  b->device = device;
  b->N = N;
  b->precision = precision;
  b->tau = flux_tau;
  b->capacity = max_solves;
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, device);
  auto bail = [&](dgw_status st, const std::string& msg) {
    drop_graph(b);
    if (b->d_solves) cudaFree(b->d_solves);
    if (b->d_hdr) cudaFree(b->d_hdr);
    if (b->d_times) cudaFree(b->d_times);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
    return bfail(nullptr, st, msg);
  };
  cudaError_t e = dgw::prepare_stage_batch(N, precision == DGW_PRECISION_MIXED, b->sm_count, &b->grid);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(DGW_ERR_CUDA, std::string("batch kernel set-up: ") + cudaGetErrorString(e));
  if (cudaMalloc(&b->d_solves, max_solves * sizeof(dgw::BatchSolve)) != cudaSuccess ||
      cudaMalloc(&b->d_hdr, sizeof(dgw::BatchHeader)) != cudaSuccess ||
      cudaMalloc(&b->d_times, max_solves * sizeof(double)) != cudaSuccess)
    return bail(DGW_ERR_OOM, "batch descriptors");
  dgw::BatchHeader h0{0, 0};
  if (cudaMemcpyAsync(b->d_hdr, &h0, sizeof(h0), cudaMemcpyHostToDevice, b->capture) != cudaSuccess ||
      cudaStreamSynchronize(b->capture) != cudaSuccess)
    return bail(DGW_ERR_CUDA, "batch header");
  // Record two LSRK steps once; the kernels read the composition from device memory.
  int epb = 0, nt = 0;
  dgw::stage_shape(N, &epb, &nt);
  dgw::BatchLaunch L{};
  L.solves = b->d_solves;
  L.hdr = b->d_hdr;
  L.tau = flux_tau ? 1.0 : 0.0;
  dgw::RefElem R;
  dgw::build_ref_elem(N, &R);
  L.w_end_inv = 1.0 / R.w[0];
  for (int i = 0; i < (N + 1) * (N + 1); ++i) L.D[i] = R.D[i];
  L.pf_elems = 2LL * b->sm_count * epb;
  cudaStream_t cs = b->capture;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bail(DGW_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    for (int st = 0; st < 5 && e == cudaSuccess; ++st) {
      L.parity = (5 * k + st) & 1;
      L.step = k;
      L.a = dgw::kA[st];
      L.b = dgw::kB[st];
      L.c = dgw::kC[st];
      e = dgw::launch_stage_batch(N, precision == DGW_PRECISION_MIXED, L, b->grid, cs);
    }
  }
  if (e == cudaSuccess) {
    dgw::batch_advance_kernel<<<(max_solves + 127) / 128, 128, 0, cs>>>(b->d_solves, b->d_hdr, 2);
    e = cudaGetLastError();
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bail(DGW_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) return bail(DGW_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  *out = b;
  return DGW_OK;
}

dgw_status dgw_batch_destroy(dgw_batch* b) {
  if (!b) return DGW_OK;
  cudaSetDevice(b->device);
  drop_graph(b);
  if (b->d_solves) cudaFree(b->d_solves);
  if (b->d_hdr) cudaFree(b->d_hdr);
  if (b->d_times) cudaFree(b->d_times);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
  return DGW_OK;
}

dgw_status dgw_batch_set(dgw_batch* b, int n, dgw_ctx* const* ctxs, double* const* u, double* const* res,
                         const double* dt, const double* t0, void* stream) {
  if (!b) return bfail(nullptr, DGW_ERR_ARG, "null batch");
  if (n < 0 || (n > 0 && (!ctxs || !u || !res || !dt || !t0))) return bfail(b, DGW_ERR_ARG, "bad arguments");
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, DGW_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<dgw::BatchSolve> hs(n);
  long long tiles = 0;
  int epb = 0, nt = 0;
  dgw::stage_shape(b->N, &epb, &nt);
  for (int i = 0; i < n; ++i) {
    dgw_ctx* c = ctxs[i];
    if (!c || !c->has_mesh || !c->has_material) return bfail(b, DGW_ERR_STATE, "solve without mesh or material");
    if (c->cfg.N != b->N || c->cfg.precision != b->precision || c->cfg.flux_tau != b->tau || c->device != b->device)
      return bfail(b, DGW_ERR_ARG, "solve " + std::to_string(i) + " differs in degree, precision, flux or device");
    if (!u[i] || !res[i] || u[i] == res[i] || !device_ptr(u[i]) || !device_ptr(res[i]))
      return bfail(b, DGW_ERR_ARG, "solve " + std::to_string(i) + ": u and res must be distinct device buffers");
    if (!(dt[i] > 0.0) || !std::isfinite(t0[i])) return bfail(b, DGW_ERR_ARG, "need dt > 0 and finite t0");
    dgw::BatchSolve& d = hs[i];
    d.u[0] = u[i];
    d.u[1] = c->u2;
    d.res = res[i];
    d.geo = c->geo;
    d.fz = c->fz;
    d.vmapP = c->vmapP;
    d.mat = c->mat;
    d.nel = c->nel;
    d.dt = dt[i];
    d.src_elem = c->src_elem;
    d.src_w = c->src_w;
    d.src_f0 = c->src_f0;
    d.src_t0 = c->src_t0;
    d.tile0 = tiles;
    tiles += (c->nel + epb - 1) / epb;
  }
  if (n > b->capacity) return bfail(b, DGW_ERR_ARG, "more solves than the batch capacity");
  for (int i = 0; i < n; ++i) hs[i].t = b->d_times + i;
  // Stream-ordered uploads: earlier replays on this stream finish first.  The
  // host copies live in the batch until the next set (pageable sources are
  // staged by the runtime before the call returns).
  b->h_solves = hs;
  dgw::BatchHeader hdr{n, tiles};
  if ((n > 0 && cudaMemcpyAsync(b->d_solves, b->h_solves.data(), n * sizeof(dgw::BatchSolve), cudaMemcpyHostToDevice,
                                s) != cudaSuccess) ||
      (n > 0 && cudaMemcpyAsync(b->d_times, t0, n * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemcpyAsync(b->d_hdr, &hdr, sizeof(hdr), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return bfail(b, DGW_ERR_CUDA, "upload batch descriptors");
  b->nsolves = n;
  b->total_tiles = tiles;
  return DGW_OK;
}

dgw_status dgw_batch_run(dgw_batch* b, int npairs, void* stream) {
  if (!b) return bfail(nullptr, DGW_ERR_ARG, "null batch");
  if (npairs < 0) return bfail(b, DGW_ERR_ARG, "npairs must be >= 0");
  if (b->nsolves == 0 || npairs == 0) return DGW_OK;
  if (!b->exec) return bfail(b, DGW_ERR_STATE, "batch has no recorded graph");
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, DGW_ERR_CUDA, "cudaSetDevice failed");
  for (int i = 0; i < npairs; ++i) {
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return bfail(b, DGW_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  }
  return DGW_OK;
}

const char* dgw_batch_last_error(const dgw_batch* b) { return b ? b->err.c_str() : dgw_last_error(nullptr); }

}  // extern "C"
