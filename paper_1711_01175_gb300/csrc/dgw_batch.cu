// Batches of solves advanced together (the serving path).
//
// A batch holds solves of one degree, precision and flux, each owned by its
// own context (mesh, medium, source) with caller-owned state and register.
// dgw_batch_create records a CUDA graph of two LSRK steps: ten launches of the
// batched stage kernel (one CTA per tile of all solves; the state alternates
// between the caller's buffer and the context's second buffer and is back in
// the caller's buffer after ten stages) and one launch that advances each
// solve's device time by 2 dt.  The solve descriptors are parameters of the
// stage launches: dgw_batch_set rewrites them, with the grid, in the ten stage
// nodes of the instantiated graph (an update that applies to later replays
// only, so replays already enqueued keep their composition) and enqueues the
// upload of the solves' times and steps on the caller's stream; no new
// recording, no synchronisation.  dgw_batch_run replays the graph.
#include <cmath>
#include <string>
#include <vector>

#include "dgw_internal.cuh"

namespace dgw {

cudaError_t launch_stage_batch_fp64(int N, const BatchLaunch& L, const BatchSet& S, int grid, cudaStream_t s);
cudaError_t launch_stage_batch_mixed(int N, const BatchLaunch& L, const BatchSet& S, int grid, cudaStream_t s);
cudaError_t prepare_stage_batch_fp64(int N);
cudaError_t prepare_stage_batch_mixed(int N);

cudaError_t launch_stage_batch(int N, bool mixed, const BatchLaunch& L, const BatchSet& S, int grid, cudaStream_t s) {
  return mixed ? launch_stage_batch_mixed(N, L, S, grid, s) : launch_stage_batch_fp64(N, L, S, grid, s);
}

cudaError_t prepare_stage_batch(int N, bool mixed) {
  return mixed ? prepare_stage_batch_mixed(N) : prepare_stage_batch_fp64(N);
}

namespace {

// times[i] += nsteps dt[i] over every slot (unused slots hold dt = 0).
__global__ void batch_advance_kernel(double* times, const double* dts, int nsteps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kBatchMaxSolves) times[i] += nsteps * dts[i];
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
  int nsolves = 0;
  int capacity = 0;
  double* d_times = nullptr;             // [kBatchMaxSolves] start time of the current step pair
  double* d_dts = nullptr;               // [kBatchMaxSolves] step sizes (0 in unused slots)
  double h_tdt[2 * dgw::kBatchMaxSolves];   // staging of the times and steps of the last set
  dgw::BatchSet set{};                   // composition of the last set
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphNode_t> stage_nodes;   // the ten stage launches of the graph
  std::vector<cudaKernelNodeParams> stage_params;
  std::vector<dgw::BatchLaunch> stage_launch;   // their fixed parameters
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
  if (precision == DGW_PRECISION_MIXED_TC_FP16 || precision == DGW_PRECISION_MIXED_TC_BF16)
    return bfail(nullptr, DGW_ERR_UNSUPPORTED, "batches run the FP64 and MIXED forms only");
  if (precision != DGW_PRECISION_FP64 && precision != DGW_PRECISION_MIXED)
    return bfail(nullptr, DGW_ERR_ARG, "unknown precision");
  if (flux_tau != 0 && flux_tau != 1) return bfail(nullptr, DGW_ERR_ARG, "flux_tau must be 0 or 1");
  if (max_solves < 1 || max_solves > dgw::kBatchMaxSolves)
    return bfail(nullptr, DGW_ERR_ARG, "max_solves outside 1..DGW_BATCH_MAX_SOLVES");
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
    if (b->d_times) cudaFree(b->d_times);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
    return bfail(nullptr, st, msg);
  };
  cudaError_t e = dgw::prepare_stage_batch(N, precision == DGW_PRECISION_MIXED);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(DGW_ERR_CUDA, std::string("batch kernel set-up: ") + cudaGetErrorString(e));
  if (cudaMalloc(&b->d_times, 2 * dgw::kBatchMaxSolves * sizeof(double)) != cudaSuccess)
    return bail(DGW_ERR_OOM, "batch times");
  b->d_dts = b->d_times + dgw::kBatchMaxSolves;
  if (cudaMemsetAsync(b->d_times, 0, 2 * dgw::kBatchMaxSolves * sizeof(double), b->capture) != cudaSuccess ||
      cudaStreamSynchronize(b->capture) != cudaSuccess)
    return bail(DGW_ERR_CUDA, "batch times");
  // Record two LSRK steps once, for an empty composition.
  int epb = 0, nt = 0;
  dgw::stage_shape(N, &epb, &nt);
  dgw::BatchLaunch L{};
  L.times = b->d_times;
  L.tau = flux_tau ? 1.0 : 0.0;
  dgw::RefElem R;
  dgw::build_ref_elem(N, &R);
  L.w_end_inv = 1.0 / R.w[0];
  L.tau_f = static_cast<float>(L.tau);
  L.hlift_f = static_cast<float>(0.5 * L.w_end_inv);
  for (int i = 0; i < (N + 1) * (N + 1); ++i) L.D[i] = R.D[i];
  L.pf_elems = 1LL * b->sm_count * epb * dgw::stage_pf_tenths(N, b->precision) / 10;
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
      L.first = st == 0 ? 1 : 0;
      e = dgw::launch_stage_batch(N, precision == DGW_PRECISION_MIXED, L, b->set, 1, cs);
    }
  }
  if (e == cudaSuccess) {
    dgw::batch_advance_kernel<<<(dgw::kBatchMaxSolves + 127) / 128, 128, 0, cs>>>(b->d_times, b->d_dts, 2);
    e = cudaGetLastError();
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bail(DGW_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  b->graph = g;
  // The stage launches are the kernel nodes other than the time advance.
  size_t nn = 0;
  e = cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (e == cudaSuccess && nn > 0) e = cudaGraphGetNodes(g, nodes.data(), &nn);
  for (size_t i = 0; i < nn && e == cudaSuccess; ++i) {
    cudaGraphNodeType ty;
    e = cudaGraphNodeGetType(nodes[i], &ty);
    if (e != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp{};
    e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
    if (e == cudaSuccess && kp.func != reinterpret_cast<void*>(&dgw::batch_advance_kernel)) {
      b->stage_nodes.push_back(nodes[i]);
      b->stage_params.push_back(kp);
      b->stage_launch.push_back(*static_cast<const dgw::BatchLaunch*>(kp.kernelParams[0]));
    }
  }
  if (e == cudaSuccess && b->stage_nodes.size() != 10) e = cudaErrorUnknown;
  if (e != cudaSuccess) return bail(DGW_ERR_CUDA, std::string("graph nodes: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) return bail(DGW_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  *out = b;
  return DGW_OK;
}

dgw_status dgw_batch_destroy(dgw_batch* b) {
  if (!b) return DGW_OK;
  cudaSetDevice(b->device);
  drop_graph(b);
  if (b->d_times) cudaFree(b->d_times);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
  return DGW_OK;
}

dgw_status dgw_batch_set(dgw_batch* b, int n, dgw_ctx* const* ctxs, double* const* u, double* const* res,
                         const double* dt, const double* t0, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_batch_set");
  if (!b) return bfail(nullptr, DGW_ERR_ARG, "null batch");
  if (n < 0 || (n > 0 && (!ctxs || !u || !res || !dt || !t0))) return bfail(b, DGW_ERR_ARG, "bad arguments");
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, DGW_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = (cudaStream_t)stream;
  if (n > b->capacity) return bfail(b, DGW_ERR_ARG, "more solves than the batch capacity");
  dgw::BatchSet hs{};
  long long tiles = 0;
  int epb = 0, nt = 0;
  dgw::stage_shape(b->N, &epb, &nt);
  for (int i = 0; i < n; ++i) {
    dgw_ctx* c = ctxs[i];
    if (!c || !c->has_mesh || !c->has_material) return bfail(b, DGW_ERR_STATE, "solve without mesh or material");
    if (c->cfg.system != DGW_SYSTEM_ELASTIC)
      return bfail(b, DGW_ERR_UNSUPPORTED, "solve " + std::to_string(i) + ": batches hold elastic solves only");
    if (c->cfg.N != b->N || c->cfg.precision != b->precision || c->cfg.flux_tau != b->tau || c->device != b->device)
      return bfail(b, DGW_ERR_ARG, "solve " + std::to_string(i) + " differs in degree, precision, flux or device");
    if (!u[i] || !res[i] || u[i] == res[i] || !device_ptr(u[i]) || !device_ptr(res[i]))
      return bfail(b, DGW_ERR_ARG, "solve " + std::to_string(i) + ": u and res must be distinct device buffers");
    if (!(dt[i] > 0.0) || !std::isfinite(t0[i])) return bfail(b, DGW_ERR_ARG, "need dt > 0 and finite t0");
    dgw::BatchSolve& d = hs.s[i];
    d.u[0] = u[i];
    d.u[1] = c->u2;
    d.res = res[i];
    d.geo = c->geo;
    d.fz = c->fz;
    d.vmapP = c->vmapP;
    d.mat = c->mat;
    d.nel = c->nel;
    d.dt = dt[i];
    d.dt_f = static_cast<float>(dt[i]);
    d.src_elem = c->src_elem;
    d.src_w = c->src_w;
    d.src_f0 = c->src_f0;
    d.src_t0 = c->src_t0;
    d.tile0 = tiles;
    tiles += (c->nel + epb - 1) / epb;
  }
  if (tiles > 0x7fffffffLL) return bfail(b, DGW_ERR_ARG, "more than 2^31 - 1 tiles in the batch");
  hs.nsolves = n;
  hs.total_tiles = tiles;
  // Times and steps: a stream-ordered upload (earlier replays on this stream
  // finish first; the runtime stages the pageable source before returning).
  for (int i = 0; i < dgw::kBatchMaxSolves; ++i) {
    b->h_tdt[i] = i < n ? t0[i] : 0.0;
    b->h_tdt[dgw::kBatchMaxSolves + i] = i < n ? dt[i] : 0.0;
  }
  if (cudaMemcpyAsync(b->d_times, b->h_tdt, sizeof(b->h_tdt), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return bfail(b, DGW_ERR_CUDA, "upload batch times");
  // Descriptors and grid (one CTA per tile) of the stage nodes, from the next
  // replay on; replays already enqueued keep the composition they had.
  b->set = hs;
  const unsigned grid = tiles > 0 ? (unsigned)tiles : 1u;
  for (size_t k = 0; k < b->stage_nodes.size(); ++k) {
    cudaKernelNodeParams kp = b->stage_params[k];
    void* args[2] = {&b->stage_launch[k], &b->set};
    kp.kernelParams = args;
    kp.extra = nullptr;
    kp.gridDim = dim3(grid, 1, 1);
    cudaError_t e = cudaGraphExecKernelNodeSetParams(b->exec, b->stage_nodes[k], &kp);
    if (e != cudaSuccess) return bfail(b, DGW_ERR_CUDA, std::string("graph update: ") + cudaGetErrorString(e));
  }
  b->nsolves = n;
  return DGW_OK;
}

dgw_status dgw_batch_run(dgw_batch* b, int npairs, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_batch_run");
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
