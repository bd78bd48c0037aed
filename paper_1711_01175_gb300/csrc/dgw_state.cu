// Checkpoint and resume of a solve: a self-describing host copy of its state
// (u, the Runge-Kutta register, time and step) that a context on the same
// mesh can load back bit for bit.
#include <cstring>
#include <string>

#include "dgw_internal.cuh"

namespace {

constexpr char kMagic[8] = {'D', 'G', 'W', 'S', 'T', 'A', 'T', '1'};

// Checkpoint layout: this header, then u ([m][nel][Np] doubles) and, when
// has_res, the register (same shape).  All fields little-endian as written by
// the host.
struct StateHeader {
  char magic[8];
  uint32_t abi;
  uint32_t has_res;
  int32_t N;
  int32_t m;
  int64_t nel;
  int64_t step;
  double t;
  uint64_t mesh_fingerprint;   // FNV-1a over degree, system, connectivity, boundary tags, h_min, c_max, medium
  uint64_t payload_hash;       // FNV-1a over the payload's 64-bit words
  uint64_t payload_bytes;
  uint64_t reserved;
};
static_assert(sizeof(StateHeader) == 80, "checkpoint header layout");

constexpr uint64_t kFnvOffset = 1469598103934665603ull;
constexpr uint64_t kFnvPrime = 1099511628211ull;

uint64_t fnv_bytes(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= kFnvPrime;
  }
  return h;
}

uint64_t fnv_words(const void* p, size_t bytes) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  uint64_t h = kFnvOffset;
  for (size_t i = 0; i + 8 <= bytes; i += 8) {
    uint64_t w;
    std::memcpy(&w, b + i, 8);
    h ^= w;
    h *= kFnvPrime;
  }
  return h;
}

uint64_t mesh_fingerprint(const dgw_ctx* c) {
  uint64_t h = kFnvOffset;
  const int32_t head[3] = {c->cfg.N, c->cfg.system, c->m};
  h = fnv_bytes(h, head, sizeof head);
  h = fnv_bytes(h, &c->nel, sizeof c->nel);
  h = fnv_bytes(h, c->etoe.data(), c->etoe.size() * sizeof(int64_t));
  h = fnv_bytes(h, c->etof.data(), c->etof.size());
  h = fnv_bytes(h, c->bc.data(), c->bc.size());
  h = fnv_bytes(h, &c->h_min, sizeof c->h_min);
  h = fnv_bytes(h, &c->c_max, sizeof c->c_max);
  h = fnv_bytes(h, &c->medium_hash, sizeof c->medium_hash);
  return h;
}

dgw_status sfail(dgw_ctx* c, dgw_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    dgw::set_no_context_error(msg);
  return st;
}

size_t state_doubles(const dgw_ctx* c) {
  const size_t n = c->cfg.N + 1;
  return (size_t)c->m * c->nel * n * n * n;
}

}  // namespace

extern "C" {

dgw_status dgw_state_bytes(dgw_ctx* c, int with_res, size_t* bytes) {
  if (!c) return sfail(nullptr, DGW_ERR_ARG, "null context");
  if (!bytes) return sfail(c, DGW_ERR_ARG, "null output");
  if (!c->has_mesh) return sfail(c, DGW_ERR_STATE, "checkpoint before the mesh");
  *bytes = sizeof(StateHeader) + (with_res ? 2 : 1) * state_doubles(c) * sizeof(double);
  return DGW_OK;
}

dgw_status dgw_get_state(dgw_ctx* c, const double* u, const double* res, double t, int64_t step, void* buf,
                         size_t buf_bytes, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_get_state");
  if (!c) return sfail(nullptr, DGW_ERR_ARG, "null context");
  if (!c->has_mesh) return sfail(c, DGW_ERR_STATE, "checkpoint before the mesh");
  if (!u || !buf) return sfail(c, DGW_ERR_ARG, "null u or buffer");
  const size_t sb = state_doubles(c) * sizeof(double);
  const size_t need = sizeof(StateHeader) + (res ? 2 : 1) * sb;
  if (buf_bytes < need)
    return sfail(c, DGW_ERR_ARG, "checkpoint buffer of " + std::to_string(buf_bytes) + " bytes, " +
                                     std::to_string(need) + " needed");
  if (cudaSetDevice(c->device) != cudaSuccess) return sfail(c, DGW_ERR_CUDA, "cudaSetDevice");
  unsigned char* out = static_cast<unsigned char*>(buf);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(out + sizeof(StateHeader), u, sb, cudaMemcpyDefault, s);
  if (e == cudaSuccess && res) e = cudaMemcpyAsync(out + sizeof(StateHeader) + sb, res, sb, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return sfail(c, DGW_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
  StateHeader h{};
  std::memcpy(h.magic, kMagic, 8);
  h.abi = DGW_ABI_VERSION;
  h.has_res = res ? 1u : 0u;
  h.N = c->cfg.N;
  h.m = c->m;
  h.nel = c->nel;
  h.step = step;
  h.t = t;
  h.mesh_fingerprint = mesh_fingerprint(c);
  h.payload_bytes = need - sizeof(StateHeader);
  h.payload_hash = fnv_words(out + sizeof(StateHeader), h.payload_bytes);
  std::memcpy(out, &h, sizeof h);
  return DGW_OK;
}

dgw_status dgw_set_state(dgw_ctx* c, const void* buf, size_t buf_bytes, double* u, double* res, double* t,
                         int64_t* step, void* stream) {
  dgw::NvtxRange nvtx_range("dgw_set_state");
  if (!c) return sfail(nullptr, DGW_ERR_ARG, "null context");
  if (!c->has_mesh) return sfail(c, DGW_ERR_STATE, "resume before the mesh");
  if (!buf || !u) return sfail(c, DGW_ERR_ARG, "null buffer or u");
  if (buf_bytes < sizeof(StateHeader)) return sfail(c, DGW_ERR_ARG, "checkpoint shorter than its header");
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, kMagic, 8) != 0) return sfail(c, DGW_ERR_ARG, "not a checkpoint of this library");
  if (h.abi != DGW_ABI_VERSION)
    return sfail(c, DGW_ERR_ARG, "checkpoint of ABI " + std::to_string(h.abi) + ", library ABI " +
                                     std::to_string(DGW_ABI_VERSION));
  if (h.N != c->cfg.N || h.m != c->m || h.nel != c->nel)
    return sfail(c, DGW_ERR_ARG, "checkpoint of another degree, system or element count");
  if (h.mesh_fingerprint != mesh_fingerprint(c)) return sfail(c, DGW_ERR_ARG, "checkpoint of another mesh or medium");
  const size_t sb = state_doubles(c) * sizeof(double);
  if (h.payload_bytes != (h.has_res ? 2 : 1) * sb || buf_bytes < sizeof(StateHeader) + h.payload_bytes)
    return sfail(c, DGW_ERR_ARG, "checkpoint payload size does not match the mesh or the buffer");
  if (res && !h.has_res) return sfail(c, DGW_ERR_ARG, "the checkpoint holds no register");
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  if (fnv_words(in + sizeof(StateHeader), h.payload_bytes) != h.payload_hash)
    return sfail(c, DGW_ERR_ARG, "checkpoint payload does not match its checksum");
  if (cudaSetDevice(c->device) != cudaSuccess) return sfail(c, DGW_ERR_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(u, in + sizeof(StateHeader), sb, cudaMemcpyDefault, s);
  if (e == cudaSuccess && res) e = cudaMemcpyAsync(res, in + sizeof(StateHeader) + sb, sb, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return sfail(c, DGW_ERR_CUDA, std::string("resume copy: ") + cudaGetErrorString(e));
  if (t) *t = h.t;
  if (step) *step = h.step;
  return DGW_OK;
}

}  // extern "C"
