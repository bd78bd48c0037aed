// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dgw.h"

namespace dgw {

// NVTX range over one library call (header-only NVTX3: inert unless a
// profiler such as Nsight Systems or ncu --nvtx is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxN = 7;
constexpr int kFields = 9;
constexpr int kMaxNp() { return (kMaxN + 1) * (kMaxN + 1) * (kMaxN + 1); }

// Reference element on the host: GLL nodes/weights and the 1-D derivative
// matrix D[i*(N+1)+j] = l_j'(r_i).
struct RefElem {
  int N = 0;
  double r[kMaxN + 1] = {};
  double w[kMaxN + 1] = {};
  double D[(kMaxN + 1) * (kMaxN + 1)] = {};
};
bool build_ref_elem(int N, RefElem* out);

// Elements per CTA and threads per CTA of the fused stage kernel, per degree.
template <int N>
struct Shape {
  static constexpr int n = N + 1;
  static constexpr int Np = n * n * n;
  static constexpr int nf = n * n;
  static constexpr int EPB = (N == 1) ? 16 : (N == 2) ? 9 : (N == 3) ? 4 : 1;
  static constexpr int NTILE = EPB * Np;
  static constexpr int NT = ((NTILE + 31) / 32) * 32;
  static constexpr int NFACE_ITEMS = EPB * 6 * nf;
};

// Device-side checks of the debug build (compiled with -DDGW_DEBUG_CHECKS): a
// stage kernel records the first fault it meets in the context's fault word
// (code << 56 | element) and counts them, and skips the access a bad index
// would make instead of performing it.
#ifdef DGW_DEBUG_CHECKS
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif
enum { kFaultNone = 0, kFaultNonFiniteState = 1, kFaultNeighbourIndex = 2 };

__device__ __forceinline__ void debug_record(unsigned long long* fault, int code, long long element) {
  if (fault == nullptr) return;
  atomicAdd(fault + 1, 1ull);
  atomicCAS(fault, 0ull, (static_cast<unsigned long long>(code) << 56) | static_cast<unsigned long long>(element));
}

// Neighbour-map sentinels for boundary faces (the map holds e*Np + node otherwise).
constexpr int kGhostFreeSurface = -1;
constexpr int kGhostAbsorbing = -2;

// Arguments of one fused stage launch.  Real is double (FP64 path) or float
// (mixed path) for the geometry, face and material arrays.
struct StageParams {
  const double* u_in;     // [9][nel][Np]
  double* out;            // rhs (rhs mode) or u_out (LSRK mode), [9][nel][Np]
  double* res;            // LSRK register [9][nel][Np] (LSRK mode only)
  const void* geo;        // Real [10][nel][Np]: Ja^i_k at 3*i+k, then 1/J
  const void* fz;         // Real [4][nel*6]: Zs, Zp-Zs, 1/Zs, 1/Zp-1/Zs of the face medium
  const int* vmapP;       // [nel][6*nf]: neighbour flat node index or ghost sentinel
  const void* mat;        // Real [3][nel]: 1/rho, lambda, mu
  long long nel;
  double a, b, dt;        // LSRK coefficients of this stage and the step size
  double tau;             // 0 central, 1 upwind
  double w_end_inv;       // 1 / w_0 (GLL end weight)
  double* energy_partials;  // LSRK mode, optional: one partial sum of w J u_out^T Q u_out per CTA
  const double* wJ;         // [nel][Np] (with energy_partials)
  const double* ec;         // [4][nel] energy constants (with energy_partials)
  long long pf_elems;       // L2 prefetch distance in elements (0: off)
  double* grad_el;          // GRAD mode: [3][nel] element terms (accumulated)
  double* grad_face;        // GRAD mode: [2][nel*6*nf] face-node terms for Zs, Zp (accumulated)
  long long src_elem;       // element holding the point force, -1 for none
  double src_amp;           // Ricker amplitude R(t + c_s dt) of this stage
  const double* src_w;      // [3][Np]: F_q l_j(xi_s) / (rho w_j J_j)
  // FP32 copies of dt, tau and w_end_inv / 2, and a == 0, set by the launcher so
  // that the FP32 path reads them from the constant bank without conversions.
  float dt_f, tau_f, hlift_f;
  int first;
  double beta[3];           // transport velocity (generic-system kernel only)
  int self_only;            // generic-system kernel: neighbour states taken as zero (L_K^self)
  unsigned long long* fault;  // debug build: [first fault, count] (NULL: not recorded)
  double* rout;             // FP64 LSRK mode, optional: dt (K u + f) before Q^{-1} [9][nel][Np];
                            // GRAD_FACE mode: read from there
  double D[(kMaxN + 1) * (kMaxN + 1)];
};

// Fill the FP32 copies of a stage's scalar parameters.
inline void finish_stage_params(StageParams& p) {
  p.dt_f = static_cast<float>(p.dt);
  p.tau_f = static_cast<float>(p.tau);
  p.hlift_f = static_cast<float>(0.5 * p.w_end_inv);
  p.first = p.a == 0.0 ? 1 : 0;
}

// Solves per batch.  Their descriptors travel in the stage kernel's parameters
// (constant bank: uniform, re-loadable, no registers held across the tile).
constexpr int kBatchMaxSolves = 128;

// One solve of a batch.
struct BatchSolve {
  double* u[2];           // state ping-pong: u[0] is the caller's state, u[1] the context's second buffer
  double* res;            // LSRK register
  const void* geo;
  const void* fz;
  const int* vmapP;
  const void* mat;
  long long nel;
  double dt;
  float dt_f;             // FP32 copy of dt
  long long src_elem;
  const double* src_w;
  double src_f0, src_t0;
  long long tile0;        // first batch tile of this solve
};

// Composition of a batch: the solves in tile order.
struct BatchSet {
  int nsolves;
  long long total_tiles;
  BatchSolve s[kBatchMaxSolves];
};

// One launch of the batched stage kernel (fixed when the graph is recorded).
struct BatchLaunch {
  const double* times;    // [kBatchMaxSolves] device start time of the current step pair
  int parity;             // stage index within the replayed step pair, mod 2
  int step;               // step within the pair (0 or 1)
  double a, b, c;         // LSRK coefficients of this stage
  double tau;
  double w_end_inv;
  float tau_f, hlift_f;   // FP32 copies of tau and w_end_inv / 2
  int first;              // a == 0
  long long pf_elems;
  double D[(kMaxN + 1) * (kMaxN + 1)];
};

// Launchers implemented in dgw_stage_fp64.cu / dgw_stage_mixed.cu.
cudaError_t launch_stage_batch(int N, bool mixed, const BatchLaunch& L, const BatchSet& S, int grid, cudaStream_t s);
cudaError_t prepare_stage_batch(int N, bool mixed);
cudaError_t launch_stage_fp64(int N, bool lsrk, const StageParams& p, cudaStream_t s);
cudaError_t launch_stage_mixed(int N, bool lsrk, const StageParams& p, cudaStream_t s);
// Mixed path with the volume term's derivative contractions on the tensor cores
// (split FP16 or BF16 operands, FP32 accumulation): fmt is DGW_PRECISION_MIXED_TC_FP16
// or DGW_PRECISION_MIXED_TC_BF16 (dgw_stage_mixed_tc.cu).
cudaError_t launch_stage_mixed_tc(int N, int fmt, bool lsrk, const StageParams& p, cudaStream_t s);
// Precisions whose geometry, face and material arrays are FP32.
inline bool fp32_arrays(int precision) { return precision != DGW_PRECISION_FP64; }
// L2 bulk prefetch distance of the stage kernels, in tenths of one CTA per SM
// ahead (StageParams::pf_elems = SMs x elements per CTA x tenths / 10).
// FP64: one CTA per SM (its stage is bound by the FP64 pipe; 0.5 and 1 time alike
// at N = 4 and 7).  FP32 CUDA-core stage: the fastest of 0 (off), 0.1, 0.2, 0.3,
// 0.5 and 1 at each degree on 64^3 (N <= 4), 56^3 (N = 5, 6) and 48^3 (N = 7);
// at N = 3, 5, 6 and 7 the kernel's L1 prefetch of the neighbour traces covers
// the gather and an L2 prefetch ahead only evicts traces before they are
// gathered.  Tensor-core forms (no L1 prefetch): 0.2 at N = 7 (the fastest of 0,
// 0.2, 0.5 and 1 on 48^3), one CTA per SM elsewhere (0.2 to 1 alike at N = 4).
inline int stage_pf_tenths(int N, int precision) {
  static const int kMixed[8] = {10, 2, 2, 0, 10, 0, 0, 0};
  if (precision == DGW_PRECISION_MIXED) return kMixed[N];
  if (precision != DGW_PRECISION_FP64 && N == 7) return 2;
  return 10;
}
cudaError_t launch_stage_adjoint(int N, int mode, const StageParams& p, cudaStream_t s);   // mode 2: ADJ, 3: GRAD
// GRAD (params g) then ADJ (params a) on every tile, in one launch.
cudaError_t launch_stage_adjgrad(int N, const StageParams& g, const StageParams& a, cudaStream_t s);
void stage_shape(int N, int* epb, int* threads);

// Geometry (dgw_geometry.cu).
struct GeometryOut {
  double* geo;       // [10][nel][Np]  Ja (9) then 1/J
  double* wJ;        // [nel][Np]       w_i w_j w_k J
  double* minJ;      // [nel]
};
cudaError_t launch_geometry(int N, const double* x, long long nel, const double* D, const double* w,
                            const GeometryOut& out, cudaStream_t s);
cudaError_t launch_to_float(const double* src, float* dst, size_t n, cudaStream_t s);

// Energy (dgw_energy.cu): partial sums per block, then one final block.
constexpr int kEnergyBlocks = 152 * 4;
constexpr int kEnergyThreads = 256;
cudaError_t launch_energy(const double* u, const double* wJ, const double* ec, long long nel, int Np,
                          double* partials, double* result, cudaStream_t s);
// Generic Friedrichs systems (dgw_friedrichs.cu): stage launch (FP64) and the
// energy 1/2 sum w J |u|^2 of an m-field state (partials: kEnergyBlocks doubles).
cudaError_t launch_friedrichs(int system, int N, bool lsrk, const StageParams& p, cudaStream_t s);
cudaError_t launch_plain_energy(const double* u, const double* wJ, int m, long long total, double* partials,
                                double* result, cudaStream_t s);

// Free the iHDG-II buffers of a context (dgw_ihdg.cu).
void ihdg_release(dgw_ctx* c);

// Sum nparts partials into *result (x 1/2); scratch holds kEnergyBlocks doubles.
cudaError_t launch_energy_final(const double* partials, int nparts, double* scratch, double* result,
                                cudaStream_t s);

// Message storage of calls without a context (read by dgw_last_error(NULL)).
void set_no_context_error(const std::string& msg);

}  // namespace dgw

struct dgw_ctx {
  int device = 0;
  int sm_count = 0;
  cudaStream_t setup = nullptr;    // private non-blocking stream for uploads and geometry
  dgw_config cfg{};
  int m = 9;                       // fields of the system (9 elastic, 1 transport, 3 shallow water)
  dgw::RefElem ref;
  long long nel = 0;
  bool has_mesh = false;
  bool has_material = false;
  // device memory owned by the context
  void* geo = nullptr;       // Real [10][nel][Np]
  void* fz = nullptr;        // Real [4][nel*6] face impedance constants
  int* vmapP = nullptr;      // [nel][6*nf]
  void* mat = nullptr;       // Real [3][nel]
  double* ec = nullptr;      // [4][nel] energy constants: rho, 1/(2 mu), lam/(3 lam + 2 mu), 1/mu
  double* wJ = nullptr;      // [nel][Np]
  double* u2 = nullptr;      // second state buffer for the stage ping-pong
  double* partials = nullptr;  // energy partial sums + result slot
  double* stage_partials = nullptr;  // per-CTA energy partials of a fused stage, result slot, reduction scratch
  unsigned long long* fault = nullptr;  // debug build: [first fault, count] of the stage kernels
  int stage_ctas = 0;
  double* stage_u = nullptr;   // host-pointer staging buffers
  double* stage_res = nullptr;
  double* src_w = nullptr;     // point-force weights [3][Np] (device)
  long long src_elem = -1;
  double src_f0 = 0.0, src_t0 = 0.0;
  std::vector<int64_t> etoe;   // host copy of the connectivity (face media)
  std::vector<int8_t> etof;
  std::vector<int8_t> bc;
  // receivers and adjoint scratch
  int rec_n = 0;
  long long* rec_elem = nullptr;     // [rec_n]
  double* rec_w = nullptr;           // [rec_n][Np] Lagrange basis at the receiver
  double* adj_scratch = nullptr;
  size_t adj_scratch_bytes = 0;
  double* adj_gface = nullptr;
  size_t adj_gface_bytes = 0;
  long long* etoe_d = nullptr;
  signed char* etof_d = nullptr;
  double h_min = 0.0;
  double c_max = 0.0;
  uint64_t medium_hash = 0;          // FNV-1a of the uploaded (rho, lambda, mu) (checkpoint fingerprint)
  // iHDG-II (transport): inverses of sigma I - L_K^self, transposed, and the
  // neighbour-coupling coefficient of every face node
  double* ihdg_inv = nullptr;        // [nel][Np][Np], entry (e, j, i) = inverse(e)[i][j]
  double* ihdg_cf = nullptr;         // [nel][6*nf]
  double* ihdg_part = nullptr;       // per-element partial sums + result + scratch
  double* ihdg_u2 = nullptr;         // second iterate buffer [nel][Np]
  double ihdg_sigma = 0.0;
  bool ihdg_ready = false;
  std::string err;
};
