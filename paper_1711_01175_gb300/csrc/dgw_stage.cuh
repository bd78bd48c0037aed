// Fused DG stage kernel: split-form volume term, face gather + upwind flux,
// diagonal GLL lift, Q^{-1}, and (optionally) the 2N-storage Runge-Kutta update.
//
// One CTA holds EPB elements; thread t owns node t % Np of element t / Np.
//   1. u of the tile (FP64 in HBM) -> shared memory in Real, with the metric
//      terms (node-major packed tiles, 16-byte vector access).
//   2. Volume term per direction i (eq. LPDE in curvilinear split form):
//        acc += D_i (A(Ja^i) u)   [conservative part]
//        acc += A(Ja^i) (D_i u)   [non-conservative part]
//      and vol = -1/2 * (1/J) * acc, with A(m)u = -(sigma m, Voigt(sym(m (x) v))).
//      A is linear in m, so along the line through node a both parts are
//      sum_b A(D_ab (Ja^i_a + Ja^i_b)) u_b, accumulated from the state and
//      metric tiles (no staging, no barrier between directions); FP64 from
//      N = 6 on stages A(Ja^i)u instead, which takes fewer FP64 operations.
//   3. Face items (EPB*6*nf of them, spread over all threads): own trace from
//      smem, neighbour trace from HBM/L2 through the neighbour map (FP32 tiles
//      of several elements: from smem when the neighbour is in the tile) or
//      the boundary ghost, flux difference 1/2 (A(m) - tau S(m))(u^- - u^+) with
//      m = n sJ the scaled outward normal and S(m) = sJ Q|Q^{-1}A(n)| the
//      impedance-weighted upwind stabilisation of the face medium -- the upwind
//      HDG flux of eq. RiemannFluxBoth (for the flux matrix Q^{-1}A(n)) with the
//      trace eliminated by eq. HDGeqn/iHDGtrace -- scaled by the lift factor
//      (1/J)/w_0 and staged in smem.
//   4. Each node adds the lifted flux of the faces it lies on, applies
//      Q^{-1} = diag(1/rho, C_V), then writes rhs or performs
//      res <- a res + dt rhs, u_out <- u_in + b res in FP64 (optionally
//      accumulating the energy of u_out for a fixed-order block sum).
#pragma once

#include <atomic>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dgw_internal.cuh"

namespace dgw {

// out = A_+(m) w with A(m) = -A_+(m):  (sigma m, Voigt(sym(m (x) v))).
template <typename Real>
__device__ __forceinline__ void apply_Apos(Real m1, Real m2, Real m3, const Real* w, Real* out) {
  out[0] = m1 * w[3] + m2 * w[8] + m3 * w[7];
  out[1] = m1 * w[8] + m2 * w[4] + m3 * w[6];
  out[2] = m1 * w[7] + m2 * w[6] + m3 * w[5];
  out[3] = m1 * w[0];
  out[4] = m2 * w[1];
  out[5] = m3 * w[2];
  out[6] = m2 * w[2] + m3 * w[1];
  out[7] = m1 * w[2] + m3 * w[0];
  out[8] = m1 * w[1] + m2 * w[0];
}

// acc += A_+(m) w.
template <typename Real>
__device__ __forceinline__ void acc_Apos(Real m1, Real m2, Real m3, const Real* w, Real* acc) {
  acc[0] += m1 * w[3];
  acc[0] += m2 * w[8];
  acc[0] += m3 * w[7];
  acc[1] += m1 * w[8];
  acc[1] += m2 * w[4];
  acc[1] += m3 * w[6];
  acc[2] += m1 * w[7];
  acc[2] += m2 * w[6];
  acc[2] += m3 * w[5];
  acc[3] += m1 * w[0];
  acc[4] += m2 * w[1];
  acc[5] += m3 * w[2];
  acc[6] += m2 * w[2];
  acc[6] += m3 * w[1];
  acc[7] += m1 * w[2];
  acc[7] += m3 * w[0];
  acc[8] += m1 * w[1];
  acc[8] += m2 * w[0];
}

// FP64 -> FP32 (round half up on the 29 dropped mantissa bits, flush below
// the smallest normal float, overflow to infinity) and FP32 -> FP64 (exact)
// with integer instructions.  The GB300 FP64 pipe, which also executes the
// F2F conversions, issues about two operations per clock per SM; integer
// operations are much wider.  Narrowing works on the two 32-bit halves: a
// funnel shift lines up the low 9 exponent bits and the top 23 mantissa bits,
// and subtracting 0x180 << 23 rebiases the exponent (1023 - 127 = 896 = 0x380,
// which is 0x180 modulo 2^9) wherever the result is a normal float.
__device__ __forceinline__ float narrow_int(double d) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(d));
  const unsigned lo = static_cast<unsigned>(__double2loint(d));
  const unsigned ahi = hi & 0x7fffffffu;
  unsigned f = __funnelshift_l(lo, ahi, 3) - 0xC0000000u + ((lo >> 28) & 1u);
  const unsigned e11 = ahi >> 20;
  f = (e11 - 897u <= 253u) ? f : (e11 < 897u ? 0u : 0x7f800000u);
  return __uint_as_float(f | (hi & 0x80000000u));
}

__device__ __forceinline__ double widen_int(float x) {
  // exponent + 896 and mantissa << 29 on the two 32-bit halves
  const unsigned u = __float_as_uint(x);
  const unsigned a = u & 0x7fffffffu;
  const unsigned e = a >> 23;
  unsigned hi = (a >> 3) + (e == 255u ? (1792u << 20) : (896u << 20));
  unsigned lo = u << 29;
  hi = e == 0u ? 0u : hi;
  lo = e == 0u ? 0u : lo;
  return __hiloint2double(static_cast<int>(hi | (u & 0x80000000u)), static_cast<int>(lo));
}

// A scalar parameter in the path's precision: the double, or its FP32 copy.
template <typename Real>
__device__ __forceinline__ Real pick(double d, float f) {
  if constexpr (std::is_same<Real, double>::value) {
    return d;
  } else {
    return f;
  }
}

template <typename Real>
__device__ __forceinline__ Real to_real(double d) {
  if constexpr (std::is_same<Real, double>::value) {
    return d;
  } else {
    return narrow_int(d);
  }
}

// Node-major packed tiles: PK Reals per node, read and written as 16-byte
// vectors (3 x float4 for FP32, 5 x double2 for FP64).  Strides of 48 B and
// 80 B keep eight consecutive nodes on distinct 16-byte bank groups.
template <typename Real>
struct Pack;
template <>
struct Pack<float> {
  static constexpr int PK = 12;
  static __device__ __forceinline__ void load9(const float* p, float* v) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    const float4 c = reinterpret_cast<const float4*>(p)[2];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    v[8] = c.x; v[9] = c.y;
  }
  static __device__ __forceinline__ void store10(float* p, const float* v) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
    reinterpret_cast<float4*>(p)[2] = make_float4(v[8], v[9], 0.f, 0.f);
  }
};
template <>
struct Pack<double> {
  static constexpr int PK = 10;
  static __device__ __forceinline__ void load9(const double* p, double* v) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const double2 a = reinterpret_cast<const double2*>(p)[k];
      v[2 * k] = a.x;
      v[2 * k + 1] = a.y;
    }
  }
  static __device__ __forceinline__ void store10(double* p, const double* v) {
#pragma unroll
    for (int k = 0; k < 5; ++k) reinterpret_cast<double2*>(p)[k] = make_double2(v[2 * k], v[2 * k + 1]);
  }
};

// Hint: bring [lo, hi) (rounded out to 16 B) into L2 with one bulk prefetch.
// Callers keep the rounded range inside the buffer.
__device__ __forceinline__ void prefetch_l2(const void* lo, const void* hi) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(lo) & ~15ull;
  const unsigned long long b = (reinterpret_cast<unsigned long long>(hi) + 15ull) & ~15ull;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a), "r"((unsigned)(b - a)) : "memory");
}

// Hint: bring the line holding a into L1.
__device__ __forceinline__ void prefetch_l1(const void* a) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
}

// Volume-term form.  Combined: per direction and line node b, A_+(D_ab (m_a + m_b)) u_b
// (24 operations).  Staged: A_+(m) u of the tile staged in shared memory, then
// the two contractions and A_+(m_a) applied to D u (36 + 18 n operations per
// node and direction, two barriers per direction).  FP64 is bound by its FP64
// pipe and takes the staged form where it has fewer operations (n >= 7); FP32
// always takes the combined form (fewer instructions, no barriers).
template <int N, typename Real>
__host__ __device__ constexpr bool staged_volume() {
  return std::is_same<Real, double>::value && N >= 6;
}

// Volume-term arithmetic of the FP32 path: CUDA cores (the combined form), or
// the derivative contractions on the tensor cores with split operands.
enum { kVolCuda = 0, kVolTcFp16 = 1, kVolTcBf16 = 2 };

// Tensor-core volume form (FP32 path).  Along direction i the conservative and
// non-conservative parts need the contractions D_i u and D_i F, F = A_+(Ja^i) u,
// of 18 fields.  Their lines of n values are laid out line-major in shared memory
// with a pitch of P >= n floats (a power of two; positions n..P-1 are zero), so
// that one 8-float row holds SEG = 8/P lines and 16 rows form the A operand of
// one mma.sync.m16n8k8 (FP32 accumulation) whose B operand is the block-diagonal
// matrix of SEG copies of D^T.  Each field occupies FS floats (whole 32-word
// blocks), and within a field a pair of positions (2t, 2t+1) is stored at pair
// slot t ^ h(block) of its row, which spreads the node-wise writes of the three
// directions over the banks while each half-warp still reads 32 distinct words.
template <int N>
struct TcShape {
  using S = Shape<N>;
  static constexpr int n = S::n;
  static constexpr int P = n <= 2 ? 2 : (n <= 4 ? 4 : 8);
  static constexpr int SEG = 8 / P;
  static constexpr int L = S::EPB * S::nf;                 // lines per field and direction
  static constexpr int FS = ((L * P + 31) / 32) * 32;      // floats per field
  static constexpr int FSB = FS / 32;                      // 32-word blocks per field
  static constexpr int TILES = (18 * FS + 127) / 128;      // 16 x 8 tiles per direction
  static constexpr int WORDS = TILES * 128;
  static constexpr bool ZERO = P > n || FS > L * P;        // padding to clear once per CTA
};

__device__ __forceinline__ int tc_swz(int block) { return ((block & 1) << 1) | ((block >> 1) & 1); }

// Preferred shared-memory carveout of a stage kernel, in percent of the
// largest (100: the most shared memory, the least L1).  The FP32 CUDA-core
// kernels read the neighbour traces and re-read the FP64 state in the epilogue
// through L1, and gain from a larger L1 even at a resident CTA fewer.  Measured
// on GB300, mixed stage in ms at 100 % / 72 % / 58 % (72 %: 164 KB of shared
// memory, 58 %: 132 KB): N = 1 3.92 / 4.33 / 6.90, N = 2 3.48 / 3.94 / 4.82,
// N = 3 3.14 / 3.10 / 3.54, N = 4 2.99 / 2.70 / 2.83, N = 5 2.85 / 2.73 / 2.73,
// N = 6 3.16 / 3.00 / 2.99, N = 7 3.36 / 3.31 / 4.10.  The tensor-core forms
// (BF16, 100 % / 86 % / 72 %): N = 4 4.83 / 4.82 / 4.76, N = 7 (48^3) 6.05 /
// 6.05 / 5.81 ms; other degrees not measured.  FP64 kernels (bound by their
// FP64 pipe) do not change and keep the largest shared memory.
template <int N, typename Real, int VOL>
__host__ __device__ constexpr int stage_carveout() {
  if constexpr (std::is_same<Real, float>::value && VOL == kVolCuda) {
    return N <= 2 ? 100 : ((N == 5 || N == 6) ? 58 : 72);
  } else if constexpr (std::is_same<Real, float>::value) {
    return (N == 4 || N == 7) ? 72 : 100;
  } else {
    return 100;
  }
}

// L1 prefetch of the RK register (read in the epilogue) and of the face items'
// neighbour traces (read in the face phase), issued with the tile load.  Measured
// on GB300, mixed stage, with the L2 bulk prefetch off at the same degrees (the
// two compete for L2: an L2 prefetch ahead evicts traces before their gather):
// N = 3 +1.5 %, 5 +1.7 %, 6 +0.9 %, 7 +6 % over the best L2 prefetch distance
// alone; N = 4 1 % slower.  Used for the FP32 CUDA-core kernel at N = 3, 5, 6, 7.
template <int N, typename Real, int VOL>
__host__ __device__ constexpr bool l1_prefetch() {
  return std::is_same<Real, float>::value && VOL == kVolCuda && (N == 3 || N >= 5);
}

template <int N, typename Real, int VOL = kVolCuda>
struct StageSmem {
  using S = Shape<N>;
  static constexpr int PK = Pack<Real>::PK;
  static constexpr size_t u_off = 0;                                    // Real [NTILE][PK] state
  // Real [9][NFACE_ITEMS] face fluxes; the staged volume form first keeps
  // A_+(Ja^i)u [NTILE][PK] of one direction in the same region, the tensor-core
  // form its line-major operands.
  static constexpr size_t f_off = u_off + sizeof(Real) * S::NTILE * PK;
  static constexpr size_t fwords0 = (staged_volume<N, Real>() && S::NTILE * PK > 9 * S::NFACE_ITEMS)
                                        ? S::NTILE * PK
                                        : 9 * S::NFACE_ITEMS;
  static constexpr size_t fwords = (VOL != kVolCuda && TcShape<N>::WORDS > fwords0) ? TcShape<N>::WORDS : fwords0;
  static constexpr size_t fbytes = sizeof(Real) * fwords;
  static constexpr size_t g_off = f_off + ((fbytes + 15) / 16) * 16;     // Real [NTILE][PK] Ja, 1/J
  static constexpr size_t d_off = g_off + sizeof(Real) * S::NTILE * PK;  // Real [n*n]
  static constexpr size_t e_off = ((d_off + sizeof(Real) * S::n * S::n + 15) / 16) * 16;  // double [NT/32] reduction
  static constexpr size_t bytes = e_off + sizeof(double) * (S::NT / 32);
};

// Slots of the metric terms in a node's geometry tile: Ja^dir_k and 1/J.  FP32
// keeps each direction in its own 16-byte group (one vector load), with 1/J in
// the first group's spare slot; FP64 packs them (10 of 10 slots).
template <typename Real>
__host__ __device__ constexpr int gslot(int dir, int k) {
  return std::is_same<Real, float>::value ? 4 * dir + k : 3 * dir + k;
}
template <typename Real>
__host__ __device__ constexpr int gslot_ij() {
  return std::is_same<Real, float>::value ? 3 : 9;
}

// ---- tensor-core volume form (FP32 path) -----------------------------------
// Split x into hi + lo in the 16-bit format: hi = round(x), lo = round(x - hi),
// two values packed per 32-bit register (the first in the low half).
template <int VOL>
__device__ __forceinline__ void tc_split(float x0, float x1, unsigned& hi, unsigned& lo) {
  if constexpr (VOL == kVolTcFp16) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(x0 - f.x, x1 - f.y);
    hi = *reinterpret_cast<const unsigned*>(&h);
    lo = *reinterpret_cast<const unsigned*>(&l);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const unsigned hb = *reinterpret_cast<const unsigned*>(&h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - __uint_as_float(hb << 16), x1 - __uint_as_float(hb & 0xffff0000u));
    hi = hb;
    lo = *reinterpret_cast<const unsigned*>(&l);
  }
}

// c += A B for one m16n8k8 tile: A 16 x 8 (a01: row g, a23: row g + 8), B 8 x 8.
template <int VOL>
__device__ __forceinline__ void tc_mma(float (&c)[4], unsigned a01, unsigned a23, unsigned b) {
  if constexpr (VOL == kVolTcFp16) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a01), "r"(a23), "r"(b));
  } else {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a01), "r"(a23), "r"(b));
  }
}

// This thread's B fragment (rows k = 2t, 2t+1 of column g) of the block-diagonal
// B with B[k][a] = D[a][k] inside each P x P block, split into hi and lo.  The
// entries of D are O(1) to O(N^2): no scaling is needed in either format.
template <int N, int VOL>
__device__ __forceinline__ void tc_b_fragment(const float* D_s, unsigned& bhi, unsigned& blo) {
  using T = TcShape<N>;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float v[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int k = 2 * t + j;
    const bool in = (k / T::P == g / T::P) && (k % T::P) < T::n && (g % T::P) < T::n;
    v[j] = in ? D_s[(g % T::P) * T::n + (k % T::P)] : 0.f;
  }
  tc_split<VOL>(v[0], v[1], bhi, blo);
}

// Field-local word of (line l, position b) of one direction's operands.
template <int N>
__device__ __forceinline__ int tc_word(int l, int b) {
  const int w = l * TcShape<N>::P + b;
  return w ^ (tc_swz(w >> 5) << 1);
}

// The contractions of one direction, in place: every warp takes 16 x 8 tiles
// of the operand region and replaces each row's lines x by D x.  FP16: each row
// is scaled by the power of two 2^s that brings its largest magnitude into
// [2^14, 2^15) (the exponent maximum over the four threads of the row's quad;
// s <= 126 so that 2^-s is a normal float, which leaves rows below 2^-112 one
// bit of headroom short); the products hi*hi + hi*lo + lo*hi are exact and
// summed in FP32, and the result is scaled back by 2^-s.  BF16 keeps the FP32
// exponent range and needs no scaling.
template <int N, int VOL>
__device__ __forceinline__ void tc_contract(float* X, unsigned bhi, unsigned blo) {
  using T = TcShape<N>;
  constexpr int NW = Shape<N>::NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int tile = warp; tile < T::TILES; tile += NW) {
    const int blk0 = 4 * tile + (g >> 2), blk1 = blk0 + 2;     // 32-word blocks of rows g and g + 8
    float* p0 = X + tile * 128 + g * 8 + 2 * (t ^ tc_swz(blk0 % T::FSB));
    float* p1 = X + tile * 128 + (g + 8) * 8 + 2 * (t ^ tc_swz(blk1 % T::FSB));
    float2 x0 = *reinterpret_cast<const float2*>(p0);
    float2 x1 = *reinterpret_cast<const float2*>(p1);
    float inv0 = 1.f, inv1 = 1.f;
    if constexpr (VOL == kVolTcFp16) {
      const unsigned m0 = max(__float_as_uint(fabsf(x0.x)), __float_as_uint(fabsf(x0.y)));
      const unsigned m1 = max(__float_as_uint(fabsf(x1.x)), __float_as_uint(fabsf(x1.y)));
      unsigned e = ((m0 >> 23) << 16) | (m1 >> 23);
      e = __vmaxu2(e, __shfl_xor_sync(0xffffffffu, e, 1));
      e = __vmaxu2(e, __shfl_xor_sync(0xffffffffu, e, 2));
      const int s0 = min(141 - static_cast<int>(e >> 16), 126);
      const int s1 = min(141 - static_cast<int>(e & 0xffffu), 126);
      const float sc0 = __int_as_float((127 + s0) << 23), sc1 = __int_as_float((127 + s1) << 23);
      inv0 = __int_as_float((127 - s0) << 23);
      inv1 = __int_as_float((127 - s1) << 23);
      x0.x *= sc0;
      x0.y *= sc0;
      x1.x *= sc1;
      x1.y *= sc1;
    }
    unsigned ah0, al0, ah1, al1;
    tc_split<VOL>(x0.x, x0.y, ah0, al0);
    tc_split<VOL>(x1.x, x1.y, ah1, al1);
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    tc_mma<VOL>(c, al0, al1, bhi);    // small terms first
    tc_mma<VOL>(c, ah0, ah1, blo);
    tc_mma<VOL>(c, ah0, ah1, bhi);
    *reinterpret_cast<float2*>(p0) = make_float2(c[0] * inv0, c[1] * inv0);
    *reinterpret_cast<float2*>(p1) = make_float2(c[2] * inv1, c[3] * inv1);
  }
}

// Kernel modes.  RHS: write L(u).  LSRK: fused 2N-storage stage update.
// ADJ: the reversed operator (A_k -> -A_k, same stabilisation) without Q^{-1}
//   on a prepared adjoint weight z = (M Q)^{-1} w, and lu <- lu + dt w J r,
//   which together apply dt L^T w (L^T = (M Q) L_rev (M Q)^{-1}).
// GRAD: the forward operator on a stage input u, accumulating the material
//   gradient terms dt w^T (dL/dm) u of the adjoint weight w.
// GRAD_FACE: GRAD with the operator output taken from p.rout (written by the
//   forward LSRK stage on the same input): only the face terms are computed.
enum { kModeRhs = 0, kModeLsrk = 1, kModeAdj = 2, kModeGrad = 3, kModeGradFace = 4 };

// One tile (EPB consecutive elements) of one solve.  The caller has filled the
// D tile of shared memory; p may live in parameter or shared memory.
template <int N, typename Real, int MODE, int VOL = kVolCuda>
__device__ __forceinline__ void stage_tile(const StageParams& p, long long tile, unsigned char* smem_raw) {
  constexpr bool LSRK = MODE == kModeLsrk;
  constexpr bool GRADM = MODE == kModeGrad || MODE == kModeGradFace;
  static_assert(VOL == kVolCuda || (std::is_same<Real, float>::value && (MODE == kModeRhs || MODE == kModeLsrk)),
                "the tensor-core volume form belongs to the FP32 forward path");
  const Real sgnA = MODE == kModeAdj ? Real(-1) : Real(1);
  using S = Shape<N>;
  using L = StageSmem<N, Real, VOL>;
  using V = Pack<Real>;
  constexpr int n = S::n, Np = S::Np, nf = S::nf, EPB = S::EPB, NT = S::NT;
  constexpr int NTILE = S::NTILE, NFI = S::NFACE_ITEMS, PK = L::PK;

  Real* u_s = reinterpret_cast<Real*>(smem_raw + L::u_off);
  Real* f_s = reinterpret_cast<Real*>(smem_raw + L::f_off);   // staged A_+(Ja^i)u (staged form)
  Real* x_s = f_s;                                             // then the face fluxes [9][NFI]
  Real* g_s = reinterpret_cast<Real*>(smem_raw + L::g_off);
  Real* D_s = reinterpret_cast<Real*>(smem_raw + L::d_off);
  double* red_s = reinterpret_cast<double*>(smem_raw + L::e_off);

  const int t = threadIdx.x;
  const long long e0 = tile * EPB;
  const int el = t / Np;
  const int node = t - el * Np;
  const long long e = e0 + el;
  const bool in_tile = t < NTILE;
  const bool active = in_tile && (e < p.nel);
  const size_t fstride = static_cast<size_t>(p.nel) * Np;
  const size_t gidx = active ? static_cast<size_t>(e) * Np + node : 0;
  const Real* geo = static_cast<const Real*>(p.geo);
  const bool first = p.first != 0;

  if (p.pf_elems > 0) {
    // L2 prefetch of the tile that starts p.pf_elems elements later, so that its
    // loads hit L2: the state, metric terms and register, and the small per-element
    // arrays read behind them (neighbour map, face impedances, medium).  The tile
    // must end before the last element: the 16-byte rounding of each range then
    // stays inside every field of the buffers.
    const long long ep = e0 + p.pf_elems;
    if (t < 36 && ep + EPB < p.nel) {
      const size_t off = static_cast<size_t>(ep) * Np;
      const size_t len = static_cast<size_t>(EPB) * Np;
      if (t < 9) {
        const double* a = p.u_in + t * fstride + off;
        prefetch_l2(a, a + len);
      } else if (t < 19) {
        const Real* a = geo + (t - 9) * fstride + off;
        prefetch_l2(a, a + len);
      } else if (t < 28) {
        if (LSRK && !first) {
          const double* a = p.res + (t - 19) * fstride + off;
          prefetch_l2(a, a + len);
        }
      } else if (t == 28) {
        const int* a = p.vmapP + static_cast<size_t>(ep) * 6 * nf;
        prefetch_l2(a, a + static_cast<size_t>(EPB) * 6 * nf);
      } else if (t < 33) {
        if (p.fz != nullptr) {
          const Real* a = static_cast<const Real*>(p.fz) + static_cast<size_t>(t - 29) * p.nel * 6 + ep * 6;
          prefetch_l2(a, a + EPB * 6);
        }
      } else if (p.mat != nullptr && ep + EPB + 16 / static_cast<long long>(sizeof(Real)) <= p.nel) {
        // one Real per element: keep 16 bytes of elements after the range
        const Real* a = static_cast<const Real*>(p.mat) + static_cast<size_t>(t - 33) * p.nel + ep;
        prefetch_l2(a, a + EPB);
      }
    }
  }

  if constexpr (l1_prefetch<N, Real, VOL>()) {
    // neighbour traces of this thread's face items into L1
    for (int it = t; it < NFI; it += NT) {
      const int eli = it / (6 * nf);
      if (e0 + eli >= p.nel) break;
      const int g = p.vmapP[static_cast<size_t>(e0 + eli) * 6 * nf + (it - eli * 6 * nf)];
      if (g >= 0 && static_cast<long long>(g) < p.nel * Np) {
#pragma unroll
        for (int q = 0; q < 9; ++q) prefetch_l1(p.u_in + q * fstride + g);
      }
    }
  }
  Real uw[9];      // this node's state (kept for the tensor-core volume form)
  if (in_tile) {
    Real w[10], gj[10];
    if (active) {
#pragma unroll
      for (int q = 0; q < 9; ++q) w[q] = to_real<Real>(p.u_in[q * fstride + gidx]);
#pragma unroll
      for (int c = 0; c < 10; ++c) gj[c] = geo[c * fstride + gidx];
      if constexpr (LSRK && l1_prefetch<N, Real, VOL>()) {
        if (!first) {
#pragma unroll
          for (int q = 0; q < 9; ++q) prefetch_l1(p.res + q * fstride + gidx);
        }
      }
      if constexpr (kDebugChecks) {
        bool finite = true;
#pragma unroll
        for (int q = 0; q < 9; ++q) finite = finite && isfinite(w[q]);
        if (!finite) debug_record(p.fault, kFaultNonFiniteState, e);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 10; ++c) w[c] = gj[c] = 0;
    }
    w[9] = 0;
#pragma unroll
    for (int q = 0; q < 9; ++q) uw[q] = w[q];
    V::store10(u_s + t * PK, w);
    if constexpr (std::is_same<Real, float>::value) {
      float4* gp = reinterpret_cast<float4*>(g_s + t * PK);
      gp[0] = make_float4(gj[0], gj[1], gj[2], gj[9]);
      gp[1] = make_float4(gj[3], gj[4], gj[5], 0.f);
      gp[2] = make_float4(gj[6], gj[7], gj[8], 0.f);
    } else {
      V::store10(g_s + t * PK, gj);
    }
  }
  if constexpr (VOL != kVolCuda) {
    if constexpr (TcShape<N>::ZERO) {
      // zero the padding positions and lines of the operand region once
      float4* z = reinterpret_cast<float4*>(f_s);
      for (int i = t; i < TcShape<N>::WORDS / 4; i += NT) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  __syncthreads();

  const int ix = node % n;
  const int iy = (node / n) % n;
  const int iz = node / nf;

  Real acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0;

  // Volume term, direction by direction along the line of n nodes through this
  // one (a its index on the line): the conservative part D_i(A_+(Ja^i) u) and
  // the non-conservative part A_+(Ja^i)(D_i u) together are
  //   sum_b D_ab A_+(m_b) u_b + A_+(m_a) sum_b D_ab u_b = sum_b A_+(D_ab (m_a + m_b)) u_b,
  // m = Ja^i (A_+ is linear in m).  Combined form: the right-hand side,
  // accumulated term by term from the state and metric tiles (no staging, no
  // barrier between directions).  Staged form: the left-hand side, with
  // A_+(m_b) u_b staged per direction.
  if constexpr (MODE == kModeGradFace) {
    // no volume term: the operator output comes from the forward stage
  } else if constexpr (VOL != kVolCuda) {
    // Tensor-core form: per direction, write u and F = A_+(Ja^i) u line-major,
    // contract all lines by D on the tensor cores, then acc += D F + A_+(Ja^i_a) D u.
    using T = TcShape<N>;
    float* X = reinterpret_cast<float*>(f_s);
    unsigned bhi, blo;
    tc_b_fragment<N, VOL>(reinterpret_cast<const float*>(D_s), bhi, blo);
#pragma unroll 1
    for (int dir = 0; dir < 3; ++dir) {
      int lw = 0;
      float4 mt = make_float4(0.f, 0.f, 0.f, 0.f);
      if (in_tile) {
        const int l = el * nf + (dir == 0 ? iy + n * iz : (dir == 1 ? ix + n * iz : ix + n * iy));
        const int b = dir == 0 ? ix : (dir == 1 ? iy : iz);
        lw = tc_word<N>(l, b);
        mt = reinterpret_cast<const float4*>(g_s + t * PK)[dir];
        float F[9];
        apply_Apos(mt.x, mt.y, mt.z, uw, F);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          X[q * T::FS + lw] = uw[q];
          X[(9 + q) * T::FS + lw] = F[q];
        }
      }
      __syncthreads();
      tc_contract<N, VOL>(X, bhi, blo);
      __syncthreads();
      if (in_tile) {
        float du[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          du[q] = X[q * T::FS + lw];
          acc[q] += X[(9 + q) * T::FS + lw];
        }
        acc_Apos(mt.x, mt.y, mt.z, du, acc);
      }
      __syncthreads();    // the region is overwritten next (next direction, or the face fluxes)
    }
  } else if constexpr (staged_volume<N, Real>()) {
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
      Real m1 = 0, m2 = 0, m3 = 0;
      if (in_tile) {
        m1 = g_s[t * PK + gslot<Real>(dir, 0)];
        m2 = g_s[t * PK + gslot<Real>(dir, 1)];
        m3 = g_s[t * PK + gslot<Real>(dir, 2)];
        Real w[10], F[10];
        V::load9(u_s + t * PK, w);
        apply_Apos(m1, m2, m3, w, F);
        F[9] = 0;
        V::store10(f_s + t * PK, F);
      }
      __syncthreads();
      if (in_tile) {
        const int stride = dir == 0 ? 1 : (dir == 1 ? n : nf);
        const int a = dir == 0 ? ix : (dir == 1 ? iy : iz);
        const int base = t - a * stride;
        Real ds[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) ds[q] = 0;
#pragma unroll
        for (int b = 0; b < n; ++b) {
          const Real Dab = D_s[a * n + b];
          Real F[10], w[10];
          V::load9(f_s + (base + b * stride) * PK, F);
          V::load9(u_s + (base + b * stride) * PK, w);
#pragma unroll
          for (int q = 0; q < 9; ++q) {
            acc[q] += Dab * F[q];
            ds[q] += Dab * w[q];
          }
        }
        acc_Apos(m1, m2, m3, ds, acc);
      }
      __syncthreads();
    }
  } else if (in_tile) {
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
      const int stride = dir == 0 ? 1 : (dir == 1 ? n : nf);
      const int a = dir == 0 ? ix : (dir == 1 ? iy : iz);
      const int base = t - a * stride;
      Real ma0, ma1, ma2;
      if constexpr (std::is_same<Real, float>::value) {
        const float4 mt = reinterpret_cast<const float4*>(g_s + t * PK)[dir];
        ma0 = mt.x;
        ma1 = mt.y;
        ma2 = mt.z;
      } else {
        ma0 = g_s[t * PK + gslot<Real>(dir, 0)];
        ma1 = g_s[t * PK + gslot<Real>(dir, 1)];
        ma2 = g_s[t * PK + gslot<Real>(dir, 2)];
      }
#pragma unroll
      for (int b = 0; b < n; ++b) {
        const Real Dab = D_s[a * n + b];
        const int nb = base + b * stride;
        Real w[10];
        V::load9(u_s + nb * PK, w);
        Real mb0, mb1, mb2;
        if constexpr (std::is_same<Real, float>::value) {
          const float4 mb = reinterpret_cast<const float4*>(g_s + nb * PK)[dir];
          mb0 = mb.x;
          mb1 = mb.y;
          mb2 = mb.z;
        } else {
          mb0 = g_s[nb * PK + gslot<Real>(dir, 0)];
          mb1 = g_s[nb * PK + gslot<Real>(dir, 1)];
          mb2 = g_s[nb * PK + gslot<Real>(dir, 2)];
        }
        acc_Apos(Dab * (ma0 + mb0), Dab * (ma1 + mb1), Dab * (ma2 + mb2), w, acc);
      }
    }
  }

  // Face items: lifted flux differences.
  {
    const Real* fz = static_cast<const Real*>(p.fz);
    const Real tau = pick<Real>(p.tau, p.tau_f);
    // LSRK: the right-hand side is produced already multiplied by dt (Q^{-1} is linear)
    const Real half_lift = pick<Real>(0.5 * p.w_end_inv, p.hlift_f) * (LSRK ? pick<Real>(p.dt, p.dt_f) : Real(1));
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
      const int vn = c0 + n * (c1 + n * c2);
      const int sidx = eli * Np + vn;

      Real um[10], du[9];
      V::load9(u_s + sidx * PK, um);
      int g = p.vmapP[static_cast<size_t>(ei) * 6 * nf + r];
      if constexpr (kDebugChecks) {
        if (g >= 0 && static_cast<long long>(g) >= p.nel * Np) {
          debug_record(p.fault, kFaultNeighbourIndex, ei);
          g = kGhostAbsorbing;            // skip the out-of-range read
        }
      }
      // FP32 tiles of several elements (N <= 3): a neighbour node inside this
      // tile is read from the shared state tile (the same narrowed values) instead
      // of L2 (mixed N = 2: +5 %; the FP64 path, bound by its FP64 pipe, lost 2-3 %
      // to the extra branch and keeps the L2 read).
      long long gl = -1;
      if constexpr (EPB > 1 && std::is_same<Real, float>::value) {
        gl = static_cast<long long>(g) - e0 * Np;
        if (g < 0 || gl >= NTILE) gl = -1;
      }
      if (gl >= 0) {
        Real up[10];
        V::load9(u_s + gl * PK, up);
#pragma unroll
        for (int q = 0; q < 9; ++q) du[q] = um[q] - up[q];
      } else if (g >= 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) du[q] = um[q] - to_real<Real>(p.u_in[q * fstride + g]);
      } else if (g == kGhostFreeSurface) {
        // exterior (v, -sigma): jump (0, 2 sigma)
#pragma unroll
        for (int q = 0; q < 3; ++q) du[q] = 0;
#pragma unroll
        for (int q = 3; q < 9; ++q) du[q] = 2 * um[q];
      } else {
#pragma unroll
        for (int q = 0; q < 9; ++q) du[q] = um[q];
      }
      const Real sgn = hi ? Real(1) : Real(-1);
      const Real m1 = sgn * g_s[sidx * PK + gslot<Real>(d, 0)];
      const Real m2 = sgn * g_s[sidx * PK + gslot<Real>(d, 1)];
      const Real m3 = sgn * g_s[sidx * PK + gslot<Real>(d, 2)];
      const Real jv = g_s[sidx * PK + gslot_ij<Real>()];

      Real Ad[9];
      apply_Apos(m1, m2, m3, du, Ad);      // A_+(m) du = -A(m) du
      Real flux[9];
      const Real s = -half_lift * jv;
      if (tau != Real(0)) {
        // Impedance-weighted upwind stabilisation S(m) = sJ Q|Q^{-1}A(n)| of the
        // face medium (Zp = rho cp, Zs = rho cs):
        //   velocity rows  sJ [Zs dv + (Zp - Zs)(n.dv) n]
        //   stress rows    sJ B(n) [y/Zs + (1/Zp - 1/Zs)(n.y) n],  y = B(n)^T dsigma.
        const size_t fzi = static_cast<size_t>(ei) * 6 + f;
        const size_t fzs = static_cast<size_t>(p.nel) * 6;
        const Real zs = fz[fzi], dz = fz[fzs + fzi], izs = fz[2 * fzs + fzi], diz = fz[3 * fzs + fzi];
        const Real mm = m1 * m1 + m2 * m2 + m3 * m3;
        Real isJ;
        if constexpr (std::is_same<Real, double>::value) {
          isJ = rsqrt(mm);                   // one refinement sequence instead of sqrt and a division
        } else {
          isJ = Real(1) / sqrt(mm);
        }
        const Real sJ = mm * isJ;
        const Real av = dz * (m1 * du[0] + m2 * du[1] + m3 * du[2]) * isJ;
        const Real zsJ = zs * sJ;
        // y = dsigma m = Ad[0..2] (scaled by sJ); z = isJ (y/Zs + (1/Zp-1/Zs)(m.y) m / sJ^2)
        const Real by = diz * (m1 * Ad[0] + m2 * Ad[1] + m3 * Ad[2]) * isJ * isJ;
        const Real z0 = isJ * (izs * Ad[0] + by * m1);
        const Real z1 = isJ * (izs * Ad[1] + by * m2);
        const Real z2 = isJ * (izs * Ad[2] + by * m3);
        const Real Sd[9] = {zsJ * du[0] + av * m1, zsJ * du[1] + av * m2, zsJ * du[2] + av * m3,
                            m1 * z0, m2 * z1, m3 * z2,
                            m2 * z2 + m3 * z1, m1 * z2 + m3 * z0, m1 * z1 + m2 * z0};
        // 1/2 (A(m) - tau S(m)) du (1/J)/w_0 = -1/2 (A_+ du + tau S du) (1/J)/w_0
#pragma unroll
        for (int q = 0; q < 9; ++q) flux[q] = s * (sgnA * Ad[q] + tau * Sd[q]);
        if constexpr (GRADM) {
          // d(flux)/dZs and d(flux)/dZp against Q_e^{-1} w at this node.
          const size_t gi = static_cast<size_t>(ei) * Np + vn;
          const Real* matg = static_cast<const Real*>(p.mat);
          const Real irho = matg[ei], lamg = matg[p.nel + ei], mug = matg[2 * p.nel + ei];
          Real w[9], qh[9];
#pragma unroll
          for (int q = 0; q < 9; ++q) w[q] = p.res[q * fstride + gi];
          qh[0] = irho * w[0];
          qh[1] = irho * w[1];
          qh[2] = irho * w[2];
          const Real trw = w[3] + w[4] + w[5];
          qh[3] = lamg * trw + 2 * mug * w[3];
          qh[4] = lamg * trw + 2 * mug * w[4];
          qh[5] = lamg * trw + 2 * mug * w[5];
          qh[6] = mug * w[6];
          qh[7] = mug * w[7];
          qh[8] = mug * w[8];
          Real zq[9], Bq[9];
#pragma unroll
          for (int q = 0; q < 3; ++q) zq[q] = 0;
#pragma unroll
          for (int q = 3; q < 9; ++q) zq[q] = qh[q];
          apply_Apos(m1, m2, m3, zq, Bq);                 // Bq[0..2] = B(m)^T qh_sigma
          const Real mdv = (m1 * du[0] + m2 * du[1] + m3 * du[2]) * isJ;
          const Real mqv = (m1 * qh[0] + m2 * qh[1] + m3 * qh[2]) * isJ;
          const Real my = (m1 * Ad[0] + m2 * Ad[1] + m3 * Ad[2]) * isJ;    // (n.y) sJ
          const Real mbq = (m1 * Bq[0] + m2 * Bq[1] + m3 * Bq[2]) * isJ;
          const Real yb = Ad[0] * Bq[0] + Ad[1] * Bq[1] + Ad[2] * Bq[2];
          const Real qdv = qh[0] * du[0] + qh[1] * du[1] + qh[2] * du[2];
          // velocity rows: dS/dZs = sJ (I - n n^T), dS/dZp = sJ n n^T
          // stress rows:   dS/dZs = -(1/Zs^2) (1/sJ) B_m (I - n n^T) B_m^T, dS/dZp = -(1/Zp^2) (1/sJ) B_m n n^T B_m^T
          const Real izp = izs + diz;
          const Real gzs = sJ * (qdv - mdv * mqv) - izs * izs * isJ * (yb - my * mbq);
          const Real gzp = sJ * mdv * mqv - izp * izp * isJ * my * mbq;
          const size_t ii = static_cast<size_t>(ei) * 6 * nf + r;
          const Real sc = static_cast<Real>(p.dt) * s * tau;
          p.grad_face[ii] += sc * gzs;
          p.grad_face[static_cast<size_t>(p.nel) * 6 * nf + ii] += sc * gzp;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 9; ++q) flux[q] = s * sgnA * Ad[q];
      }
      if constexpr (MODE != kModeGradFace) {
#pragma unroll
        for (int q = 0; q < 9; ++q) x_s[q * NFI + it] = flux[q];
      }
    }
  }
  __syncthreads();

  double e_node = 0.0;     // w J u_out^T Q u_out of this node (fused energy)
  Real gnode[3] = {0, 0, 0};   // GRAD mode: this node's material gradient terms
  if (active) {
    // vol = -1/2 (1/J) (-acc_+) = +1/2 (1/J) acc_+  (acc holds A_+ terms)
    Real r[9];
    const Real hv = static_cast<Real>(0.5) * g_s[t * PK + gslot_ij<Real>()] *
                    (LSRK ? pick<Real>(p.dt, p.dt_f) : Real(1));
#pragma unroll
    for (int q = 0; q < 9; ++q) r[q] = hv * sgnA * acc[q];
    const int fb0 = el * 6 * nf;
    auto add_face = [&](int f, int pidx) {
#pragma unroll
      for (int q = 0; q < 9; ++q) r[q] += x_s[q * NFI + fb0 + f * nf + pidx];
    };
    if constexpr (MODE == kModeGradFace) {
      // dt (K u + f) of this node from the forward stage (below)
#pragma unroll
      for (int q = 0; q < 9; ++q) r[q] = p.rout[q * fstride + gidx];
    } else {
      if (ix == 0) add_face(0, iy + n * iz);
      if (ix == N) add_face(1, iy + n * iz);
      if (iy == 0) add_face(2, ix + n * iz);
      if (iy == N) add_face(3, ix + n * iz);
      if (iz == 0) add_face(4, ix + n * iy);
      if (iz == N) add_face(5, ix + n * iy);
    }

    if constexpr (MODE == kModeAdj) {
      // lu <- lu + dt (w J) r : M Q L_rev z without Q^{-1} (Q^{-1} and Q cancel)
      const double wj = p.wJ[gidx];
#pragma unroll
      for (int q = 0; q < 9; ++q) p.out[q * fstride + gidx] = p.res[q * fstride + gidx] + p.dt * wj * r[q];
    }
    if constexpr (GRADM) {
      // dt w^T (d Q^{-1}/dm) (K u + f) at this node, f the point force (before Q^{-1});
      // GRAD_FACE reads dt (K u + f) as the forward stage produced it
      const Real* matg = static_cast<const Real*>(p.mat);
      const Real irho = matg[e];
      if (MODE == kModeGrad && e == p.src_elem) {
#pragma unroll
        for (int q = 0; q < 3; ++q) r[q] += static_cast<Real>(p.src_amp * p.src_w[q * Np + node]) / irho;
      }
      Real w[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) w[q] = p.res[q * fstride + gidx];
      const Real dtg = MODE == kModeGrad ? static_cast<Real>(p.dt) : Real(1);
      gnode[0] = -dtg * irho * irho * (w[0] * r[0] + w[1] * r[1] + w[2] * r[2]);
      gnode[1] = dtg * (w[3] + w[4] + w[5]) * (r[3] + r[4] + r[5]);
      gnode[2] = dtg * (2 * (w[3] * r[3] + w[4] * r[4] + w[5] * r[5]) + w[6] * r[6] + w[7] * r[7] + w[8] * r[8]);
    }

    if constexpr (MODE == kModeRhs || MODE == kModeLsrk) {
    // Q^{-1}: velocity rows / rho, stress rows by the isotropic stiffness C_V.
    const Real* mat = static_cast<const Real*>(p.mat);
    const Real irho = mat[e];
    const Real lam = mat[p.nel + e];
    const Real mu = mat[2 * p.nel + e];
    if constexpr (LSRK && std::is_same<Real, double>::value) {
      if (p.rout != nullptr) {
        // dt (K u + f) before Q^{-1}, kept for the adjoint's gradient terms
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          double v = r[q];
          if (q < 3 && e == p.src_elem) v += p.dt * p.src_amp * p.src_w[q * Np + node] / irho;
          p.rout[q * fstride + gidx] = v;
        }
      }
    }
    Real rr[9];
    rr[0] = irho * r[0];
    rr[1] = irho * r[1];
    rr[2] = irho * r[2];
    const Real tr = r[3] + r[4] + r[5];
    const Real two_mu = mu + mu;
    rr[3] = lam * tr + two_mu * r[3];
    rr[4] = lam * tr + two_mu * r[4];
    rr[5] = lam * tr + two_mu * r[5];
    rr[6] = mu * r[6];
    rr[7] = mu * r[7];
    rr[8] = mu * r[8];
    if (e == p.src_elem) {
      // point force (already divided by rho and the mass weight at set-up)
#pragma unroll
      for (int q = 0; q < 3; ++q) rr[q] += static_cast<Real>((LSRK ? p.dt : 1.0) * p.src_amp * p.src_w[q * Np + node]);
    }

    if constexpr (!LSRK) {
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        if constexpr (std::is_same<Real, double>::value) {
          p.out[q * fstride + gidx] = rr[q];
        } else {
          p.out[q * fstride + gidx] = widen_int(rr[q]);
        }
      }
    } else {
      // res <- a res + dt rhs; u_out <- u_in + b res, both FP64.  a_0 = 0: the
      // incoming register is not read in the first stage.
      double uout[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const double uq = p.u_in[q * fstride + gidx];     // FP64 state (L2-resident re-read)
        double dtr;
        if constexpr (std::is_same<Real, double>::value) {
          dtr = rr[q];                                // dt already applied
        } else {
          dtr = widen_int(rr[q]);
        }
        const double rin = first ? 0.0 : p.res[q * fstride + gidx];
        const double rn = first ? dtr : fma(p.a, rin, dtr);
        p.res[q * fstride + gidx] = rn;
        const double uo = fma(p.b, rn, uq);
        p.out[q * fstride + gidx] = uo;
        uout[q] = uo;
      }
      if (p.energy_partials != nullptr) {
        const double rho = p.ec[e], i2mu = p.ec[p.nel + e], lfac = p.ec[2 * p.nel + e], imu = p.ec[3 * p.nel + e];
        const double tr2 = uout[3] + uout[4] + uout[5];
        const double kin = rho * (uout[0] * uout[0] + uout[1] * uout[1] + uout[2] * uout[2]);
        const double pot = i2mu * (uout[3] * uout[3] + uout[4] * uout[4] + uout[5] * uout[5] - lfac * tr2 * tr2) +
                           imu * (uout[6] * uout[6] + uout[7] * uout[7] + uout[8] * uout[8]);
        e_node = p.wJ[gidx] * (kin + pot);
      }
    }
    }
  }
  if constexpr (GRADM) {
    // Sum the node terms of each element in a fixed order (the state tile is free now).
    __syncthreads();
    if (in_tile) {
#pragma unroll
      for (int c = 0; c < 3; ++c) u_s[t * PK + c] = gnode[c];
    }
    __syncthreads();
    if (t < 3 * EPB) {
      const int ee = t / 3, c = t - 3 * (t / 3);
      const long long eg = e0 + ee;
      if (eg < p.nel) {
        Real sum = 0;
        for (int k = 0; k < Np; ++k) sum += u_s[(ee * Np + k) * PK + c];
        p.grad_el[c * p.nel + eg] += sum;
      }
    }
  }
  if constexpr (LSRK) {
    if (p.energy_partials != nullptr) {
      // Block sum of the node energies in a fixed order (bit-reproducible).
      double v = e_node;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if ((t & 31) == 0) red_s[t >> 5] = v;
      __syncthreads();
      if (t < 32) {
        double w2 = t < NT / 32 ? red_s[t] : 0.0;
        for (int off = 16; off > 0; off >>= 1) w2 += __shfl_down_sync(0xffffffffu, w2, off);
        if (t == 0) p.energy_partials[tile] = w2;
      }
    }
  }
}

template <int N, typename Real, int MODE, int VOL = kVolCuda>
__device__ __forceinline__ void stage_kernel_body(const StageParams& p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* D_s = reinterpret_cast<Real*>(smem_raw + StageSmem<N, Real, VOL>::d_off);
  for (int i = threadIdx.x; i < Shape<N>::n * Shape<N>::n; i += Shape<N>::NT) D_s[i] = to_real<Real>(p.D[i]);
  stage_tile<N, Real, MODE, VOL>(p, blockIdx.x, smem_raw);
}

template <int N, typename Real, int MODE, int VOL = kVolCuda>
__global__ void __launch_bounds__(Shape<N>::NT) stage_kernel(const StageParams p) {
  stage_kernel_body<N, Real, MODE, VOL>(p);
}

// FP32 at N = 7 (512 threads): three CTAs per SM fit in shared memory but only
// two at the 56 registers a thread the default allocation takes; asking for
// three (40 registers, a few spilled words) is 5 % faster on 48^3.  The other
// kernels keep the default allocation (a minimum-CTA bound changes it at every
// degree; N = 4 measured: 10 CTAs at 48 registers +0.3 %, 12 at 40 spilled and
// lost 9 %).
template <int MODE>
__global__ void __launch_bounds__(Shape<7>::NT, 3) stage_kernel_f32_n7(const StageParams p) {
  stage_kernel_body<7, float, MODE>(p);
}

// The tensor-core form at N = 7 holds 86 KB of shared memory: two CTAs per SM,
// which the default register allocation already allows; the bound keeps it so.
template <int MODE, int VOL>
__global__ void __launch_bounds__(Shape<7>::NT, 2) stage_kernel_tc_n7(const StageParams p) {
  stage_kernel_body<7, float, MODE, VOL>(p);
}

template <int N, typename Real, int MODE, int VOL = kVolCuda>
constexpr void (*stage_kernel_ptr())(const StageParams) {
  if constexpr (N == 7 && std::is_same<Real, float>::value && VOL == kVolCuda) {
    return &stage_kernel_f32_n7<MODE>;
  } else if constexpr (N == 7 && VOL != kVolCuda) {
    return &stage_kernel_tc_n7<MODE, VOL>;
  } else {
    return &stage_kernel<N, Real, MODE, VOL>;
  }
}

__device__ __forceinline__ double ricker_dev(double t, double f0, double t0) {
  const double a = 3.14159265358979323846 * f0 * (t - t0);
  return (1.0 - 2.0 * a * a) * exp(-a * a);
}

// Batched stage: one CTA per tile of the concatenated tile ranges of every
// solve of the batch (solves of one degree and precision, each with its own
// mesh, medium, state and source).  The descriptors are kernel parameters:
// each thread finds its tile's solve by a binary search over their first
// tiles and reads the solve's parameters from the constant bank, as the
// single-solve kernel does.  The stage time of the source is
// t + (step + c_s) dt with t read from device memory, so the launches can be
// replayed from a CUDA graph; CTAs past the tile total exit.
template <int N, typename Real>
__device__ __forceinline__ void stage_batch_body(const BatchLaunch& L, const BatchSet& S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long tile = blockIdx.x;
  if (tile >= S.total_tiles) return;
  Real* D_s = reinterpret_cast<Real*>(smem_raw + StageSmem<N, Real>::d_off);
  for (int i = threadIdx.x; i < Shape<N>::n * Shape<N>::n; i += Shape<N>::NT) D_s[i] = to_real<Real>(L.D[i]);
  int lo = 0, hi = S.nsolves - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (S.s[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  const BatchSolve& b = S.s[lo];
  StageParams ps;
  ps.u_in = b.u[L.parity];
  ps.out = b.u[L.parity ^ 1];
  ps.res = b.res;
  ps.geo = b.geo;
  ps.fz = b.fz;
  ps.vmapP = b.vmapP;
  ps.mat = b.mat;
  ps.nel = b.nel;
  ps.a = L.a;
  ps.b = L.b;
  ps.dt = b.dt;
  ps.tau = L.tau;
  ps.w_end_inv = L.w_end_inv;
  ps.energy_partials = nullptr;
  ps.wJ = nullptr;
  ps.ec = nullptr;
  ps.pf_elems = L.pf_elems;
  ps.grad_el = nullptr;
  ps.grad_face = nullptr;
  ps.rout = nullptr;        // no adjoint output in batches
  ps.fault = nullptr;       // batches record no debug faults
  ps.src_elem = b.src_elem;
  ps.src_w = b.src_w;
  ps.dt_f = b.dt_f;
  ps.tau_f = L.tau_f;
  ps.hlift_f = L.hlift_f;
  ps.first = L.first;
  ps.src_amp = 0.0;
  if (b.src_elem >= 0 && b.src_elem / Shape<N>::EPB == tile - b.tile0)
    ps.src_amp = ricker_dev(L.times[lo] + (L.step + L.c) * b.dt, b.src_f0, b.src_t0);
  stage_tile<N, Real, kModeLsrk>(ps, tile - b.tile0, smem_raw);
}

template <int N, typename Real>
__global__ void __launch_bounds__(Shape<N>::NT) stage_batch_kernel(const BatchLaunch L, const BatchSet S) {
  stage_batch_body<N, Real>(L, S);
}

// FP32 batched kernels with a resident-CTA bound where the default allocation
// costs a CTA per SM against the single-solve kernel: N = 3 (256 threads) took
// 62 registers (four CTAs) against 48 (five), N = 5 (224 threads) 64 (four)
// against 56 (five).  Asking for five CTAs gives 48 and 56 registers without
// spills.  Other degrees keep the default allocation.
template <int N, typename Real, int MIN_CTAS>
__global__ void __launch_bounds__(Shape<N>::NT, MIN_CTAS)
    stage_batch_kernel_bounded(const BatchLaunch L, const BatchSet S) {
  stage_batch_body<N, Real>(L, S);
}

template <int N, typename Real>
constexpr void (*stage_batch_kernel_ptr())(const BatchLaunch, const BatchSet) {
  if constexpr ((N == 3 || N == 5) && std::is_same<Real, float>::value) {
    return &stage_batch_kernel_bounded<N, Real, 5>;
  } else {
    return &stage_batch_kernel<N, Real>;
  }
}

template <int N, typename Real>
cudaError_t launch_stage_batch_t(const BatchLaunch& L, const BatchSet& S, int grid, cudaStream_t s) {
  const size_t smem = StageSmem<N, Real>::bytes;
  constexpr auto kernel = stage_batch_kernel_ptr<N, Real>();
  kernel<<<grid, Shape<N>::NT, smem, s>>>(L, S);
  return cudaGetLastError();
}

// Set the kernel attributes of the batched stage kernel.
template <int N, typename Real>
cudaError_t prepare_stage_batch_t() {
  const size_t smem = StageSmem<N, Real>::bytes;
  constexpr auto kernel = stage_batch_kernel_ptr<N, Real>();
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              stage_carveout<N, Real, kVolCuda>());
}

template <typename Real>
cudaError_t launch_stage_batch_any(int N, const BatchLaunch& L, const BatchSet& S, int grid, cudaStream_t s) {
  switch (N) {
#define DGW_BCASE(NN) \
  case NN:            \
    return launch_stage_batch_t<NN, Real>(L, S, grid, s);
    DGW_BCASE(1) DGW_BCASE(2) DGW_BCASE(3) DGW_BCASE(4) DGW_BCASE(5) DGW_BCASE(6) DGW_BCASE(7)
#undef DGW_BCASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename Real>
cudaError_t prepare_stage_batch_any(int N) {
  switch (N) {
#define DGW_PCASE(NN) \
  case NN:            \
    return prepare_stage_batch_t<NN, Real>();
    DGW_PCASE(1) DGW_PCASE(2) DGW_PCASE(3) DGW_PCASE(4) DGW_PCASE(5) DGW_PCASE(6) DGW_PCASE(7)
#undef DGW_PCASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int N, typename Real, int MODE, int VOL = kVolCuda>
cudaError_t launch_stage_t(const StageParams& p, cudaStream_t s) {
  using S = Shape<N>;
  const size_t smem = StageSmem<N, Real, VOL>::bytes;
  // Kernel attributes, set once per device (bit d of `ready`; devices 0..63).
  static std::atomic<unsigned long long> ready{0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  constexpr auto kernel = stage_kernel_ptr<N, Real, MODE, VOL>();
  if (!(ready.load(std::memory_order_relaxed) & bit)) {
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               stage_carveout<N, Real, VOL>());
    if (err != cudaSuccess) return err;
    ready.fetch_or(bit, std::memory_order_relaxed);
  }
  const long long blocks = (p.nel + S::EPB - 1) / S::EPB;
  if (blocks <= 0) return cudaSuccess;
  StageParams q = p;
  finish_stage_params(q);
  kernel<<<(unsigned)blocks, S::NT, smem, s>>>(q);
  return cudaGetLastError();
}

template <typename Real, int VOL = kVolCuda>
cudaError_t launch_stage_any(int N, bool lsrk, const StageParams& p, cudaStream_t s) {
#define DGW_CASE(NN)                                                                   \
  case NN:                                                                             \
    return lsrk ? launch_stage_t<NN, Real, kModeLsrk, VOL>(p, s) : launch_stage_t<NN, Real, kModeRhs, VOL>(p, s);
  switch (N) {
    DGW_CASE(1)
    DGW_CASE(2)
    DGW_CASE(3)
    DGW_CASE(4)
    DGW_CASE(5)
    DGW_CASE(6)
    DGW_CASE(7)
    default:
      return cudaErrorInvalidValue;
  }
#undef DGW_CASE
}

// One adjoint stage in one launch: every CTA takes its tile in GRAD (or
// GRAD_FACE) mode (the gradient terms of the stage input against the weight w),
// then in ADJ mode (the reversed operator on z, added to lu).  The two modes
// read the same metric terms, neighbour map, face impedances and medium of the
// tile, which the second pass finds in cache; they write disjoint outputs.
template <int N, int GMODE>
__global__ void __launch_bounds__(Shape<N>::NT) stage_adjgrad_kernel(const StageParams g, const StageParams a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* D_s = reinterpret_cast<double*>(smem_raw + StageSmem<N, double>::d_off);
  for (int i = threadIdx.x; i < Shape<N>::n * Shape<N>::n; i += Shape<N>::NT) D_s[i] = g.D[i];
  stage_tile<N, double, GMODE>(g, blockIdx.x, smem_raw);
  __syncthreads();
  stage_tile<N, double, kModeAdj>(a, blockIdx.x, smem_raw);
}

template <int N, int GMODE>
cudaError_t launch_stage_adjgrad_t(const StageParams& g, const StageParams& a, cudaStream_t s) {
  const size_t smem = StageSmem<N, double>::bytes;
  static std::atomic<unsigned long long> ready{0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (!(ready.load(std::memory_order_relaxed) & bit)) {
    err = cudaFuncSetAttribute(stage_adjgrad_kernel<N, GMODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    ready.fetch_or(bit, std::memory_order_relaxed);
  }
  const long long blocks = (g.nel + Shape<N>::EPB - 1) / Shape<N>::EPB;
  if (blocks <= 0) return cudaSuccess;
  StageParams gq = g, aq = a;
  finish_stage_params(gq);
  finish_stage_params(aq);
  stage_adjgrad_kernel<N, GMODE><<<(unsigned)blocks, Shape<N>::NT, smem, s>>>(gq, aq);
  return cudaGetLastError();
}

// g.rout set: the gradient terms take the operator output from it (GRAD_FACE).
inline cudaError_t launch_stage_adjgrad_any(int N, const StageParams& g, const StageParams& a, cudaStream_t s) {
  switch (N) {
#define DGW_GCASE(NN)                                                                                      \
  case NN:                                                                                                 \
    return g.rout ? launch_stage_adjgrad_t<NN, kModeGradFace>(g, a, s) : launch_stage_adjgrad_t<NN, kModeGrad>(g, a, s);
    DGW_GCASE(1) DGW_GCASE(2) DGW_GCASE(3) DGW_GCASE(4) DGW_GCASE(5) DGW_GCASE(6) DGW_GCASE(7)
#undef DGW_GCASE
    default:
      return cudaErrorInvalidValue;
  }
}

// Adjoint modes (FP64 only).
inline cudaError_t launch_stage_adjoint_any(int N, int mode, const StageParams& p, cudaStream_t s) {
#define DGW_ACASE(NN)                                                                                  \
  case NN:                                                                                             \
    return mode == kModeAdj ? launch_stage_t<NN, double, kModeAdj>(p, s) : launch_stage_t<NN, double, kModeGrad>(p, s);
  switch (N) {
    DGW_ACASE(1) DGW_ACASE(2) DGW_ACASE(3) DGW_ACASE(4) DGW_ACASE(5) DGW_ACASE(6) DGW_ACASE(7)
#undef DGW_ACASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace dgw
