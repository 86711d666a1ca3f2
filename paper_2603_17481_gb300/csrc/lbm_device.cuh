// lbm_device.cuh -- device-side building blocks shared by the sm_103a kernels of liblbm.
//
// Lattice tables, population storage formats, the fixed-point phi format, the kernel parameter
// block and the tile geometry. The velocity order is the one of include/lbm.h: |c|^2 ascending,
// then (c_z, c_y, c_x) lexicographic.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

constexpr float kCs2 = 1.0f / 3.0f;

// ---------------------------------------------------------------------------------------------
// Lattices (Sec. 2.1). c(i, a) and w(i) fold to immediates inside unrolled loops.
// ---------------------------------------------------------------------------------------------
struct D2Q9 {
  static constexpr int Q = 9, D = 2;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0},  {0, -1, 0}, {-1, 0, 0}, {1, 0, 0}, {0, 1, 0},
                             {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}};
    return t[i][a];
  }
  __host__ __device__ static constexpr float w(int i) {
    return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
  }
  __host__ __device__ static constexpr double wd(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
  // index of -c_i: within each |c|^2 class the order is reversed by negation
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i < 5 ? 5 - i : 13 - i); }
};

struct D3Q19 {
  static constexpr int Q = 19, D = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[19][3] = {{0, 0, 0},   {0, 0, -1},  {0, -1, 0},  {-1, 0, 0}, {1, 0, 0},
                              {0, 1, 0},   {0, 0, 1},   {0, -1, -1}, {-1, 0, -1}, {1, 0, -1},
                              {0, 1, -1},  {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0}, {1, 1, 0},
                              {0, -1, 1},  {-1, 0, 1},  {1, 0, 1},   {0, 1, 1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr float w(int i) {
    return i == 0 ? 1.0f / 3.0f : (i < 7 ? 1.0f / 18.0f : 1.0f / 36.0f);
  }
  __host__ __device__ static constexpr double wd(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i < 7 ? 7 - i : 25 - i); }
};

struct D3Q27 {
  static constexpr int Q = 27, D = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[27][3] = {{0, 0, 0},   {0, 0, -1},  {0, -1, 0},  {-1, 0, 0},  {1, 0, 0},
                              {0, 1, 0},   {0, 0, 1},   {0, -1, -1}, {-1, 0, -1}, {1, 0, -1},
                              {0, 1, -1},  {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 1, 0},
                              {0, -1, 1},  {-1, 0, 1},  {1, 0, 1},   {0, 1, 1},   {-1, -1, -1},
                              {1, -1, -1}, {-1, 1, -1}, {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},
                              {-1, 1, 1},  {1, 1, 1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr float w(int i) {
    return i == 0 ? 8.0f / 27.0f : (i < 7 ? 2.0f / 27.0f : (i < 19 ? 1.0f / 54.0f : 1.0f / 216.0f));
  }
  __host__ __device__ static constexpr double wd(int i) {
    return i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i < 7 ? 7 - i : (i < 19 ? 25 - i : 45 - i));
  }
};

// Stencil lattice of the discrete derivatives of phi: D2Q9 in 2D, D3Q27 in 3D (Eqs. 22-23, 35, 57).
template <int DIM> struct StencilOf;
template <> struct StencilOf<2> { using type = D2Q9; };
template <> struct StencilOf<3> { using type = D3Q27; };

// A direction is "positive" when its first non-zero component in (z, y, x) order is +1; every
// link of the stencil is visited once through its positive direction.
template <class L> __host__ __device__ constexpr bool positive(int i) {
  return L::c(i, 2) > 0 || (L::c(i, 2) == 0 && (L::c(i, 1) > 0 || (L::c(i, 1) == 0 && L::c(i, 0) > 0)));
}

// ---------------------------------------------------------------------------------------------
// Population storage. FP32 stores f itself; FP16/BF16 store f / w_i (deviation from the rest
// equilibrium f = w_i p* with p* = 0), computed and accumulated in FP32.
// ---------------------------------------------------------------------------------------------
template <int S> struct Store;
template <> struct Store<0> {
  using T = float;
  __device__ static __forceinline__ float ld(const T *p, float) { return __ldg(p); }
  __device__ static __forceinline__ void st(T *p, float v, float) { *p = v; }
  // stores f given f / w
  __device__ static __forceinline__ void st_w(T *p, float v_over_w, float w) { *p = w * v_over_w; }
};
template <> struct Store<1> {
  using T = __half;
  __device__ static __forceinline__ float ld(const T *p, float w) { return __half2float(__ldg(p)) * w; }
  __device__ static __forceinline__ void st(T *p, float v, float w) { *p = __float2half_rn(v / w); }
  __device__ static __forceinline__ void st_w(T *p, float v_over_w, float) { *p = __float2half_rn(v_over_w); }
};
template <> struct Store<2> {
  using T = __nv_bfloat16;
  __device__ static __forceinline__ float ld(const T *p, float w) { return __bfloat162float(__ldg(p)) * w; }
  __device__ static __forceinline__ void st(T *p, float v, float w) { *p = __float2bfloat16_rn(v / w); }
  __device__ static __forceinline__ void st_w(T *p, float v_over_w, float) { *p = __float2bfloat16_rn(v_over_w); }
};

// Moment-record storage (the paper's thread-safe representation, Sec. 2.1): instead of Q
// populations a cell stores the 16-float record of its post-collision state, four float4 kept as
// four arrays of N float4 (buf[k * N + n] = q_k of cell n, so a warp's loads of one q_k are 512
// contiguous bytes):
//   q0 = (C0, C1, u0, u1), q1 = (u2, r0, r1, r2), q2 = (B00, B11, B22, B01), q3 = (B02, B12, 0, 0)
// with r = F / rho, B = (1 - omega) A2 (the regularized non-equilibrium moment of Eq. 14 after
// relaxation), C0 = p* - 1.5 |u|^2 - 1.5 tr B - 1.5 u.r and C1 = 3 - 4.5 |u|^2 - 4.5 tr B. The
// post-collision population of direction c is then (Eqs. 3, 11, 15-17 with cs^2 = 1/3)
//   f / w = E + O,  E = C0 + 4.5 (c.u)(c.u + c.r) + 4.5 c.B.c,
//                   O = (c.u)(C1 + 4.5 (c.u)^2 + 13.5 c.B.c) - 9 c.B.u + 1.5 c.r,
// so a cell pulls f_i(x) by evaluating this at the record of x - c_i.
constexpr int kStoreRecord = 3;
template <> struct Store<kStoreRecord> {
  using T = float4;
};
constexpr int kRecordWords = 4;  // float4 per cell (arrays of the buffer)

// f_i / w_i of direction i of the record (q0, q1, q2, q3)
template <class L>
__device__ __forceinline__ float record_f_over_w(int i, const float4 q0, const float4 q1, const float4 q2,
                                                 const float4 q3) {
  const int c0 = L::c(i, 0), c1 = L::c(i, 1), c2 = L::c(i, 2);
  if (c0 == 0 && c1 == 0 && c2 == 0) return q0.x;
  const float u0 = q0.z, u1 = q0.w, u2 = q1.x;
  const float B00 = q2.x, B11 = q2.y, B22 = q2.z, B01 = q2.w, B02 = q3.x, B12 = q3.y;
  // c.u, c.r, c.B.c and c.B.u with the zero components of c dropped after unrolling
  float cu = 0.f, cr = 0.f, cbc = 0.f, cbu = 0.f;
  if (c0) { cu += c0 * u0; cr += c0 * q1.y; cbc += B00; cbu += c0 * (B00 * u0 + B01 * u1 + B02 * u2); }
  if (c1) { cu += c1 * u1; cr += c1 * q1.z; cbc += B11; cbu += c1 * (B01 * u0 + B11 * u1 + B12 * u2); }
  if (c2) { cu += c2 * u2; cr += c2 * q1.w; cbc += B22; cbu += c2 * (B02 * u0 + B12 * u1 + B22 * u2); }
  if (c0 && c1) cbc += 2.0f * c0 * c1 * B01;
  if (c0 && c2) cbc += 2.0f * c0 * c2 * B02;
  if (c1 && c2) cbc += 2.0f * c1 * c2 * B12;
  const float t = 4.5f * cu;
  const float E = q0.x + t * (cu + cr) + 4.5f * cbc;
  const float O = cu * (q0.y + t * cu + 13.5f * cbc) - 9.0f * cbu + 1.5f * cr;
  return E + O;
}

// ---------------------------------------------------------------------------------------------
// phi is stored as a signed 2.30 fixed-point integer: phi = v * 2^-30. Every term of the phase
// update is applied as an antisymmetric link transfer rounded once to this grid, so sum(phi) is
// conserved exactly (integer arithmetic), and stencil differences are exact integer differences.
// ---------------------------------------------------------------------------------------------
constexpr float kQ30 = 1073741824.0f;          // 2^30
constexpr float kInvQ30 = 1.0f / 1073741824.0f; // 2^-30
__device__ __forceinline__ float phi_of(int32_t v) { return __int2float_rn(v) * kInvQ30; }
// a - b taken modulo 2^32: exact whenever |phi_a - phi_b| < 2
__device__ __forceinline__ float dphi_of(int32_t a, int32_t b) {
  return __int2float_rn((int32_t)((uint32_t)a - (uint32_t)b)) * kInvQ30;
}

// Interfacial indicator of Eq. 58 on phi clamped to [0, 1] (Sec. 2.3.1). Used by the gate of the
// near-contact kernel and by the hydrodynamic kernel to know where a repulsive force was written:
// both must take the same decision, so both call this one function.
__device__ __forceinline__ float q_gate_value(int32_t v) {
  float pc = fminf(fmaxf(phi_of(v), 0.0f), 1.0f);
  return __fmul_rn(pc, __fsub_rn(1.0f, pc));
}

__host__ __device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}
// Programmatic dependent launch. The step kernels are launched so that each may be scheduled while
// the kernel before it on the stream finishes; the first thing each does is wait for that grid to
// complete (its memory operations done and visible), so nothing is read or written earlier. It then
// lets the next step kernel be scheduled. Launched without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Periodic wrap with a fast path for in-range coordinates.
__device__ __forceinline__ int wrapn(int a, int n) { return (unsigned)a < (unsigned)n ? a : wrapi(a, n); }

// ---------------------------------------------------------------------------------------------
// Kernel parameter block (derived on the host in FP64, stored as FP32).
// ---------------------------------------------------------------------------------------------
struct KParams {
  int nx, ny, nz;
  long long N;
  float rho_g, drho;     // rho(phi) = rho_g + drho * phi
  float mu_g, dmu;       // mu(phi)  = mu_g + dmu * phi
  float beta4, kap;      // mu_phi = beta4 phi (phi-1)(phi-1/2) - kap lap(phi)
  float rho_bar;         // buoyancy reference
  float g[3];
  int nci_on, w;
  float A_rep, h0, p, q_th, eta, cos_opp, eps_q, eps_n, eps;
  float Dlap;            // D * 2 / cs^2  (Laplacian link weight factor, Eq. 23 times D)
  float kc;              // kappa / cs^2  (compressive link factor, Eq. 35)
  double rho_g64, drho64;  // the density rule in FP64 for the FP64 momentum integral
};

// Near-contact window offsets sorted by (|r|^2, canonical index); filled by the host.
struct NciOffset {
  int8_t dx, dy, dz, d2;
};
constexpr int kMaxOffsets = 342;  // (2*3+1)^3 - 1

// Tile geometry (threads per block = TX*TY*TZ, one cell per thread).
template <int DIM> struct Tile;
template <> struct Tile<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct Tile<3> { static constexpr int X = 32, Y = 4, Z = 2; };

template <int DIM> struct NciTile;
template <> struct NciTile<2> { static constexpr int X = 32, Y = 16, Z = 1; };
template <> struct NciTile<3> { static constexpr int X = 32, Y = 8, Z = 4; };

// The phase-field kernel lists near-contact tiles, so both use the same tiling.
template <int DIM> struct PhaseTile : NciTile<DIM> {};

}  // namespace lbm
