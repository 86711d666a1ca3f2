// kernels_phase.cu -- the phase-field half of a time step (Sec. 2.1.1): Eq. 28,
//   phi^{n+1} = phi^n - div_h(u phi) + D lap_h(phi) + S_comp,
// with MUSCL-minmod face fluxes (Eqs. 29-34), the isotropic Laplacian (Eq. 23) and the
// isotropic compressive divergence S_comp = -(kappa / cs^2) sum_i w_i c_i . a(x + c_i),
// a = phi (1 - phi) n, kappa = 4 D / eps (Eqs. 26, 35).
//
// Face-flux form. The D2Q9 and D3Q27 weights are tensor products of the 1D weights
// (1, 4, 1) / 6, w_i = s(c_x) s(c_y) [s(c_z)] / 6^d with s(0) = 4, s(+-1) = 1. Writing s = 6 + d2
// (d2 the 1D second difference), the isotropic Laplacian 6 (sum_i w_i phi(x + c_i) - phi) expands
// into sum_a d2_a(B_a phi) with, in 3D, B_x = s_y s_z / 36, B_y = s_z / 6, B_z = 1 (2D: B_x = s_y / 6,
// B_y = 1), and the isotropic divergence sum_i w_i c_i . a(x + c_i) into a difference of face
// sums with weights s_b s_c / 216 (2D: s_b / 36) over the two transverse axes. Hence
//   phi^{n+1}(x) - phi^n(x) = sum_a [ tau_a(x - e_a / 2) - tau_a(x + e_a / 2) ],
//   tau_a(x + e_a/2) = u_f phi_up + D B_a (phi(x) - phi(x + e_a))
//                      + 3 kappa W_a (a_a(x) + a_a(x + e_a)),   W_a = s_b s_c / 216 (2D s_b / 36),
// which equals Eq. 28 term by term in exact arithmetic. Each face transfer tau is computed once
// per block (the cells of a tile plus the faces on its low boundary), rounded once to the 2^-30
// fixed-point phi grid and applied with opposite signs on its two cells, so sum(phi) is exactly
// conserved. The kernel also lists the tiles of the near-contact kernel (same tiling) that hold an
// interfacial cell of phi^{n+1}, so the next near-contact pass visits only those.
#include <cstdlib>

#include "launch.h"
#include "phase3_march.cuh"

namespace lbm {

template <int DIM> struct PhaseGeom {
  static constexpr int TX = PhaseTile<DIM>::X, TY = PhaseTile<DIM>::Y, TZ = PhaseTile<DIM>::Z;
  static constexpr int HX = TX + 4, HY = TY + 4, HZ = DIM == 3 ? TZ + 4 : 1;  // phi, halo 2
  static constexpr int AX = TX + 2, AY = TY + 2, AZ = DIM == 3 ? TZ + 2 : 1;  // a, halo 1
  static constexpr int NB = HX * HY * HZ, NA = AX * AY * AZ, NT = TX * TY * TZ;
  // face transfers: faces of the tile cells on their high side plus the low boundary faces
  static constexpr int FX = (TX + 1) * TY * TZ, FY = TX * (TY + 1) * TZ, FZ = DIM == 3 ? TX * TY * (TZ + 1) : 0;
};

__device__ __forceinline__ int32_t minmod_i(int32_t a, int32_t b) {
  if (a > 0 && b > 0) return a < b ? a : b;
  if (a < 0 && b < 0) return a > b ? a : b;
  return 0;
}

// Transfer across the face between cells p and p + e_AX (tile-local coordinates, p may be one
// cell below the tile). s_phi has halo 2, s_a halo 1.
template <int DIM, int AXIS>
__device__ __forceinline__ int32_t face_transfer(const KParams &P, const int32_t *s_phi, const float *s_a,
                                                 const float *__restrict__ u, int px, int py, int pz,
                                                 int gx, int gy, int gz) {
  using G = PhaseGeom<DIM>;
  constexpr int SX = 1, SY = G::HX, SZ = G::HX * G::HY;         // phi-box strides
  constexpr int AXS = 1, AYS = G::AX, AZS = G::AX * G::AY;       // a-box strides
  constexpr int E = AXIS == 0 ? SX : (AXIS == 1 ? SY : SZ);
  constexpr int EA = AXIS == 0 ? AXS : (AXIS == 1 ? AYS : AZS);
  const int b = (DIM == 3 ? (pz + 2) * SZ : 0) + (py + 2) * SY + px + 2;
  const int ba = (DIM == 3 ? (pz + 1) * AZS : 0) + (py + 1) * AYS + px + 1;
  const int32_t v0 = s_phi[b], v1 = s_phi[b + E];

  // diffusion D B_a (phi(p) - phi(p + e)) with exact integer differences
  float dif;
  if (DIM == 3 && AXIS == 0) {
    // B_x = s_y s_z / 36
    float acc = 0.f;
#pragma unroll
    for (int dz = -1; dz <= 1; dz++)
#pragma unroll
      for (int dy = -1; dy <= 1; dy++) {
        const float wgt = (dy ? 1.f : 4.f) * (dz ? 1.f : 4.f);
        const int o = dy * SY + dz * SZ;
        acc = __fmaf_rn(wgt, dphi_of(s_phi[b + o], s_phi[b + o + E]), acc);
      }
    dif = __fmul_rn(acc, 1.0f / 36.0f);
  } else if ((DIM == 3 && AXIS == 1) || (DIM == 2 && AXIS == 0)) {
    // B = s_z / 6 (3D, y faces) or s_y / 6 (2D, x faces)
    constexpr int T = DIM == 3 ? SZ : SY;
    float acc = __fmul_rn(4.f, dphi_of(v0, v1));
    acc = __fadd_rn(acc, dphi_of(s_phi[b - T], s_phi[b - T + E]));
    acc = __fadd_rn(acc, dphi_of(s_phi[b + T], s_phi[b + T + E]));
    dif = __fmul_rn(acc, 1.0f / 6.0f);
  } else {
    dif = dphi_of(v0, v1);
  }
  float tau = __fmul_rn(P.Dlap * (1.0f / 6.0f), dif);  // Dlap = 6 D

  // compressive transfer 3 kappa W_a (a_a(p) + a_a(p + e)), W_a = s_b s_c / 216 (2D: s_b / 36)
  {
    const float *sa = s_a + AXIS * G::NA;
    float acc = 0.f;
    if (DIM == 3) {
      constexpr int T1 = AXIS == 0 ? AYS : AXS, T2 = AXIS == 2 ? AYS : AZS;
#pragma unroll
      for (int d2 = -1; d2 <= 1; d2++)
#pragma unroll
        for (int d1 = -1; d1 <= 1; d1++) {
          const float wgt = (d1 ? 1.f : 4.f) * (d2 ? 1.f : 4.f);
          const int o = d1 * T1 + d2 * T2;
          acc = __fmaf_rn(wgt, __fadd_rn(sa[ba + o], sa[ba + o + EA]), acc);
        }
      acc = __fmul_rn(acc, 1.0f / 216.0f);
    } else {
      constexpr int T1 = AXIS == 0 ? AYS : AXS;
      acc = __fmul_rn(4.f, __fadd_rn(sa[ba], sa[ba + EA]));
      acc = __fadd_rn(acc, __fadd_rn(sa[ba - T1], sa[ba - T1 + EA]));
      acc = __fadd_rn(acc, __fadd_rn(sa[ba + T1], sa[ba + T1 + EA]));
      acc = __fmul_rn(acc, 1.0f / 36.0f);
    }
    tau = __fadd_rn(tau, __fmul_rn(P.kc * kCs2 * 3.0f, acc));  // kc = kappa / cs^2 -> 3 kappa
  }

  // MUSCL face flux u_f phi_up (Eqs. 30-34)
  {
    const int32_t vm = s_phi[b - E], vp = s_phi[b + 2 * E];
    const int32_t s0 = minmod_i(v0 - vm, v1 - v0);
    const int32_t s1 = minmod_i(v1 - v0, vp - v1);
    // global cells p and p + e (periodic)
    const int n0x = P.nx, n0y = P.ny, n0z = P.nz;
    int qx = gx, qy = gy, qz = gz;
    if (AXIS == 0) qx = qx == n0x - 1 ? 0 : qx + 1;
    if (AXIS == 1) qy = qy == n0y - 1 ? 0 : qy + 1;
    if (AXIS == 2) qz = qz == n0z - 1 ? 0 : qz + 1;
    const long long N = P.N;
    const float ua = __ldg(u + AXIS * N + gx + (long long)n0x * (gy + (long long)n0y * gz));
    const float ub = __ldg(u + AXIS * N + qx + (long long)n0x * (qy + (long long)n0y * qz));
    const float uf = __fmul_rn(0.5f, __fadd_rn(ua, ub));
    // upwind state; exact integer slopes, FP32 sum (no 64-bit conversion, which runs on the FP64 pipe)
    const float pup = uf >= 0.0f ? (__int2float_rn(v0) + 0.5f * __int2float_rn(s0)) * kInvQ30
                                 : (__int2float_rn(v1) - 0.5f * __int2float_rn(s1)) * kInvQ30;
    tau = __fadd_rn(tau, __fmul_rn(uf, pup));
  }
  return __float2int_rn(__fmul_rn(tau, kQ30));
}

template <int DIM>
__global__ void __launch_bounds__(PhaseGeom<DIM>::NT)
k_phase(const KParams P, const int32_t *__restrict__ phi, const float *__restrict__ u,
        int32_t *__restrict__ phi_out, int *__restrict__ tiles, int *__restrict__ ntiles) {
  pdl_enter();
  using G = PhaseGeom<DIM>;
  using SL = typename StencilOf<DIM>::type;
  __shared__ int32_t s_phi[G::NB];
  __shared__ float s_a[3 * G::NA];
  __shared__ int32_t s_tx[G::FX], s_ty[G::FY], s_tz[DIM == 3 ? G::FZ : 1];

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + G::TX * (ty + G::TY * tz);
  const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * G::TY, z0 = blockIdx.z * G::TZ;
  const int nx = P.nx, ny = P.ny, nz = P.nz;

  // stage phi (halo 2) row by row: rows of HX = TX + 4 values
  {
    const int xl = wrapn(x0 - 2 + tx, nx);
    const int xr = wrapn(x0 + 30 + (tx & 3), nx);
    constexpr int NROWS = G::HY * G::HZ, NW = G::TY * G::TZ;
    for (int r = ty + G::TY * tz; r < NROWS; r += NW) {
      const int ry = r % G::HY, rz = r / G::HY;
      const int Y = wrapn(y0 + ry - 2, ny);
      const int Z = DIM == 3 ? wrapn(z0 + rz - 2, nz) : 0;
      const int32_t *row = phi + (long long)nx * (Y + (long long)ny * Z);
      s_phi[r * G::HX + tx] = row[xl];
      if (tx < 4) s_phi[r * G::HX + 32 + tx] = row[xr];
    }
  }
  __syncthreads();

  // compressive vector a = phi (1 - phi) grad(phi) / (|grad(phi)| + eps_n) on the tile + 1 halo
  for (int t = tid; t < G::NA; t += G::NT) {
    const int ax = t % G::AX, ay = (t / G::AX) % G::AY, az = t / (G::AX * G::AY);
    const int b = (DIM == 3 ? (az + 1) * G::HX * G::HY : 0) + (ay + 1) * G::HX + ax + 1;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int i = 1; i < SL::Q; i++) {
      if (!positive<SL>(i)) continue;
      const int o = SL::c(i, 0) + G::HX * (SL::c(i, 1) + G::HY * SL::c(i, 2));
      const float d = SL::w(i) * dphi_of(s_phi[b + o], s_phi[b - o]);
      g0 += SL::c(i, 0) * d;
      g1 += SL::c(i, 1) * d;
      if (DIM == 3) g2 += SL::c(i, 2) * d;
    }
    g0 *= 3.0f; g1 *= 3.0f; g2 *= 3.0f;
    const float ph = phi_of(s_phi[b]);
    const float s = ph * (1.0f - ph) / (sqrtf(g0 * g0 + g1 * g1 + g2 * g2) + P.eps_n);
    s_a[t] = g0 * s;
    s_a[G::NA + t] = g1 * s;
    s_a[2 * G::NA + t] = g2 * s;
  }
  __syncthreads();

  // face transfers: x faces (TX + 1) x TY x TZ with the low face of the tile first
  for (int t = tid; t < G::FX; t += G::NT) {
    const int fx = t % (G::TX + 1), fy = (t / (G::TX + 1)) % G::TY, fz = t / ((G::TX + 1) * G::TY);
    const int px = fx - 1;  // left cell, tile-local
    const int gx = wrapn(x0 + px, nx), gy = wrapn(y0 + fy, ny), gz = DIM == 3 ? wrapn(z0 + fz, nz) : 0;
    s_tx[t] = face_transfer<DIM, 0>(P, s_phi, s_a, u, px, fy, fz, gx, gy, gz);
  }
  for (int t = tid; t < G::FY; t += G::NT) {
    const int fx = t % G::TX, fy = (t / G::TX) % (G::TY + 1), fz = t / (G::TX * (G::TY + 1));
    const int py = fy - 1;
    const int gx = wrapn(x0 + fx, nx), gy = wrapn(y0 + py, ny), gz = DIM == 3 ? wrapn(z0 + fz, nz) : 0;
    s_ty[t] = face_transfer<DIM, 1>(P, s_phi, s_a, u, fx, py, fz, gx, gy, gz);
  }
  if (DIM == 3) {
    for (int t = tid; t < G::FZ; t += G::NT) {
      const int fx = t % G::TX, fy = (t / G::TX) % G::TY, fz = t / (G::TX * G::TY);
      const int pz = fz - 1;
      const int gx = wrapn(x0 + fx, nx), gy = wrapn(y0 + fy, ny), gz = wrapn(z0 + pz, nz);
      s_tz[t] = face_transfer<DIM, 2>(P, s_phi, s_a, u, fx, fy, pz, gx, gy, gz);
    }
  }
  __syncthreads();

  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  const bool inb = x < nx && y < ny && z < nz;
  bool gated = false;
  if (inb) {
    const int b = (DIM == 3 ? (tz + 2) * G::HX * G::HY : 0) + (ty + 2) * G::HX + tx + 2;
    int32_t acc = s_tx[tx + (G::TX + 1) * (ty + G::TY * tz)] - s_tx[tx + 1 + (G::TX + 1) * (ty + G::TY * tz)];
    acc += s_ty[tx + G::TX * (ty + (G::TY + 1) * tz)] - s_ty[tx + G::TX * (ty + 1 + (G::TY + 1) * tz)];
    if (DIM == 3) acc += s_tz[tx + G::TX * (ty + G::TY * tz)] - s_tz[tx + G::TX * (ty + G::TY * (tz + 1))];
    const int32_t vn = s_phi[b] + acc;
    phi_out[(long long)x + (long long)nx * (y + (long long)ny * z)] = vn;
    gated = q_gate_value(vn) >= P.q_th;
  }
  if (tiles) {
    const int any = __syncthreads_or(gated);
    if (any && tid == 0) {
      const int tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
      tiles[atomicAdd(ntiles, 1)] = tile;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// 3D: a block owns a 32 x 8 column of cells over zc planes (zc = 16, or 8 or 4 on grids too small
// to fill the GPU with 16-plane columns) and marches along z, keeping ring
// buffers of planes in shared memory. The D3Q27 weights factor as s(c_x) s(c_y) s(c_z) / 216, so
//   RZ(k)   = phi(k-1) + 4 phi(k) + phi(k+1)
//   PSXY(k) = s_x s_y phi(k)
//   grad_x phi = (1/72) s_y [RZ(x+1) - RZ(x-1)],  grad_y phi = (1/72) s_x [RZ(y+1) - RZ(y-1)],
//   grad_z phi = (1/72) [PSXY(k+1) - PSXY(k-1)],
// and the face transfers of the header use the same planes: B_x (phi(p) - phi(p+e)) =
// (1/36) s_y [RZ(p) - RZ(p+e)], B_y (...) = (1/6) [RZ(p) - RZ(p+e)], and the compressive sums
// s_y s_z a_x, s_x s_z a_y, s_x s_y a_z from the z-smoothed planes AXZ, AYZ and the in-plane ASXY.
// Every a value and every face transfer is computed once per block; the faces on block borders
// are computed by both neighbours from identical inputs with the same rounded operations. The plane
// sums are FP32 over an FP32 copy of each phi plane (PF); the fixed-point planes (PH) give the exact
// z-face differences and the update itself. Nothing here converts from 64-bit integers: those
// conversions run on the FP64 pipe, which GB300 keeps narrow. Each face transfer is rounded once to
// the 2^-30 grid, so the sum of phi is conserved exactly whatever the FP32 rounding inside.
// ---------------------------------------------------------------------------------------------
struct Phase3 {
  static constexpr int TX = 32, TY = 8, ZC = 16, NT = TX * TY;  // ZC: the largest z chunk
  static constexpr int PX = TX + 4, PY = TY + 4, NP = PX * PY;  // phi / RZ planes (halo 2)
  // PSXY / a planes (halo 1): TX + 2 columns used, stored with the pitch of the phi planes so that
  // a warp's consecutive entries are consecutive words (no bank conflicts) and pi() = qi() + PX + 1
  static constexpr int QW = TX + 2, QX = PX, QY = TY + 2, NQ = QX * QY;
  static constexpr int NC = TX * TY;
  static constexpr int NFX = PX * TY, NFY = TX * (TY + 1);  // x faces at pitch PX (TX + 1 used)
  // near-contact tiles (NY x NZ in y, z) of the block's column: flags per z chunk of the march
  static constexpr int NY = NciTile<3>::Y, NZ = NciTile<3>::Z, FY = TY / NY;
  static_assert(TY % NY == 0 && ZC % NZ == 0 && NZ == 4, "near-contact tiles nest in the march blocks");
  static constexpr int NFLG = (ZC / NZ) * FY;
  static constexpr size_t smem = sizeof(float) * (2 * NP + 4 * NQ) + sizeof(int32_t) * 4 * NP +
                                 sizeof(float) * 4 * NP +
                                 sizeof(float) * (NQ + 2 * NQ + 2 * NC + QX * TY + TX * QY + 2 * NC) +
                                 sizeof(int32_t) * (NFX + NFY + 2 * NC + NFLG);
  __device__ static __forceinline__ int pi(int lx, int ly) { return (ly + 2) * PX + lx + 2; }
  __device__ static __forceinline__ int qi(int lx, int ly) { return (ly + 1) * QX + lx + 1; }
};

__device__ __forceinline__ float s141(float a, float b, float c) { return a + 4.0f * b + c; }

// minmod(a, b): the argument of smaller magnitude when both have the same sign, else 0. a b cannot
// underflow here (nonzero phi differences are at least 2^-30), so the sign test is exact.
__device__ __forceinline__ float minmod_f(float a, float b) {
  return a * b > 0.0f ? copysignf(fminf(fabsf(a), fabsf(b)), a) : 0.0f;
}

// Upwind MUSCL state at the face between cells p and p + e (Eqs. 30-34) from phi at p - e, p, p + e,
// p + 2e: phi(p) + minmod(phi(p) - phi(p-e), phi(p+e) - phi(p)) / 2 when u_f >= 0, else
// phi(p+e) - minmod(phi(p+e) - phi(p), phi(p+2e) - phi(p+e)) / 2. The triple (L, C, R) is selected
// first and one limiter evaluated: minmod(-a, -b) = -minmod(a, b) makes C + minmod(C - L, R - C) / 2
// with (L, C, R) = (phi(p+2e), phi(p+e), phi(p)) equal to the second form, bit for bit.
__device__ __forceinline__ float upwind_f(float uf, float vm, float v0, float v1, float vp) {
  const bool pos = uf >= 0.0f;
  const float L = pos ? vm : vp, C = pos ? v0 : v1, R = pos ? v1 : v0;
  return C + 0.5f * minmod_f(C - L, R - C);
}

// Resident k_phase3 blocks per SM its registers are sized for: 4 (64 registers) measured 0.110 ms on
// 256x128x128, against 0.123 ms for 3 and 0.153 ms for 5 (which spills).
#ifndef LBM_PHASE_MINB
#define LBM_PHASE_MINB 4
#endif

__global__ void __launch_bounds__(Phase3::NT, LBM_PHASE_MINB)
k_phase3(const KParams P, const int32_t *__restrict__ phi, const float *__restrict__ u,
         int32_t *__restrict__ phi_out, int *__restrict__ tiles, int *__restrict__ ntiles, const int zc) {
  pdl_enter();
  using G = Phase3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *RZ = reinterpret_cast<float *>(smem_raw);           // [2][NP]
  float *PS = RZ + 2 * G::NP;                                // [4][NQ]
  int32_t *PH = reinterpret_cast<int32_t *>(PS + 4 * G::NQ);  // [4][NP] fixed point
  float *PF = reinterpret_cast<float *>(PH + 4 * G::NP);      // [4][NP] FP32 copy
  float *AZ = PF + 4 * G::NP;                                // [NQ]: a_z of plane k + 1
  float *AXZ = AZ + G::NQ;                                   // [NQ]
  float *AYZ = AXZ + G::NQ;                                  // [NQ]
  float *ASXY = AYZ + G::NQ;                                 // [2][NC]
  float *UX = ASXY + 2 * G::NC;                              // [TY][QX]: lx -1..32 at columns 0..33
  float *UY = UX + G::QX * G::TY;                            // [QY][TX]: ly -1..TY
  float *UZ = UY + G::TX * G::QY;                            // [2][NC]
  int32_t *TXF = reinterpret_cast<int32_t *>(UZ + 2 * G::NC);  // [TY][TX+1]
  int32_t *TYF = TXF + G::NFX;                                 // [TY+1][TX]
  int32_t *TZF = TYF + G::NFY;                                 // [2][NC]
  int *FLG = TZF + 2 * G::NC;                                  // near-contact tile flags

  const int lane = threadIdx.x, wy = threadIdx.y, tid = lane + 32 * wy;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const long long N = P.N;
  const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * G::TY;
  const int zb = blockIdx.z * zc, ze = min(zb + zc, nz);
  // face coefficients: D of the z link, with the 1/36 (x) and 1/6 (y) of the smoothed differences;
  // 3 kappa / 216 on the smoothed compressive sums
  const float D = P.Dlap * (1.0f / 6.0f), Dx = D * (1.0f / 36.0f), Dy = D * (1.0f / 6.0f);
  const float k3s = P.kc * kCs2 * 3.0f * (1.0f / 216.0f);
  // this thread's x columns for plane loads: phi planes (lx = lane - 2, and 30..33 for lanes 0..3),
  // u_x planes (lx = lane - 1, and 31..32 for lanes 0..1)
  const int xa = wrapn(x0 + lane - 2, nx), xb = wrapn(x0 + 30 + (lane & 3), nx);
  const int ua = wrapn(x0 + lane - 1, nx), ub = wrapn(x0 + 31 + (lane & 1), nx);
  const int xc = wrapn(x0 + lane, nx);
  // row offsets within a plane (constant over the march): phi rows y0 + r - 2, u_y rows y0 + r - 1
  int yph[2], yuy[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    yph[h] = nx * wrapn(y0 + wy + h * G::TY - 2, ny);
    yuy[h] = nx * wrapn(y0 + wy + h * G::TY - 1, ny);
  }
  const int yown = nx * wrapn(y0 + wy, ny);
  const long long plane = (long long)nx * ny;
  // shared-memory index of the halo-1 entries t = tid and tid + NT, and of the x faces t = tid and
  // tid + NT as (plane index, row): also constant over the march
  static_assert(G::NQ <= 2 * G::NT && G::NFX <= 2 * G::NT && G::NFY <= 2 * G::NT, "two entries per thread");
  // which of this thread's entries t = tid and tid + NT are used columns (entry t of a halo-1 plane
  // is the cell at phi-plane index t + PX + 1; x face t lies left of the cell at t + 2 PX + 1)
  bool vq[2], vfx[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int t = tid + h * G::NT;
    vq[h] = t < G::NQ && t % G::QX < G::QW;
    vfx[h] = t < G::NFX && t % G::PX < G::TX + 1;
  }
  if (tid < G::NFLG) FLG[tid] = 0;

  // Plane loads are software-pipelined: the values for iteration k + 1 (phi plane k + 3, u_z plane
  // k + 2, u_x and u_y planes k + 1) are loaded into registers during iteration k.
  int32_t rphi[4];
  float ruz, rux[2], ruy[2];
  auto prefetch = [&](int kk) {
    const int32_t *pp = phi + plane * wrapn(kk + 2, nz);
#pragma unroll
    for (int h = 0; h < 2; h++) {
      if (wy + h * G::TY < G::PY) {
        rphi[2 * h] = pp[yph[h] + xa];
        if (lane < 4) rphi[2 * h + 1] = pp[yph[h] + xb];
      }
    }
    const float *uk = u + plane * wrapn(kk, nz);
    ruz = __ldg(u + 2 * N + plane * wrapn(kk + 1, nz) + yown + xc);
    rux[0] = __ldg(uk + yown + ua);
    if (lane < 2) rux[1] = __ldg(uk + yown + ub);
#pragma unroll
    for (int h = 0; h < 2; h++) {
      if (wy + h * G::TY < G::QY) ruy[h] = __ldg(uk + N + yuy[h] + xc);
    }
  };
  prefetch(zb - 4);
  // per-thread histories along z: phi of this thread's phi-plane entries (planes k, k + 1) and a_x,
  // a_y of its halo-1 entries (planes k - 1, k), so the z sums need no shared-memory reads
  float hpf[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  float hax[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, hay[2][2] = {{0.f, 0.f}, {0.f, 0.f}};

  for (int k = zb - 4; k < ze; k++) {
    const int s4k = (k + 8) & 3, s4k1 = (k + 9) & 3, s4k2 = (k + 10) & 3, s4km = (k + 7) & 3;
    // S1: phi plane k+2; u_z plane k+1; u_x, u_y planes k (from registers), then prefetch k+1
    {
      int32_t *ph = PH + s4k2 * G::NP;
      float *pf = PF + s4k2 * G::NP;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int r = wy + h * G::TY;
        if (r < G::PY) {
          ph[r * G::PX + lane] = rphi[2 * h];
          pf[r * G::PX + lane] = phi_of(rphi[2 * h]);
          if (lane < 4) {
            ph[r * G::PX + 32 + lane] = rphi[2 * h + 1];
            pf[r * G::PX + 32 + lane] = phi_of(rphi[2 * h + 1]);
          }
        }
      }
      UZ[((k + 1) & 1) * G::NC + tid] = ruz;
      UX[wy * G::QX + lane] = rux[0];
      if (lane < 2) UX[wy * G::QX + 32 + lane] = rux[1];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int r = wy + h * G::TY;
        if (r < G::QY) UY[r * G::TX + lane] = ruy[h];
      }
      if (k + 1 < ze) prefetch(k + 1);
    }
    __syncthreads();
    // S2: RZ(k+1) and PSXY(k+2)
    {
      const float *p2 = PF + s4k2 * G::NP;
      float *rz = RZ + ((k + 1) & 1) * G::NP;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int t = tid + h * G::NT;
        if (t >= G::NP) break;
        const float v2 = p2[t];  // phi plane k + 2; planes k and k + 1 of this entry are in registers
        if (k >= zb - 2) rz[t] = s141(hpf[h][0], hpf[h][1], v2);
        hpf[h][0] = hpf[h][1];
        hpf[h][1] = v2;
      }
      float *ps = PS + s4k2 * G::NQ;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int t = tid + h * G::NT;
        if (!vq[h]) continue;
        const int c = t + G::PX + 1;
        const float r0 = s141(p2[c - G::PX - 1], p2[c - G::PX], p2[c - G::PX + 1]);
        const float r1 = s141(p2[c - 1], p2[c], p2[c + 1]);
        const float r2 = s141(p2[c + G::PX - 1], p2[c + G::PX], p2[c + G::PX + 1]);
        ps[t] = s141(r0, r1, r2);
      }
    }
    __syncthreads();
    // S3: a(k+1) = phi (1 - phi) grad(phi) / (|grad(phi)| + eps_n)
    if (k >= zb - 2) {
      const float *rz = RZ + ((k + 1) & 1) * G::NP;
      const float *psp = PS + s4k2 * G::NQ, *psm = PS + s4k * G::NQ;
      const float *p1 = PF + s4k1 * G::NP;
      constexpr float gs = 1.0f / 72.0f;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int t = tid + h * G::NT;
        if (!vq[h]) continue;
        const int c = t + G::PX + 1;
        const float g0 = gs * s141(rz[c - G::PX + 1] - rz[c - G::PX - 1], rz[c + 1] - rz[c - 1],
                                   rz[c + G::PX + 1] - rz[c + G::PX - 1]);
        const float g1 = gs * s141(rz[c + G::PX - 1] - rz[c - G::PX - 1], rz[c + G::PX] - rz[c - G::PX],
                                   rz[c + G::PX + 1] - rz[c - G::PX + 1]);
        const float g2 = gs * (psp[t] - psm[t]);
        const float ph = p1[c];
        const float gg = g0 * g0 + g1 * g1 + g2 * g2;
        const float gn = gg > 0.0f ? gg * rsqrtf(gg) : 0.0f;
        const float sc = __fdividef(ph * (1.0f - ph), gn + P.eps_n);
        const float ax = g0 * sc, ay = g1 * sc;
        AZ[t] = g2 * sc;
        // z-smoothed a_x, a_y of plane k from this entry's planes k - 1, k (registers) and k + 1
        if (k >= zb) {
          AXZ[t] = s141(hax[h][0], hax[h][1], ax);
          AYZ[t] = s141(hay[h][0], hay[h][1], ay);
        }
        hax[h][0] = hax[h][1]; hax[h][1] = ax;
        hay[h][0] = hay[h][1]; hay[h][1] = ay;
      }
    }
    __syncthreads();
    // S4: in-plane s_x s_y a_z at plane k+1 (the z-smoothed a_x, a_y of plane k came with S3)
    if (k >= zb - 2) {
      const float *az = AZ;
      float *asxy = ASXY + ((k + 1) & 1) * G::NC;
      {
        const int lx = tid & 31, ly = tid >> 5;
        const int c = G::qi(lx, ly);
        const float r0 = s141(az[c - G::QX - 1], az[c - G::QX], az[c - G::QX + 1]);
        const float r1 = s141(az[c - 1], az[c], az[c + 1]);
        const float r2 = s141(az[c + G::QX - 1], az[c + G::QX], az[c + G::QX + 1]);
        asxy[tid] = s141(r0, r1, r2);
      }
    }
    __syncthreads();
    // S5: face transfers. x and y faces of plane k; z face between planes k and k+1
    {
      const float *p0 = PF + s4k * G::NP;
      if (k >= zb) {
        const float *rz = RZ + (k & 1) * G::NP;
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int t = tid + h * G::NT;
          if (!vfx[h]) continue;
          const int c = t + 2 * G::PX + 1;  // the cell left of the face
          const float di = s141(rz[c - G::PX] - rz[c - G::PX + 1], rz[c] - rz[c + 1],
                                rz[c + G::PX] - rz[c + G::PX + 1]);
          const int q = t + G::QX;
          const float cs = s141(AXZ[q - G::QX] + AXZ[q - G::QX + 1], AXZ[q] + AXZ[q + 1],
                                AXZ[q + G::QX] + AXZ[q + G::QX + 1]);
          const float vm = p0[c - 1], v0 = p0[c], v1 = p0[c + 1], vp = p0[c + 2];
          const float uf = 0.5f * (UX[t] + UX[t + 1]);
          const float up = upwind_f(uf, vm, v0, v1, vp);
          TXF[t] = __float2int_rn(kQ30 * fmaf(Dx, di, fmaf(k3s, cs, uf * up)));
        }
        for (int t = tid; t < G::NFY; t += G::NT) {
          const int lx = t % G::TX, ly = t / G::TX - 1;
          const int c = G::pi(lx, ly);
          const float di = rz[c] - rz[c + G::PX];
          const int q = G::qi(lx, ly);
          const float cs = s141(AYZ[q - 1] + AYZ[q - 1 + G::QX], AYZ[q] + AYZ[q + G::QX],
                                AYZ[q + 1] + AYZ[q + 1 + G::QX]);
          const float vm = p0[c - G::PX], v0 = p0[c], v1 = p0[c + G::PX], vp = p0[c + 2 * G::PX];
          const float uf = 0.5f * (UY[(ly + 1) * G::TX + lx] + UY[(ly + 2) * G::TX + lx]);
          const float up = upwind_f(uf, vm, v0, v1, vp);
          TYF[t] = __float2int_rn(kQ30 * fmaf(Dy, di, fmaf(k3s, cs, uf * up)));
        }
      }
      if (k >= zb - 1) {
        const int lx = tid & 31, ly = tid >> 5;
        const int c = G::pi(lx, ly);
        const float di = dphi_of(PH[s4k * G::NP + c], PH[s4k1 * G::NP + c]);
        const float vm = PF[s4km * G::NP + c], v0 = p0[c], v1 = PF[s4k1 * G::NP + c], vp = PF[s4k2 * G::NP + c];
        const float cs = ASXY[(k & 1) * G::NC + tid] + ASXY[((k + 1) & 1) * G::NC + tid];
        const float uf = 0.5f * (UZ[(k & 1) * G::NC + tid] + UZ[((k + 1) & 1) * G::NC + tid]);
        const float up = upwind_f(uf, vm, v0, v1, vp);
        TZF[((k + 1) & 1) * G::NC + tid] = __float2int_rn(kQ30 * fmaf(D, di, fmaf(k3s, cs, uf * up)));
      }
    }
    __syncthreads();
    // S6: phi^{n+1} of plane k
    if (k >= zb) {
      const int lx = tid & 31, ly = tid >> 5;
      const int x = x0 + lx, y = y0 + ly;
      if (x < nx && y < ny) {
        int32_t acc = TXF[ly * G::PX + lx] - TXF[ly * G::PX + lx + 1];
        acc += TYF[ly * G::TX + lx] - TYF[(ly + 1) * G::TX + lx];
        acc += TZF[(k & 1) * G::NC + tid] - TZF[((k + 1) & 1) * G::NC + tid];
        const int32_t vn = PH[s4k * G::NP + G::pi(lx, ly)] + acc;
        phi_out[(long long)x + (long long)nx * (y + (long long)ny * k)] = vn;
        if (tiles && q_gate_value(vn) >= P.q_th) FLG[((k - zb) / G::NZ) * G::FY + ly / G::NY] = 1;
      }
    }
  }
  if (tiles) {
    __syncthreads();
    if (tid < G::NFLG && FLG[tid]) {
      const int gtx = (nx + 31) / 32, gty = (ny + G::NY - 1) / G::NY;
      const int bzt = zb / G::NZ + tid / G::FY, byt = y0 / G::NY + tid % G::FY;
      tiles[atomicAdd(ntiles, 1)] = blockIdx.x + gtx * (byt + gty * bzt);
    }
  }
}

template <int DIM>
static cudaError_t launch_phase_dim(const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out,
                                    int *tiles, int *ntiles, cudaStream_t s) {
  using G = PhaseGeom<DIM>;
  dim3 block(G::TX, G::TY, G::TZ);
  dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, (P.nz + G::TZ - 1) / G::TZ);
  return launch_pdl(k_phase<DIM>, grid, block, 0, s, P, phi, u, phi_out, tiles, ntiles);
}

// Raises k_phase3's dynamic shared-memory limit once. Context creation calls this, so that the
// launches themselves make no non-stream CUDA call (they may be captured into a graph).
// It also records how many k_phase3 blocks the device holds at once (SMs x resident blocks), and
// the same for the register-march kernel.
static int g_phase3_slots = 0;
static int g_march_slots = 0;
#ifndef LBM_MARCH_ROWS
#define LBM_MARCH_ROWS 4
#endif
constexpr int kMarchRows = LBM_MARCH_ROWS;  // rows in y per thread of k_phase3m (2 or 4)

cudaError_t phase_prepare(int dim) {
  static bool attr = false;
  if (dim != 3 || attr) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_phase3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Phase3::smem);
  int dev = 0, sms = 0, per = 0, perm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_phase3, Phase3::NT, Phase3::smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perm, k_phase3m<kMarchRows>, March3::NT, 0);
  if (e == cudaSuccess) {
    g_phase3_slots = sms * (per > 0 ? per : 1);
    g_march_slots = sms * (perm > 0 ? perm : 1);
    attr = true;
  }
  return e;
}

// z chunk of a k_phase3 launch: 16 planes (4 of them re-read as the march's prologue), halved
// while the grid of columns would not fill the device once.
int phase3_zc(int nx, int ny, int nz) {
  const long long cols = (long long)((nx + Phase3::TX - 1) / Phase3::TX) * ((ny + Phase3::TY - 1) / Phase3::TY);
  int zc = Phase3::ZC;
  while (zc > 4 && cols * ((nz + zc - 1) / zc) < g_phase3_slots) zc /= 2;
  return zc;
}

static cudaError_t launch_phase3(const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out, int *tiles,
                                 int *ntiles, int *lflag, cudaStream_t s) {
  const cudaError_t e = phase_prepare(3);
  if (e != cudaSuccess) return e;
  static const bool old_kernel = [] {
    const char *v = getenv("LBM_PHASE_KERNEL");
    return v && v[0] == 'o';
  }();
  if (old_kernel) {
    using G = Phase3;
    const int zc = phase3_zc(P.nx, P.ny, P.nz);
    dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, (P.nz + zc - 1) / zc);
    return launch_pdl(k_phase3, grid, dim3(32, G::TY), G::smem, s, P, phi, u, phi_out, tiles, ntiles, zc);
  }
  // one resident wave of warps sharing the (column, plane) units equally, at least MIN_RUN planes each
  constexpr int M = kMarchRows;
  const int ncx = (P.nx + March3::OUT - 1) / March3::OUT, ncy = (P.ny + M - 1) / M;
  const long long units = (long long)ncx * ncy * P.nz;
  const long long want = (units + March3::MIN_RUN - 1) / March3::MIN_RUN;
  long long blocks = (want + March3::WARPS - 1) / March3::WARPS;
  if (blocks > g_march_slots) blocks = g_march_slots;
  if (blocks < 1) blocks = 1;
  return launch_pdl(k_phase3m<M>, dim3((unsigned)blocks), dim3(March3::NT), 0, s, P, phi, u, phi_out, tiles, ntiles,
                    lflag, ncx, units);
}

cudaError_t launch_phase(int dim, const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out,
                         int *tiles, int *ntiles, int *lflag, cudaStream_t s) {
  return dim == 2 ? launch_phase_dim<2>(P, phi, u, phi_out, tiles, ntiles, s)
                  : launch_phase3(P, phi, u, phi_out, tiles, ntiles, lflag, s);
}

// Lists the tiles holding an interfacial cell of phi (used after the state is set from the host).
template <int DIM>
__global__ void __launch_bounds__(PhaseGeom<DIM>::NT)
k_gate_tiles(const KParams P, const int32_t *__restrict__ phi, int *__restrict__ tiles, int *__restrict__ ntiles) {
  using G = PhaseGeom<DIM>;
  const int x = blockIdx.x * G::TX + threadIdx.x, y = blockIdx.y * G::TY + threadIdx.y,
            z = blockIdx.z * G::TZ + threadIdx.z;
  bool gated = false;
  if (x < P.nx && y < P.ny && z < P.nz)
    gated = q_gate_value(phi[(long long)x + (long long)P.nx * (y + (long long)P.ny * z)]) >= P.q_th;
  const int any = __syncthreads_or(gated);
  if (any && threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0)
    tiles[atomicAdd(ntiles, 1)] = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

cudaError_t launch_gate_tiles(int dim, const KParams &P, const int32_t *phi, int *tiles, int *ntiles, cudaStream_t s) {
  if (dim == 2) {
    using G = PhaseGeom<2>;
    dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, 1);
    k_gate_tiles<2><<<grid, dim3(G::TX, G::TY, G::TZ), 0, s>>>(P, phi, tiles, ntiles);
  } else {
    using G = PhaseGeom<3>;
    dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, (P.nz + G::TZ - 1) / G::TZ);
    k_gate_tiles<3><<<grid, dim3(G::TX, G::TY, G::TZ), 0, s>>>(P, phi, tiles, ntiles);
  }
  return cudaGetLastError();
}

}  // namespace lbm
