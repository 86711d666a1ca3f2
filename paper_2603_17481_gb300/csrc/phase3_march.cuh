// phase3_march.cuh -- the 3D phase-field update (Sec. 2.1.1, Eq. 28) as a register march.
//
// The transfers are those of kernels_phase.cu (same face-flux form, same separable (1, 4, 1)
// smoothings of the D3Q27 weights, one rounding to 2^-30 per face), but organised so that a thread
// keeps everything it needs in registers:
//   - a warp owns 32 consecutive x columns and writes the middle 28 (lanes 2..29); every x
//     neighbour (x +- 1, x + 2) is a warp shuffle, and the two columns of halo on each side are
//     computed by the warp itself (12.5 % redundant lanes instead of shared-memory staging);
//   - a thread owns M consecutive rows in y (it also holds the halo rows y - 2 .. y + M + 1 of phi
//     and y - 1 .. y + M of the compressive vector a), so every y neighbour is a register;
//   - the warp marches along z over a contiguous run of planes, keeping the few planes of phi, of
//     a and of the transfers it still needs; every z neighbour is a register too.
// There is no shared memory and no block barrier. Warps take equal shares of the (column, plane)
// work units, so the grid is one resident wave. A face on the boundary between two warps' ranges is
// computed by both from identical inputs with the same operations, so its rounded transfer is the
// same on both sides and sum(phi) stays exact.
//
// With g = G / 72 the normal is n = G / (|G| + 72 eps_n) (the factor of the D3Q27 gradient folds
// into eps_n), and the face transfers are
//   x: u_f phi_up + (D / 36) s_y s_z (phi(x) - phi(x+1)) + (3 kappa / 216)(s_y s_z a_x (x) + s_y s_z a_x (x+1))
//   y: u_f phi_up + (D / 6) s_z (phi(y) - phi(y+1)) + (3 kappa / 216)(s_x s_z a_y (y) + s_x s_z a_y (y+1))
//   z: u_f phi_up + D (phi(z) - phi(z+1)) + (3 kappa / 216)(s_x s_y a_z (z) + s_x s_y a_z (z+1))
// and G = (s_y s_z d_x phi, s_x s_z d_y phi, s_x s_y d_z phi) with d the central difference, built
// from the one-sided differences phi(x) - phi(x+1) as d_x phi(x) = -(those at x and x - 1).
#pragma once

#include "launch.h"

namespace lbm {


__device__ __forceinline__ float sh_up(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }    // x - 1
__device__ __forceinline__ float sh_dn(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }  // x + 1
__device__ __forceinline__ int sh_up_i(int v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ int sh_dn_i(int v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ int sh_dn2_i(int v) { return __shfl_down_sync(0xffffffffu, v, 2); }
__device__ __forceinline__ float m141(float a, float b, float c) { return __fmaf_rn(4.0f, b, __fadd_rn(a, c)); }
__device__ __forceinline__ float i2f(int32_t v) { return __int2float_rn(v); }

// minmod of two exact fixed-point differences: the one of smaller magnitude when both have the
// same sign, else 0.
__device__ __forceinline__ int32_t mm_i(int32_t a, int32_t b) {
  const int32_t lo = min(a, b), hi = max(a, b);
  return lo > 0 ? lo : (hi < 0 ? hi : 0);
}
// Upwind MUSCL state at the face between p and p + e (Eqs. 30-34), in 2^-30 units, from the
// fixed-point phi at p - e, p, p + e, p + 2e: with (L, C, R) = (p - e, p, p + e) when u_f >= 0
// and (p + 2e, p + e, p) otherwise, C + minmod(C - L, R - C) / 2; the slopes are exact integers.
__device__ __forceinline__ float upw_i(float uf, int32_t vm, int32_t v0, int32_t v1, int32_t vp) {
  const bool pos = uf >= 0.0f;
  const int32_t L = pos ? vm : vp, C = pos ? v0 : v1, R = pos ? v1 : v0;
  return __fmaf_rn(0.5f, i2f(mm_i(C - L, R - C)), i2f(C));
}

// One warp's march over a run of planes. Phi is kept as fixed-point integers; every difference
// of phi (gradient, diffusion, MUSCL slopes) is taken exactly in integers before it is converted,
// so stencils keep their precision where phi is close to 1 (a float copy of phi near 1 resolves
// only 6e-8, which in the liquid interior, where |grad phi| is small but phi (1 - phi) is not,
// steers the normal of the compressive term). Quantities in 2^-30 units carry the suffix _q.
// Resident blocks per SM the registers are sized for.
#ifndef LBM_MARCH_MINB
#define LBM_MARCH_MINB 2
#endif

// One warp's march over the planes z0 .. z1 - 1 of the column col (x segment col % ncx, y rows
// (col / ncx) M ..) of one case.
template <int M>
__device__ __forceinline__ void march_run(const KParams &P, const int32_t *__restrict__ phi, const float *__restrict__ u,
                                          int32_t *__restrict__ phi_out, int *__restrict__ tiles,
                                          int *__restrict__ ntiles, int *__restrict__ lflag, const int ncx,
                                          const long long col, const int z0, const int z1) {
  constexpr int NR = M + 4;  // phi rows -2 .. M+1 (index r + 2)
  constexpr int NA = M + 2;  // rows -1 .. M (index r + 1)
  constexpr int NY = M + 3;  // y differences phi(r) - phi(r+1), r = -2 .. M (index r + 2)
  const int lane = threadIdx.x & 31;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int plane = nx * ny, N = (int)P.N;
  const float *__restrict__ ux = u;
  const float *__restrict__ uy = u + P.N;
  const float *__restrict__ uz = u + 2 * P.N;
  // transfer coefficients in 2^-30 units: D of the z link, D / 36 and D / 6 of the smoothed x and
  // y differences, 3 kappa / 216 on the smoothed compressive sums (a in real units)
  const float D = P.Dlap * (1.0f / 6.0f), Dx = D * (1.0f / 36.0f), Dy = D * (1.0f / 6.0f);
  const float k3s_q = P.kc * kCs2 * 3.0f * (1.0f / 216.0f) * kQ30;
  const float e72_q = 72.0f * P.eps_n * kQ30;
  const int gtx = (nx + 31) / 32, gty = (ny + 7) / 8;
  const int ix = (int)(col % ncx), iy = (int)(col / ncx);
  const int xs = ix * March3::OUT, ys = iy * M;
  const int x = wrapi(xs + lane - 2, nx);
  const bool xout = lane >= 2 && lane < 2 + March3::OUT && xs + lane - 2 < nx;
  int yo[NR];  // in-plane offsets of this thread's cells in rows -2 .. M+1
#pragma unroll
  for (int i = 0; i < NR; i++) yo[i] = wrapi(ys + i - 2, ny) * nx + x;
  // near-contact tiles (32 x 8 x 4) touched by the output columns: x tiles tx0 and tx1
  const int tx0 = xs / 32, tx1 = min(xs + March3::OUT - 1, nx - 1) / 32;
  unsigned tflag = 0;  // bit 0: tile tx0, bit 1: tile tx1, for the current group of 4 planes

  int32_t I0[NR], I1[NR], NX[NR], Im[M];  // phi of planes p-2, p-1, next (p), and p-3 rows 0..M-1
  float DX0[NR], DX1[NR];                 // phi(x) - phi(x+1) of planes p-2, p-1
  float DY0[NY], DY1[NY];                 // phi(y) - phi(y+1) of planes p-2, p-1
  float XYk[M], YZk[M + 1];               // s_y s_z (phi(x) - phi(x+1)), s_z (phi(y) - phi(y+1)), plane p-2
  float HX0[NA], HX1[NA], HY0[NA], HY1[NA];  // a_x, a_y of planes p-3, p-2
  float ASk[M], UZk[M];                   // s_x s_y a_z and u_z of plane p-2
  int TZk[M];                             // transfer of the z face below plane p-2
#pragma unroll
  for (int i = 0; i < NR; i++) { I0[i] = I1[i] = 0; DX0[i] = DX1[i] = 0.f; }
#pragma unroll
  for (int i = 0; i < NY; i++) DY0[i] = DY1[i] = 0.f;
#pragma unroll
  for (int i = 0; i < NA; i++) HX0[i] = HX1[i] = HY0[i] = HY1[i] = 0.f;
#pragma unroll
  for (int r = 0; r < M; r++) { Im[r] = 0; XYk[r] = 0.f; ASk[r] = 0.f; UZk[r] = 0.f; TZk[r] = 0; }
#pragma unroll
  for (int j = 0; j <= M; j++) YZk[j] = 0.f;

  // plane offsets of p, p - 1, p - 2 (stepped, no division in the loop); phi of the first plane
  int pz = wrapi(z0 - 2, nz) * plane;
  int pz1 = (pz == 0 ? N : pz) - plane, pz2 = (pz1 == 0 ? N : pz1) - plane;
#pragma unroll
  for (int i = 0; i < NR; i++) NX[i] = __ldg(phi + pz + yo[i]);

  for (int p = z0 - 2; p <= z1 + 1; p++) {
    int32_t I2[NR];
#pragma unroll
    for (int i = 0; i < NR; i++) I2[i] = NX[i];
    const int pzn = pz + plane == N ? 0 : pz + plane;
    if (p < z1 + 1) {  // phi of the next plane, in flight during this iteration
#pragma unroll
      for (int i = 0; i < NR; i++) NX[i] = __ldg(phi + pzn + yo[i]);
    }
    float uzn[M], uxk[M], uyk[NA];
    if (p >= z0) {
#pragma unroll
      for (int r = 0; r < M; r++) uzn[r] = __ldg(uz + pz1 + yo[r + 2]);
    }
    if (p >= z0 + 2) {
#pragma unroll
      for (int r = 0; r < M; r++) uxk[r] = __ldg(ux + pz2 + yo[r + 2]);
#pragma unroll
      for (int i = 0; i < NA; i++) uyk[i] = __ldg(uy + pz2 + yo[i + 1]);
    }
    // exact differences of the new plane
    float DXp[NR], DYp[NY];
#pragma unroll
    for (int i = 0; i < NR; i++) DXp[i] = i2f(I2[i] - sh_dn_i(I2[i]));
#pragma unroll
    for (int j = 0; j < NY; j++) DYp[j] = i2f(I2[j] - I2[j + 1]);

    float XYZ[NA], YZ[NY], ax[NA], ay[NA], ASn[M];
    if (p >= z0) {
      // a = phi (1 - phi) n at plane p - 1, rows -1..M; G = 72 grad(phi) in 2^-30 units
      float XZ[NR];
#pragma unroll
      for (int i = 0; i < NR; i++) XZ[i] = m141(DX0[i], DX1[i], DXp[i]);
#pragma unroll
      for (int i = 0; i < NA; i++) XYZ[i] = m141(XZ[i], XZ[i + 1], XZ[i + 2]);
#pragma unroll
      for (int j = 0; j < NY; j++) YZ[j] = m141(DY0[j], DY1[j], DYp[j]);
      float az[NA];
#pragma unroll
      for (int i = 0; i < NA; i++) {
        const float gx = -__fadd_rn(XYZ[i], sh_up(XYZ[i]));       // s_y s_z (phi(x+1) - phi(x-1))
        const float cy = -__fadd_rn(YZ[i], YZ[i + 1]);            // s_z (phi(y+1) - phi(y-1))
        const float gy = m141(sh_up(cy), cy, sh_dn(cy));
        const float sz = m141(i2f(I2[i] - I0[i]), i2f(I2[i + 1] - I0[i + 1]), i2f(I2[i + 2] - I0[i + 2]));
        const float gz = m141(sh_up(sz), sz, sh_dn(sz));
        const float ph = __fmul_rn(i2f(I1[i + 1]), kInvQ30);
        const float gg = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, __fmul_rn(gz, gz)));
        const float gn = gg > 0.0f ? __fmul_rn(gg, rsqrtf(gg)) : 0.0f;
        const float sc = __fdividef(__fmul_rn(ph, __fsub_rn(1.0f, ph)), __fadd_rn(gn, e72_q));
        ax[i] = __fmul_rn(gx, sc);
        ay[i] = __fmul_rn(gy, sc);
        az[i] = __fmul_rn(gz, sc);
      }
#pragma unroll
      for (int r = 0; r < M; r++) {
        const float sy = m141(az[r], az[r + 1], az[r + 2]);
        ASn[r] = m141(sh_up(sy), sy, sh_dn(sy));
      }
    }
    int TZn[M];
    if (p >= z0 + 1) {
      // z face between planes p-2 and p-1, rows 0..M-1
#pragma unroll
      for (int r = 0; r < M; r++) {
        const int32_t v0 = I0[r + 2], v1 = I1[r + 2];
        const float uf = __fmul_rn(0.5f, __fadd_rn(UZk[r], uzn[r]));
        const float up = upw_i(uf, Im[r], v0, v1, I2[r + 2]);
        TZn[r] = __float2int_rn(__fmaf_rn(D, i2f(v0 - v1), __fmaf_rn(k3s_q, __fadd_rn(ASk[r], ASn[r]), __fmul_rn(uf, up))));
      }
    }
    if (p >= z0 + 2) {
      // output plane k = p - 2: x and y faces, then the update
      const int k = p - 2;
      int TX[M], TY[M + 1];
#pragma unroll
      for (int r = 0; r < M; r++) {
        const float AX = m141(m141(HX0[r], HX1[r], ax[r]), m141(HX0[r + 1], HX1[r + 1], ax[r + 1]),
                              m141(HX0[r + 2], HX1[r + 2], ax[r + 2]));
        const int32_t v0 = I0[r + 2];
        const float uf = __fmul_rn(0.5f, __fadd_rn(uxk[r], sh_dn(uxk[r])));
        const float up = upw_i(uf, sh_up_i(v0), v0, sh_dn_i(v0), sh_dn2_i(v0));
        TX[r] = __float2int_rn(__fmaf_rn(Dx, XYk[r], __fmaf_rn(k3s_q, __fadd_rn(AX, sh_dn(AX)), __fmul_rn(uf, up))));
      }
      float AY[NA];
#pragma unroll
      for (int i = 0; i < NA; i++) {
        const float a = m141(HY0[i], HY1[i], ay[i]);
        AY[i] = m141(sh_up(a), a, sh_dn(a));
      }
#pragma unroll
      for (int j = 0; j < M + 1; j++) {  // face between rows j - 1 and j
        const float uf = __fmul_rn(0.5f, __fadd_rn(uyk[j], uyk[j + 1]));
        const float up = upw_i(uf, I0[j], I0[j + 1], I0[j + 2], I0[j + 3]);
        TY[j] = __float2int_rn(__fmaf_rn(Dy, YZk[j], __fmaf_rn(k3s_q, __fadd_rn(AY[j], AY[j + 1]), __fmul_rn(uf, up))));
      }
      bool g0 = false, g1 = false;
#pragma unroll
      for (int r = 0; r < M; r++) {
        const int acc = sh_up_i(TX[r]) - TX[r] + TY[r] - TY[r + 1] + TZk[r] - TZn[r];
        if (xout && ys + r < ny) {
          const int32_t vn = I0[r + 2] + acc;
          phi_out[pz2 + yo[r + 2]] = vn;
          if (tiles && q_gate_value(vn) >= P.q_th) {
            if ((xs + lane - 2) / 32 == tx0) g0 = true; else g1 = true;
          }
        }
      }
      if (tiles) {
        tflag |= (__any_sync(0xffffffffu, g0) ? 1u : 0u) | (__any_sync(0xffffffffu, g1) ? 2u : 0u);
        if ((k & 3) == 3 || k == z1 - 1) {
          if (lane < 2 && ((tflag >> lane) & 1u)) {
            const int tile = (lane ? tx1 : tx0) + gtx * ((ys >> 3) + gty * (k >> 2));
            if (atomicExch(lflag + tile, 1) == 0) tiles[atomicAdd(ntiles, 1)] = tile;
          }
          tflag = 0;
        }
      }
    }
    // advance the histories by one plane
    if (p >= z0 + 1) {
#pragma unroll
      for (int r = 0; r < M; r++) TZk[r] = TZn[r];
    }
    if (p >= z0) {
#pragma unroll
      for (int r = 0; r < M; r++) { ASk[r] = ASn[r]; UZk[r] = uzn[r]; XYk[r] = XYZ[r + 1]; }
#pragma unroll
      for (int j = 0; j <= M; j++) YZk[j] = YZ[j + 1];
#pragma unroll
      for (int i = 0; i < NA; i++) {
        HX0[i] = HX1[i]; HX1[i] = ax[i];
        HY0[i] = HY1[i]; HY1[i] = ay[i];
      }
    }
#pragma unroll
    for (int r = 0; r < M; r++) Im[r] = I0[r + 2];
#pragma unroll
    for (int i = 0; i < NR; i++) { I0[i] = I1[i]; I1[i] = I2[i]; DX0[i] = DX1[i]; DX1[i] = DXp[i]; }
#pragma unroll
    for (int j = 0; j < NY; j++) { DY0[j] = DY1[j]; DY1[j] = DYp[j]; }
    pz2 = pz1; pz1 = pz; pz = pzn;
  }
}

// Clears the marks of the near-contact list of phi, whose step is done (every thread of the grid
// takes a share of the list).
__device__ __forceinline__ void clear_marks(const TileList &prev, const long long rank, const long long threads) {
  if (!prev.mark) return;
  const int n = *prev.count;
  for (long long i = rank; i < n; i += threads) prev.mark[prev.tiles[i]] = 0;
}

// The grid's warps share the (column, plane) units of one case equally.
template <int M>
__global__ void __launch_bounds__(March3::NT, LBM_MARCH_MINB)
k_phase3m(const KParams P, const int32_t *__restrict__ phi, const float *__restrict__ u,
          int32_t *__restrict__ phi_out, const TileList next, const TileList prev, const int ncx,
          const long long units) {
  pdl_enter();
  clear_marks(prev, (long long)blockIdx.x * March3::NT + threadIdx.x, (long long)gridDim.x * March3::NT);
  const long long nwarps = (long long)gridDim.x * March3::WARPS;
  const long long wid = (long long)blockIdx.x * March3::WARPS + (threadIdx.x >> 5);
  long long ub = units * wid / nwarps;
  const long long ue = units * (wid + 1) / nwarps;
  const int nz = P.nz;
  while (ub < ue) {
    const long long col = ub / nz;
    const int z0 = (int)(ub - col * nz);
    const int z1 = (int)min((long long)nz, (long long)z0 + (ue - ub));
    ub += z1 - z0;
    march_run<M>(P, phi, u, phi_out, next.tiles, next.count, next.mark, ncx, col, z0, z1);
  }
}

}  // namespace lbm
