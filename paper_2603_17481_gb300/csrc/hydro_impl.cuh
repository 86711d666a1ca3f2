// hydro_impl.cuh -- the hydrodynamic half of a time step (Sec. 2.1): pull streaming, macroscopic
// moments (Eqs. 6-7), mixture properties (Eqs. 8-10), the force split (Eqs. 18-21) and the
// recursive-regularized collision with Guo forcing (Eqs. 3, 11, 14, 16, 17).
//
// Layout: populations are structure-of-arrays, buf[i * N + n]. The buffer read at step t holds
// post-collision populations of step t-1 at their source cell, so the pre-collision population
// of direction i at cell x is src[i][x - c_i] (pull); the kernel writes dst[i][x] = f_post_i(x).
// One thread per cell, 32 consecutive x per warp (coalesced stores, loads offset by one cell).
// Each thread wraps its neighbour coordinates once per axis and forms the 9 (3D) or 3 (2D) row
// offsets of its neighbourhood, so a pull address is one add. phi of the tile + 1 halo is staged
// in shared memory row by row, converted once to FP32 (the interfacial gate of the cell itself is
// taken on the stored fixed-point value, as in the near-contact kernel).
//
// The collision is evaluated from moments rather than by summing over tensors: with the
// fourth-order isotropy of D2Q9/D3Q19/D3Q27, sum f_eq c c = p* cs^2 I + u u and sum S c c =
// u F' + F' u, hence A2 = M2 - p* cs^2 I - u u + (u F' + F' u) / 2 with M2 = sum f c c, and the
// per-direction Hermite contractions reduce to
//   H2 : T   = c.T.c - cs^2 tr T,
//   H3 : uuu = (c.u)^3 - 3 cs^2 |u|^2 (c.u),
//   H3 : A3  = 3 (c.u)(c.A2.c) - 3 cs^2 [ (c.u) tr A2 + 2 c.A2.u ]   (A3 of Eq. 16).
// With cs^2 = 1/3 the post-collision population f_eq + (1 - omega) Reg + S/2 is, per direction,
//   f_i / w_i = E(c) + O(c),  f_{-i} / w_i = E(c) - O(c),
//   E = C0 + 4.5 (c.u)^2 + 4.5 (1-omega) c.A2.c + 4.5 (c.u)(c.F'),
//   O = (c.u) C1 + 4.5 (c.u)^3 + 13.5 (1-omega)(c.u)(c.A2.c) - 9 (1-omega) c.A2.u + 1.5 c.F',
//   C0 = p* - 1.5 |u|^2 - 1.5 (1-omega) tr A2 - 1.5 u.F',  C1 = 3 - 4.5 |u|^2 - 4.5 (1-omega) tr A2,
// so each pair of opposite directions shares its even and odd parts.
#pragma once

#include <type_traits>

#include "launch.h"

// Resident blocks per SM (256 threads each) that the register allocation is sized for: 5 (48
// registers, no spills, 1.05x faster than 4 on D3Q19) except D3Q27, which spills below 56.
#ifndef LBM_HYDRO_MINB
#define LBM_HYDRO_MINB 5
#endif

namespace lbm {

// I32: every population and velocity element offset fits in an unsigned 32-bit integer (Q N <= 2^32,
// checked by the launcher), so a pull or store address is one 32-bit multiply-add and one widening
// add; otherwise the offsets are 64-bit.
template <class L, int S, int MODE, bool I32>
__global__ void __launch_bounds__(Tile<L::D>::X * Tile<L::D>::Y * Tile<L::D>::Z, L::Q >= 27 ? 4 : LBM_HYDRO_MINB)
k_hydro(const KParams P, const typename Store<S>::T *__restrict__ src, typename Store<S>::T *__restrict__ dst,
        const int32_t *__restrict__ phi, const float4 *__restrict__ frep, float *__restrict__ u_out,
        float *__restrict__ ps_out, int *__restrict__ reset) {
  pdl_enter();
  constexpr int DIM = L::D;
  using SL = typename StencilOf<DIM>::type;
  using TT = Tile<DIM>;
  static_assert(TT::X == 32, "one warp per x row");
  constexpr int HX = TT::X + 2, HY = TT::Y + 2, HZ = DIM == 3 ? TT::Z + 2 : 1;
  constexpr int NROWS = HY * HZ, NWARPS = TT::Y * TT::Z;
  __shared__ float s_phi[NROWS * HX];

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int x0 = blockIdx.x * TT::X, y0 = blockIdx.y * TT::Y, z0 = blockIdx.z * TT::Z;
  // the near-contact tile list of this phi has been consumed: clear its count for reuse
  if (reset && (blockIdx.x | blockIdx.y | blockIdx.z | tx | ty | tz) == 0) *reset = 0;

  // stage phi (tile + 1 halo): warp w loads rows w, w + NWARPS, ...
  {
    const int xl = wrapn(x0 - 1 + tx, nx);
    const int xr = wrapn(x0 + 31 + (tx & 1), nx);
    for (int r = ty + TT::Y * tz; r < NROWS; r += NWARPS) {
      const int ry = r % HY, rz = r / HY;
      const int Y = wrapn(y0 + ry - 1, ny);
      const int Z = DIM == 3 ? wrapn(z0 + rz - 1, nz) : 0;
      const int32_t *row = phi + (long long)nx * (Y + (long long)ny * Z);
      s_phi[r * HX + tx] = phi_of(row[xl]);
      if (tx < 2) s_phi[r * HX + 32 + tx] = phi_of(row[xr]);
    }
  }
  __syncthreads();

  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  if (x >= nx || y >= ny || z >= nz) return;
  const int N = (int)P.N;

  // wrapped neighbour coordinates and row offsets rb[cy+1][cz+1]
  int X[3], RB[3][3];
  X[0] = x == 0 ? nx - 1 : x - 1; X[1] = x; X[2] = x == nx - 1 ? 0 : x + 1;
  {
    const int Y[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    int Z[3] = {0, 0, 0};
    if (DIM == 3) { Z[0] = z == 0 ? nz - 1 : z - 1; Z[1] = z; Z[2] = z == nz - 1 ? 0 : z + 1; }
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) RB[a][b] = nx * (Y[a] + ny * Z[b]);
  }
  const int idx = x + RB[1][1];
  using Off = typename std::conditional<I32, unsigned, long long>::type;
  const Off NO = (Off)N;

  // pull: f_i(x) = src_i(x - c_i)
  float f[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    const int s = X[1 - L::c(i, 0)] + RB[1 - L::c(i, 1)][1 - L::c(i, 2)];
    f[i] = Store<S>::ld(src + ((Off)i * NO + (Off)s), L::w(i));
  }

  // isotropic gradient and Laplacian of phi (Eqs. 22-23)
  const int b = (DIM == 3 ? (tz + 1) * HX * HY : 0) + (ty + 1) * HX + tx + 1;
  const int32_t v = __ldg(phi + idx);
  const float ph = s_phi[b];
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, lap = 0.f;
#pragma unroll
  for (int i = 1; i < SL::Q; i++) {
    if (!positive<SL>(i)) continue;
    const int o = SL::c(i, 0) + HX * (SL::c(i, 1) + HY * SL::c(i, 2));
    const float vp = s_phi[b + o], vm = s_phi[b - o];
    const float d = SL::w(i) * (vp - vm);
    g0 += SL::c(i, 0) * d;
    g1 += SL::c(i, 1) * d;
    if (DIM == 3) g2 += SL::c(i, 2) * d;
    lap += SL::w(i) * ((vp - ph) + (vm - ph));
  }
  g0 *= 3.0f; g1 *= 3.0f; g2 *= 3.0f;  // 1 / cs^2
  lap *= 6.0f;                          // 2 / cs^2

  // mixture properties, Eqs. 8-10 (linear rho and mu)
  const float rho = P.rho_g + P.drho * ph;
  const float inv_rho = __frcp_rn(rho);
  const float gr0 = P.drho * g0, gr1 = P.drho * g1, gr2 = P.drho * g2;
  const float nu = (P.mu_g + P.dmu * ph) * inv_rho;
  const float omega = __frcp_rn(0.5f + 3.0f * nu);

  // capillary force, Eq. 19
  const float muphi = P.beta4 * ph * (ph - 1.0f) * (ph - 0.5f) - P.kap * lap;
  float F0 = muphi * g0, F1 = muphi * g1, F2 = muphi * g2;

  // near-contact force where the near-contact kernel wrote one (same gate)
  if (P.nci_on && q_gate_value(v) >= P.q_th) {
    const float4 fr = __ldg(frep + idx);
    F0 += fr.x; F1 += fr.y; F2 += fr.z;
  }

  // moments, Eqs. 6-7, pairwise: s = f_i + f_-i, d = f_i - f_-i
  float ps = f[0], j0 = 0.f, j1 = 0.f, j2 = 0.f;
  float m00 = 0.f, m11 = 0.f, m22 = 0.f, m01 = 0.f, m02 = 0.f, m12 = 0.f;
#pragma unroll
  for (int i = 1; i < L::Q; i++) {
    if (!(i > L::opp(i))) continue;
    const float sp = f[i] + f[L::opp(i)], dm = f[i] - f[L::opp(i)];
    ps += sp;
    const int c0 = L::c(i, 0), c1 = L::c(i, 1), c2 = L::c(i, 2);
    if (c0) { j0 += c0 * dm; m00 += sp; }
    if (c1) { j1 += c1 * dm; m11 += sp; }
    if (c2) { j2 += c2 * dm; m22 += sp; }
    if (c0 && c1) m01 += c0 * c1 * sp;
    if (c0 && c2) m02 += c0 * c2 * sp;
    if (c1 && c2) m12 += c1 * c2 * sp;
  }

  // pressure correction (Eq. 20) and buoyancy
  const float pc = -ps * kCs2;
  const float db = rho - P.rho_bar;
  F0 += pc * gr0 + db * P.g[0];
  F1 += pc * gr1 + db * P.g[1];
  F2 += pc * gr2 + db * P.g[2];

  // velocity without F_nu, then the viscous correction (Eq. 21) from Pi = M2 - p* cs^2 I - u0 u0
  const float h2r = 0.5f * inv_rho;
  const float a0 = j0 + F0 * h2r, a1 = j1 + F1 * h2r, a2 = DIM == 3 ? j2 + F2 * h2r : 0.f;
  const float pcs = ps * kCs2;
  const float P00 = m00 - pcs - a0 * a0, P11 = m11 - pcs - a1 * a1, P01 = m01 - a0 * a1;
  const float P22 = DIM == 3 ? m22 - pcs - a2 * a2 : 0.f;
  const float P02 = DIM == 3 ? m02 - a0 * a2 : 0.f, P12 = DIM == 3 ? m12 - a1 * a2 : 0.f;
  const float cnu = -3.0f * nu * omega;
  const float Fn0 = cnu * (P00 * gr0 + P01 * gr1 + P02 * gr2);
  const float Fn1 = cnu * (P01 * gr0 + P11 * gr1 + P12 * gr2);
  const float Fn2 = DIM == 3 ? cnu * (P02 * gr0 + P12 * gr1 + P22 * gr2) : 0.f;
  F0 += Fn0; F1 += Fn1; F2 += Fn2;
  const float u0 = a0 + Fn0 * h2r, u1 = a1 + Fn1 * h2r, u2 = DIM == 3 ? a2 + Fn2 * h2r : 0.f;

  if (MODE == kMoments) {
    u_out[idx] = u0;
    u_out[NO + (Off)idx] = u1;
    u_out[2 * NO + (Off)idx] = u2;
    ps_out[idx] = ps;
    return;
  }

  const float r0 = F0 * inv_rho, r1 = F1 * inv_rho, r2 = DIM == 3 ? F2 * inv_rho : 0.f;
  // second-order non-equilibrium moment A2 (the projection of f - f_eq + S/2)
  const float A00 = P00 + a0 * a0 - u0 * u0 + u0 * r0;
  const float A11 = P11 + a1 * a1 - u1 * u1 + u1 * r1;
  const float A22 = DIM == 3 ? P22 + a2 * a2 - u2 * u2 + u2 * r2 : 0.f;
  const float A01 = P01 + a0 * a1 - u0 * u1 + 0.5f * (u0 * r1 + u1 * r0);
  const float A02 = DIM == 3 ? P02 + a0 * a2 - u0 * u2 + 0.5f * (u0 * r2 + u2 * r0) : 0.f;
  const float A12 = DIM == 3 ? P12 + a1 * a2 - u1 * u2 + 0.5f * (u1 * r2 + u2 * r1) : 0.f;
  const float trA = A00 + A11 + A22;
  const float Au0 = A00 * u0 + A01 * u1 + A02 * u2;
  const float Au1 = A01 * u0 + A11 * u1 + A12 * u2;
  const float Au2 = A02 * u0 + A12 * u1 + A22 * u2;
  const float uu = u0 * u0 + u1 * u1 + u2 * u2;
  const float ur = u0 * r0 + u1 * r1 + u2 * r2;
  const float om1 = 1.0f - omega;
  const float C0 = ps - 1.5f * uu - 1.5f * om1 * trA - 1.5f * ur;
  const float C1 = 3.0f - 4.5f * uu - 4.5f * om1 * trA;
  const float k45 = 4.5f * om1, k135 = 13.5f * om1, k9 = 9.0f * om1;

  Store<S>::st_w(dst + idx, C0, L::w(0));
  // per pair of opposite directions: c.u, c.F', c.A2.c, c.A2.u; then the even and odd parts are
  // evaluated two pairs at a time with the packed FP32x2 operations of sm_100+
  constexpr int NPAIR = (L::Q - 1) / 2;
  float pcu[NPAIR], pcr[NPAIR], pcac[NPAIR], pcau[NPAIR];
  {
    int pp = 0;
#pragma unroll
    for (int i = 1; i < L::Q; i++) {
      if (!(i > L::opp(i))) continue;
      const int c0 = L::c(i, 0), c1 = L::c(i, 1), c2 = L::c(i, 2);
      pcu[pp] = c0 * u0 + c1 * u1 + c2 * u2;
      pcr[pp] = c0 * r0 + c1 * r1 + c2 * r2;
      pcac[pp] = c0 * c0 * A00 + c1 * c1 * A11 + c2 * c2 * A22 + 2.0f * (c0 * c1 * A01 + c0 * c2 * A02 + c1 * c2 * A12);
      pcau[pp] = c0 * Au0 + c1 * Au1 + c2 * Au2;
      pp++;
    }
  }
  const float2 vC0 = make_float2(C0, C0), vC1 = make_float2(C1, C1), v45 = make_float2(4.5f, 4.5f);
  const float2 vk45 = make_float2(k45, k45), vk135 = make_float2(k135, k135), vmk9 = make_float2(-k9, -k9);
  const float2 v15 = make_float2(1.5f, 1.5f), vm1 = make_float2(-1.0f, -1.0f);
#pragma unroll
  for (int p = 0; p < NPAIR; p += 2) {
    if (p + 1 < NPAIR) {
      const float2 cu = make_float2(pcu[p], pcu[p + 1]), cr = make_float2(pcr[p], pcr[p + 1]);
      const float2 cac = make_float2(pcac[p], pcac[p + 1]), cau = make_float2(pcau[p], pcau[p + 1]);
      float2 ev = __ffma2_rn(cu, __fmul2_rn(v45, __fadd2_rn(cu, cr)), vC0);
      ev = __ffma2_rn(vk45, cac, ev);
      float2 in = __ffma2_rn(v45, __fmul2_rn(cu, cu), vC1);
      in = __ffma2_rn(vk135, cac, in);
      float2 od = __ffma2_rn(vmk9, cau, __fmul2_rn(cu, in));
      od = __ffma2_rn(v15, cr, od);
      const float2 fpos = __fadd2_rn(ev, od), fneg = __ffma2_rn(vm1, od, ev);
      // the pair indices of p and p + 1
      int ia = 0, ib = 0;
      {
        int pp = 0;
#pragma unroll
        for (int i = 1; i < L::Q; i++) {
          if (!(i > L::opp(i))) continue;
          if (pp == p) ia = i;
          if (pp == p + 1) ib = i;
          pp++;
        }
      }
      Store<S>::st_w(dst + ((Off)ia * NO + (Off)idx), fpos.x, L::w(ia));
      Store<S>::st_w(dst + ((Off)L::opp(ia) * NO + (Off)idx), fneg.x, L::w(ia));
      Store<S>::st_w(dst + ((Off)ib * NO + (Off)idx), fpos.y, L::w(ib));
      Store<S>::st_w(dst + ((Off)L::opp(ib) * NO + (Off)idx), fneg.y, L::w(ib));
    } else {
      const float cu = pcu[p], cr = pcr[p], cAc = pcac[p], cAu = pcau[p];
      const float ev = C0 + cu * (4.5f * cu + 4.5f * cr) + k45 * cAc;
      const float od = cu * (C1 + 4.5f * cu * cu + k135 * cAc) - k9 * cAu + 1.5f * cr;
      int ia = 0;
      {
        int pp = 0;
#pragma unroll
        for (int i = 1; i < L::Q; i++) {
          if (!(i > L::opp(i))) continue;
          if (pp == p) ia = i;
          pp++;
        }
      }
      Store<S>::st_w(dst + ((Off)ia * NO + (Off)idx), ev + od, L::w(ia));
      Store<S>::st_w(dst + ((Off)L::opp(ia) * NO + (Off)idx), ev - od, L::w(ia));
    }
  }
  u_out[idx] = u0;
  u_out[NO + (Off)idx] = u1;
  if (DIM == 3) u_out[2 * NO + (Off)idx] = u2;
}

template <class L, int S>
cudaError_t launch_hydro_t(int mode, const KParams &P, const void *src, void *dst, const int32_t *phi,
                           const float4 *frep, float *u, float *pstar, int *reset, cudaStream_t s) {
  using TT = Tile<L::D>;
  using T = typename Store<S>::T;
  dim3 block(TT::X, TT::Y, TT::Z);
  dim3 grid((P.nx + TT::X - 1) / TT::X, (P.ny + TT::Y - 1) / TT::Y, (P.nz + TT::Z - 1) / TT::Z);
  const bool i32 = (long long)L::Q * P.N <= (1LL << 32);  // largest offset Q N - 1 fits an unsigned
  const T *a = (const T *)src;
  T *b = (T *)dst;
  if (mode == kStep)
    return i32 ? launch_pdl(k_hydro<L, S, kStep, true>, grid, block, 0, s, P, a, b, phi, frep, u, pstar, reset)
               : launch_pdl(k_hydro<L, S, kStep, false>, grid, block, 0, s, P, a, b, phi, frep, u, pstar, reset);
  return i32 ? launch_pdl(k_hydro<L, S, kMoments, true>, grid, block, 0, s, P, a, b, phi, frep, u, pstar, reset)
             : launch_pdl(k_hydro<L, S, kMoments, false>, grid, block, 0, s, P, a, b, phi, frep, u, pstar, reset);
}

template <class L>
cudaError_t launch_hydro_lattice(int store, int mode, const KParams &P, const void *src, void *dst,
                                 const int32_t *phi, const float4 *frep, float *u, float *pstar, int *reset,
                                 cudaStream_t s) {
  switch (store) {
    case 0: return launch_hydro_t<L, 0>(mode, P, src, dst, phi, frep, u, pstar, reset, s);
    case 1: return launch_hydro_t<L, 1>(mode, P, src, dst, phi, frep, u, pstar, reset, s);
    default: return launch_hydro_t<L, 2>(mode, P, src, dst, phi, frep, u, pstar, reset, s);
  }
}

}  // namespace lbm
