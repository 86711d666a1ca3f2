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

// hydro_cell's third mode: the post-collision state as a moment record (sink(q0, q1, q2, q3)).
constexpr int kEmitRecord = 2;

// The per-cell physics of a step after the pull and the phi stencils: mixture properties, the
// force split, the velocity, then (MODE kStep) the regularized collision, handing each
// post-collision population f_i / w_i to sink(i, value), or (kEmitRecord) its moment record.
// ph, g and lap are phi, its isotropic gradient and Laplacian at the cell; fr the near-contact
// force (zero where none was written).
template <class L, int MODE, class Sink>
__device__ __forceinline__ void hydro_cell(const KParams &P, const float (&f)[L::Q], const float ph, const float g0,
                                           const float g1, const float g2, const float lap, const float4 fr,
                                           float &uo0, float &uo1, float &uo2, float &pso, Sink &&sink) {
  constexpr int DIM = L::D;
  // mixture properties, Eqs. 8-10 (linear rho and mu)
  const float rho = P.rho_g + P.drho * ph;
  const float inv_rho = __frcp_rn(rho);
  const float gr0 = P.drho * g0, gr1 = P.drho * g1, gr2 = P.drho * g2;
  const float nu = (P.mu_g + P.dmu * ph) * inv_rho;
  const float omega = __frcp_rn(0.5f + 3.0f * nu);

  // capillary force, Eq. 19
  const float muphi = P.beta4 * ph * (ph - 1.0f) * (ph - 0.5f) - P.kap * lap;
  float F0 = muphi * g0, F1 = muphi * g1, F2 = muphi * g2;

  // near-contact force where the near-contact kernel wrote one (zero elsewhere)
  F0 += fr.x; F1 += fr.y; F2 += fr.z;

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

  uo0 = u0; uo1 = u1; uo2 = u2; pso = ps;
  if (MODE == kMoments) return;

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
  if constexpr (MODE == kEmitRecord) {
    // moment-record storage: the post-collision state itself (its populations are evaluated by
    // the cells that pull them)
    sink(make_float4(C0, C1, u0, u1), make_float4(u2, r0, r1, r2),
         make_float4(om1 * A00, om1 * A11, om1 * A22, om1 * A01), make_float4(om1 * A02, om1 * A12, 0.f, 0.f));
  } else {
  const float k45 = 4.5f * om1, k135 = 13.5f * om1, k9 = 9.0f * om1;

  sink(0, C0);
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
      sink(ia, fpos.x);
      sink(L::opp(ia), fneg.x);
      sink(ib, fpos.y);
      sink(L::opp(ib), fneg.y);
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
      sink(ia, ev + od);
      sink(L::opp(ia), ev - od);
    }
  }
  }
}


// Two cells' values packed in one register pair, with the FP32x2 operations of sm_100+: each
// operation below is one instruction for both cells (rounded per lane, as the scalar one).
struct V2 {
  float2 v;
};
__device__ __forceinline__ V2 V(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ V2 V(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)}; }
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ V2 rcp2(V2 a) { return {make_float2(__frcp_rn(a.v.x), __frcp_rn(a.v.y))}; }
// s + c x for a lattice component c in {-1, 0, +1} known after unrolling
__device__ __forceinline__ V2 addc(V2 s, int c, V2 x) { return c == 0 ? s : (c > 0 ? s + x : s - x); }
// c . (x0, x1, x2) for a nonzero lattice vector c
__device__ __forceinline__ V2 cdot(int c0, int c1, int c2, V2 x0, V2 x1, V2 x2) {
  V2 r;
  if (c0) {
    r = c0 > 0 ? x0 : V(-1.0f) * x0;
    r = addc(addc(r, c1, x1), c2, x2);
  } else if (c1) {
    r = c1 > 0 ? x1 : V(-1.0f) * x1;
    r = addc(r, c2, x2);
  } else {
    r = c2 > 0 ? x2 : V(-1.0f) * x2;
  }
  return r;
}

// hydro_cell for two cells at once (3D lattices): the same equations in the same order, every
// operation on the packed pair (cell a in .x, cell b in .y). sink(i, V2) receives f_post_i / w_i
// of both cells.
template <class L, int MODE, class Sink>
__device__ __forceinline__ void hydro_cell_pair(const KParams &P, const V2 (&f)[L::Q], const V2 ph, const V2 g0,
                                                const V2 g1, const V2 g2, const V2 lap, const V2 fr0, const V2 fr1,
                                                const V2 fr2, V2 &uo0, V2 &uo1, V2 &uo2, V2 &pso, Sink &&sink) {
  static_assert(L::D == 3, "3D lattices");
  // mixture properties, Eqs. 8-10 (linear rho and mu)
  const V2 rho = fma2(V(P.drho), ph, V(P.rho_g));
  const V2 inv_rho = rcp2(rho);
  const V2 gr0 = V(P.drho) * g0, gr1 = V(P.drho) * g1, gr2 = V(P.drho) * g2;
  const V2 nu = fma2(V(P.dmu), ph, V(P.mu_g)) * inv_rho;
  const V2 omega = rcp2(fma2(V(3.0f), nu, V(0.5f)));

  // capillary force, Eq. 19, and the near-contact force (zero where none was written)
  const V2 muphi = fma2(V(-P.kap), lap, V(P.beta4) * ph * (ph - V(1.0f)) * (ph - V(0.5f)));
  V2 F0 = fma2(muphi, g0, fr0), F1 = fma2(muphi, g1, fr1), F2 = fma2(muphi, g2, fr2);

  // moments, Eqs. 6-7, pairwise: s = f_i + f_-i, d = f_i - f_-i
  V2 ps = f[0], j0 = V(0.0f), j1 = V(0.0f), j2 = V(0.0f);
  V2 m00 = V(0.0f), m11 = V(0.0f), m22 = V(0.0f), m01 = V(0.0f), m02 = V(0.0f), m12 = V(0.0f);
#pragma unroll
  for (int i = 1; i < L::Q; i++) {
    if (!(i > L::opp(i))) continue;
    const V2 sp = f[i] + f[L::opp(i)], dm = f[i] - f[L::opp(i)];
    ps = ps + sp;
    const int c0 = L::c(i, 0), c1 = L::c(i, 1), c2 = L::c(i, 2);
    if (c0) { j0 = addc(j0, c0, dm); m00 = m00 + sp; }
    if (c1) { j1 = addc(j1, c1, dm); m11 = m11 + sp; }
    if (c2) { j2 = addc(j2, c2, dm); m22 = m22 + sp; }
    if (c0 && c1) m01 = addc(m01, c0 * c1, sp);
    if (c0 && c2) m02 = addc(m02, c0 * c2, sp);
    if (c1 && c2) m12 = addc(m12, c1 * c2, sp);
  }

  // pressure correction (Eq. 20) and buoyancy
  const V2 pc = V(-kCs2) * ps;
  const V2 db = rho - V(P.rho_bar);
  F0 = fma2(pc, gr0, fma2(db, V(P.g[0]), F0));
  F1 = fma2(pc, gr1, fma2(db, V(P.g[1]), F1));
  F2 = fma2(pc, gr2, fma2(db, V(P.g[2]), F2));

  // velocity without F_nu, then the viscous correction (Eq. 21) from Pi = M2 - p* cs^2 I - u0 u0
  const V2 h2r = V(0.5f) * inv_rho;
  const V2 a0 = fma2(F0, h2r, j0), a1 = fma2(F1, h2r, j1), a2 = fma2(F2, h2r, j2);
  const V2 na0 = V(-1.0f) * a0, na1 = V(-1.0f) * a1, na2 = V(-1.0f) * a2;
  const V2 pcs = V(kCs2) * ps;
  const V2 P00 = fma2(na0, a0, m00 - pcs), P11 = fma2(na1, a1, m11 - pcs), P22 = fma2(na2, a2, m22 - pcs);
  const V2 P01 = fma2(na0, a1, m01), P02 = fma2(na0, a2, m02), P12 = fma2(na1, a2, m12);
  const V2 cnu = V(-3.0f) * nu * omega;
  const V2 Fn0 = cnu * fma2(P00, gr0, fma2(P01, gr1, P02 * gr2));
  const V2 Fn1 = cnu * fma2(P01, gr0, fma2(P11, gr1, P12 * gr2));
  const V2 Fn2 = cnu * fma2(P02, gr0, fma2(P12, gr1, P22 * gr2));
  F0 = F0 + Fn0; F1 = F1 + Fn1; F2 = F2 + Fn2;
  const V2 u0 = fma2(Fn0, h2r, a0), u1 = fma2(Fn1, h2r, a1), u2 = fma2(Fn2, h2r, a2);

  uo0 = u0; uo1 = u1; uo2 = u2; pso = ps;
  if (MODE == kMoments) return;

  const V2 r0 = F0 * inv_rho, r1 = F1 * inv_rho, r2 = F2 * inv_rho;
  // second-order non-equilibrium moment A2 (the projection of f - f_eq + S/2):
  // A_ab = P_ab + a_a a_b - u_a u_b + (u_a r_b + u_b r_a) / 2
  const V2 nu0 = V(-1.0f) * u0, nu1 = V(-1.0f) * u1, nu2 = V(-1.0f) * u2;
  const V2 A00 = fma2(u0, r0, fma2(nu0, u0, fma2(a0, a0, P00)));
  const V2 A11 = fma2(u1, r1, fma2(nu1, u1, fma2(a1, a1, P11)));
  const V2 A22 = fma2(u2, r2, fma2(nu2, u2, fma2(a2, a2, P22)));
  const V2 A01 = fma2(V(0.5f), fma2(u0, r1, u1 * r0), fma2(nu0, u1, fma2(a0, a1, P01)));
  const V2 A02 = fma2(V(0.5f), fma2(u0, r2, u2 * r0), fma2(nu0, u2, fma2(a0, a2, P02)));
  const V2 A12 = fma2(V(0.5f), fma2(u1, r2, u2 * r1), fma2(nu1, u2, fma2(a1, a2, P12)));
  const V2 trA = A00 + A11 + A22;
  const V2 Au0 = fma2(A00, u0, fma2(A01, u1, A02 * u2));
  const V2 Au1 = fma2(A01, u0, fma2(A11, u1, A12 * u2));
  const V2 Au2 = fma2(A02, u0, fma2(A12, u1, A22 * u2));
  const V2 uu = fma2(u0, u0, fma2(u1, u1, u2 * u2));
  const V2 ur = fma2(u0, r0, fma2(u1, r1, u2 * r2));
  const V2 om1 = V(1.0f) - omega;
  const V2 om1tr = om1 * trA;
  const V2 C0 = fma2(V(-1.5f), ur, fma2(V(-1.5f), om1tr, fma2(V(-1.5f), uu, ps)));
  const V2 C1 = fma2(V(-4.5f), om1tr, fma2(V(-4.5f), uu, V(3.0f)));
  const V2 k45 = V(4.5f) * om1, k135 = V(13.5f) * om1, mk9 = V(-9.0f) * om1;
  const V2 A01x2 = V(2.0f) * A01, A02x2 = V(2.0f) * A02, A12x2 = V(2.0f) * A12;

  sink(0, C0);
  // per pair of opposite directions: c.u, c.F', c.A2.c, c.A2.u, then the even and odd parts
  //   E = C0 + 4.5 (c.u)(c.u + c.F') + 4.5 (1-omega) c.A2.c,
  //   O = (c.u)(C1 + 4.5 (c.u)^2 + 13.5 (1-omega) c.A2.c) - 9 (1-omega) c.A2.u + 1.5 c.F'
#pragma unroll
  for (int i = 1; i < L::Q; i++) {
    if (!(i > L::opp(i))) continue;
    const int c0 = L::c(i, 0), c1 = L::c(i, 1), c2 = L::c(i, 2);
    const V2 cu = cdot(c0, c1, c2, u0, u1, u2);
    const V2 cr = cdot(c0, c1, c2, r0, r1, r2);
    const V2 cau = cdot(c0, c1, c2, Au0, Au1, Au2);
    V2 cac;  // c.A2.c = sum_a c_a^2 A_aa + 2 sum_{a<b} c_a c_b A_ab
    {
      bool any = false;
      auto add = [&](bool on, V2 x) {
        if (!on) return;
        cac = any ? cac + x : x;
        any = true;
      };
      add(c0 != 0, A00); add(c1 != 0, A11); add(c2 != 0, A22);
      if (c0 && c1) cac = addc(cac, c0 * c1, A01x2);
      if (c0 && c2) cac = addc(cac, c0 * c2, A02x2);
      if (c1 && c2) cac = addc(cac, c1 * c2, A12x2);
    }
    const V2 ev = fma2(k45, cac, fma2(cu, V(4.5f) * (cu + cr), C0));
    const V2 in = fma2(k135, cac, fma2(V(4.5f), cu * cu, C1));
    const V2 od = fma2(V(1.5f), cr, fma2(mk9, cau, cu * in));
    sink(i, ev + od);
    sink(L::opp(i), ev - od);
  }
}

// I32: every population and velocity element offset fits in an unsigned 32-bit integer (Q N <= 2^32,
// checked by the launcher), so a pull or store address is one 32-bit multiply-add and one widening
// add; otherwise the offsets are 64-bit.
template <class L, int S, int MODE, bool I32>
__global__ void __launch_bounds__(Tile<L::D>::X * Tile<L::D>::Y * Tile<L::D>::Z,
                                  S == kStoreRecord ? 3 : (L::Q >= 27 ? 4 : LBM_HYDRO_MINB))
k_hydro(const KParams P, const typename Store<S>::T *__restrict__ src, typename Store<S>::T *__restrict__ dst,
        const int32_t *__restrict__ phi, const float4 *__restrict__ frep, float *__restrict__ u_out,
        float *__restrict__ ps_out) {
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

  // pull: f_i(x) = src_i(x - c_i), or evaluated from the moment record of x - c_i
  float f[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    const int s = X[1 - L::c(i, 0)] + RB[1 - L::c(i, 1)][1 - L::c(i, 2)];
    if constexpr (S == kStoreRecord) {
      const float4 *q = src + (Off)s;
      f[i] = L::w(i) * record_f_over_w<L>(i, __ldg(q), __ldg(q + NO), __ldg(q + 2 * NO), __ldg(q + 3 * NO));
    } else {
      f[i] = Store<S>::ld(src + ((Off)i * NO + (Off)s), L::w(i));
    }
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

  // near-contact force where the near-contact kernel wrote one (same gate)
  float4 fr = make_float4(0.f, 0.f, 0.f, 0.f);
  if (P.nci_on && q_gate_value(v) >= P.q_th) fr = __ldg(frep + idx);
  float u0, u1, u2, ps;
  if constexpr (S == kStoreRecord && MODE == kStep) {
    float4 *q = dst + (Off)idx;
    hydro_cell<L, kEmitRecord>(P, f, ph, g0, g1, g2, lap, fr, u0, u1, u2, ps, [&](float4 a, float4 b, float4 c, float4 d) {
      q[0] = a; q[NO] = b; q[2 * NO] = c; q[3 * NO] = d;
    });
  } else {
    hydro_cell<L, MODE>(P, f, ph, g0, g1, g2, lap, fr, u0, u1, u2, ps, [&](int i, float vw) {
      if constexpr (S != kStoreRecord) Store<S>::st_w(dst + ((Off)i * NO + (Off)idx), vw, L::w(i));
    });  // (with the record store only kMoments reaches here, which stores no population)
  }
  if (MODE == kMoments) {
    u_out[idx] = u0;
    u_out[NO + (Off)idx] = u1;
    u_out[2 * NO + (Off)idx] = u2;
    ps_out[idx] = ps;
    return;
  }
  u_out[idx] = u0;
  u_out[NO + (Off)idx] = u1;
  if (DIM == 3) u_out[2 * NO + (Off)idx] = u2;
}

// Paired storage access: two populations of x-adjacent cells (x even) as one 8-byte (FP32) or
// 4-byte (FP16 / BF16) load or store, converted to FP32 as f (loads take w_i, as Store::ld).
template <int S> struct Pair;
template <> struct Pair<0> {
  __device__ static __forceinline__ float2 ld(const float *p, float) { return __ldg(reinterpret_cast<const float2 *>(p)); }
  __device__ static __forceinline__ void st_w(float *p, float a, float b, float w) {
    *reinterpret_cast<float2 *>(p) = make_float2(w * a, w * b);
  }
};
template <> struct Pair<1> {
  __device__ static __forceinline__ float2 ld(const __half *p, float w) {
    const float2 v = __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
    return make_float2(v.x * w, v.y * w);
  }
  __device__ static __forceinline__ void st_w(__half *p, float a, float b, float) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
  }
};
template <> struct Pair<2> {
  __device__ static __forceinline__ float2 ld(const __nv_bfloat16 *p, float w) {
    const float2 v = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
    return make_float2(v.x * w, v.y * w);
  }
  __device__ static __forceinline__ void st_w(__nv_bfloat16 *p, float a, float b, float) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
  }
};

// The 3D hydrodynamic step with two x-adjacent cells per thread (nx even, Q N <= 2^32): a warp
// covers 64 cells of a row, the block 64 x 4 x 2. For each direction one paired load brings the
// populations of the source cells x - c_i, x + 1 - c_i when c_x = 0; when c_x = +-1 the pair is
// shifted by one cell, so one element comes from the neighbouring lane (warp shuffle) or, at the
// warp's edge, from a single load. Stores of the post-collision populations and of u are paired.
// phi of the block + 1 halo is staged in shared memory with the cell x - 1 of lane 0 at an even
// index, so the four columns x - 1 .. x + 2 of a stencil row are two 8-byte shared loads.
// Shared memory of one tile of the paired kernel (the tile is 64 x TY x TZ cells).
template <int TY, int TZ> struct Hydro2Smem {
  static constexpr int HX = 68, HY = TY + 2, HZ = TZ + 2;  // row pitch 68: column x0 - 1 + j at index j
  static constexpr int NROWS = HY * HZ, FLOATS = NROWS * HX;
};

// One tile (bx, by, bz) of 64 x TY x TZ cells with a block of 32 x TY x TZ threads. Every thread
// of the block calls it (one barrier inside; a caller looping over tiles adds one between tiles).
// halves: bit 0 updates the cells x0 .. x0 + 31 (lanes 0 - 15), bit 1 x0 + 32 .. x0 + 63; the
// lanes of a half that is not updated still pull (their neighbours' shifted pairs need them).
template <class L, int S, int MODE, int TY, int TZ>
__device__ __forceinline__ void hydro2_tile(const KParams &P, const typename Store<S>::T *__restrict__ src,
                                            typename Store<S>::T *__restrict__ dst, const int32_t *__restrict__ phi,
                                            const float4 *__restrict__ frep, float *__restrict__ u_out,
                                            float *__restrict__ ps_out, const int bx, const int by, const int bz,
                                            const unsigned halves = 3u) {
  __shared__ __align__(16) float s_phi[Hydro2Smem<TY, TZ>::FLOATS];
  static_assert(L::D == 3, "3D lattices");
  using SL = D3Q27;
  using SM = Hydro2Smem<TY, TZ>;
  constexpr int HX = SM::HX, HY = SM::HY;
  constexpr int NROWS = SM::NROWS, NWARPS = TY * TZ;

  const int lane = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int x0 = bx * 64, y0 = by * TY, z0 = bz * TZ;

  const int x = x0 + 2 * lane, y = y0 + ty, z = z0 + tz;
  const bool in = x < nx && y < ny && z < nz;  // nx even: x + 1 < nx too
  const int N = (int)P.N;
  // row offsets RB[cy + 1][cz + 1] of the neighbourhood and the wrapped columns at the warp's edges
  int RB[3][3];
  {
    const int Y[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    const int Z[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) RB[a][b] = nx * (wrapn(Y[a], ny) + ny * Z[b]);
  }
  const int xl = x == 0 ? nx - 1 : x - 1;                  // column of x - 1
  const int xr = x + 2 >= nx ? x + 2 - nx : x + 2;          // column of x + 2
  const bool edge_l = lane == 0, edge_r = lane == 31 || x + 2 >= nx;
  const int idx = x + RB[1][1];

  // pull: f_i(x) = src_i(x - c_i), f_i(x + 1) = src_i(x + 1 - c_i), and the fixed-point phi of both
  // cells (the interfacial gate of the near-contact force)
  V2 f[L::Q];
  int2 vg = make_int2(0, 0);
  auto pull = [&] {
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
      const int cx = L::c(i, 0);
      const unsigned row = (unsigned)i * (unsigned)N + (unsigned)RB[1 - L::c(i, 1)][1 - L::c(i, 2)];
      float2 v = make_float2(0.f, 0.f);
      if (in) v = Pair<S>::ld(src + row + x, L::w(i));
      if (cx == 0) {
        f[i].v = v;
      } else if (cx == 1) {  // sources x - 1, x
        const float left = __shfl_up_sync(0xffffffffu, v.y, 1);
        f[i] = V(edge_l ? (in ? Store<S>::ld(src + row + xl, L::w(i)) : 0.f) : left, v.x);
      } else {  // sources x + 1, x + 2
        const float right = __shfl_down_sync(0xffffffffu, v.x, 1);
        f[i] = V(v.y, edge_r ? (in ? Store<S>::ld(src + row + xr, L::w(i)) : 0.f) : right);
      }
    }
    if (in && P.nci_on) vg = *reinterpret_cast<const int2 *>(phi + idx);
  };
  // With 2-byte populations the loads are issued before the phi staging and its barrier, so the two
  // round trips overlap; with FP32 populations (38 values live across the barrier) after it.
  if constexpr (S != 0) pull();
  // stage phi: the pairs (x0 - 2 + 2 lane, x0 - 1 + 2 lane) of each row cover x0 - 2 .. x0 + 61;
  // lanes 0 and 1 add the pairs at x0 + 62 and x0 + 64 (nx even keeps every pair aligned)
  {
    const int xa = wrapn(x0 - 2 + 2 * lane, nx);
    const int xb = wrapn(x0 + 62 + 2 * lane, nx);
    for (int r = ty + TY * tz; r < NROWS; r += NWARPS) {
      const int ry = r % HY, rz = r / HY;
      const int Y = wrapn(y0 + ry - 1, ny);
      const int Z = wrapn(z0 + rz - 1, nz);
      const int32_t *row = phi + (long long)nx * (Y + (long long)ny * Z);
      const int2 a = *reinterpret_cast<const int2 *>(row + xa);
      float *sr = s_phi + r * HX;
      if (lane > 0) sr[2 * lane - 1] = phi_of(a.x);
      sr[2 * lane] = phi_of(a.y);
      if (lane < 2) {
        const int2 b = *reinterpret_cast<const int2 *>(row + xb);
        sr[63 + 2 * lane] = phi_of(b.x);
        sr[64 + 2 * lane] = phi_of(b.y);
      }
    }
  }
  __syncthreads();
  if constexpr (S == 0) pull();
  if (!in || !((halves >> (lane >> 4)) & 1u)) return;  // no barrier or shuffle follows

  // isotropic gradient and Laplacian of phi (Eqs. 22-23) at both cells: columns x - 1 .. x + 2 of
  // the nine stencil rows as two 8-byte shared loads each
  float ga0 = 0.f, ga1 = 0.f, ga2 = 0.f, la = 0.f, gb0 = 0.f, gb1 = 0.f, gb2 = 0.f, lb = 0.f;
  float pha, phb;
  {
    float c[3][3][4];
#pragma unroll
    for (int dz = 0; dz < 3; dz++)
#pragma unroll
      for (int dy = 0; dy < 3; dy++) {
        const float *sr = s_phi + ((tz + dz) * HY + ty + dy) * HX + 2 * lane;
        const float2 p0 = *reinterpret_cast<const float2 *>(sr);
        const float2 p1 = *reinterpret_cast<const float2 *>(sr + 2);
        c[dz][dy][0] = p0.x; c[dz][dy][1] = p0.y; c[dz][dy][2] = p1.x; c[dz][dy][3] = p1.y;
      }
    pha = c[1][1][1];
    phb = c[1][1][2];
    // every operation is an explicit rounded intrinsic, so that each translation unit that inlines
    // this tile (the single-case and the batched kernels) rounds identically; a gradient term is
    // one fused multiply-add with the constant c_a w_i
    auto acc = [](float g, int c, float w, float d) { return c == 0 ? g : __fmaf_rn((float)c * w, d, g); };
#pragma unroll
    for (int i = 1; i < SL::Q; i++) {
      if (!positive<SL>(i)) continue;
      const int cx = SL::c(i, 0), cy = SL::c(i, 1), cz = SL::c(i, 2);
      const float w = SL::w(i);
      // cell a at column 1, cell b at column 2
      const float vpa = c[1 + cz][1 + cy][1 + cx], vma = c[1 - cz][1 - cy][1 - cx];
      const float vpb = c[1 + cz][1 + cy][2 + cx], vmb = c[1 - cz][1 - cy][2 - cx];
      const float da = __fsub_rn(vpa, vma), db = __fsub_rn(vpb, vmb);
      ga0 = acc(ga0, cx, w, da); ga1 = acc(ga1, cy, w, da); ga2 = acc(ga2, cz, w, da);
      gb0 = acc(gb0, cx, w, db); gb1 = acc(gb1, cy, w, db); gb2 = acc(gb2, cz, w, db);
      la = __fmaf_rn(w, __fadd_rn(__fsub_rn(vpa, pha), __fsub_rn(vma, pha)), la);
      lb = __fmaf_rn(w, __fadd_rn(__fsub_rn(vpb, phb), __fsub_rn(vmb, phb)), lb);
    }
  }
  ga0 = __fmul_rn(ga0, 3.0f); ga1 = __fmul_rn(ga1, 3.0f); ga2 = __fmul_rn(ga2, 3.0f); la = __fmul_rn(la, 6.0f);
  gb0 = __fmul_rn(gb0, 3.0f); gb1 = __fmul_rn(gb1, 3.0f); gb2 = __fmul_rn(gb2, 3.0f); lb = __fmul_rn(lb, 6.0f);

  float4 fra = make_float4(0.f, 0.f, 0.f, 0.f), frb = fra;
  if (P.nci_on) {
    if (q_gate_value(vg.x) >= P.q_th) fra = __ldg(frep + idx);
    if (q_gate_value(vg.y) >= P.q_th) frb = __ldg(frep + idx + 1);
  }
  V2 uo0, uo1, uo2, pso;
  auto store = [&](int i, V2 vw) {
    if constexpr (MODE == kStep) Pair<S>::st_w(dst + (unsigned)i * (unsigned)N + idx, vw.v.x, vw.v.y, L::w(i));
  };
  hydro_cell_pair<L, MODE>(P, f, V(pha, phb), V(ga0, gb0), V(ga1, gb1), V(ga2, gb2), V(la, lb), V(fra.x, frb.x),
                           V(fra.y, frb.y), V(fra.z, frb.z), uo0, uo1, uo2, pso, store);
  *reinterpret_cast<float2 *>(u_out + idx) = uo0.v;
  *reinterpret_cast<float2 *>(u_out + (unsigned)N + idx) = uo1.v;
  *reinterpret_cast<float2 *>(u_out + 2u * (unsigned)N + idx) = uo2.v;
  if constexpr (MODE == kMoments) *reinterpret_cast<float2 *>(ps_out + idx) = pso.v;
}

// The near-contact tiles (32 x 8 x 4) holding the two halves of the paired tile (bx, by, bz) of
// 64 x 4 x 2 cells: tiles 2 bx and 2 bx + 1 of the row (by / 2, bz / 2); the second is -1 beyond
// the grid.
static_assert(NciTile<3>::X == 32 && NciTile<3>::Y == 8 && NciTile<3>::Z == 4,
              "a near-contact tile holds 2 x 2 paired tiles of 64 x 4 x 2 cells in y, z, and half of one in x");
__device__ __forceinline__ int2 nci_tiles_of_pair(const KParams &P, int bx, int by, int bz) {
  const int gtx = (P.nx + 31) >> 5, gty = (P.ny + 7) >> 3;
  const int t0 = 2 * bx + gtx * ((by >> 1) + gty * (bz >> 1));
  return make_int2(t0, 2 * bx + 1 < gtx ? t0 + 1 : -1);
}

// (c_y + 1) + 4 (c_z + 1) of directions 16 w .. 16 w + 15, four bits each
template <class L> constexpr unsigned long long row_codes(int w) {
  unsigned long long m = 0;
  for (int i = 16 * w; i < L::Q && i < 16 * w + 16; i++)
    m |= (unsigned long long)((L::c(i, 1) + 1) | ((L::c(i, 2) + 1) << 2)) << (4 * (i - 16 * w));
  return m;
}

// Asks L2 for the source rows of the populations that tile (bx, by, bz) of 64 x TY x TZ cells will
// pull: warp (ty, tz) takes its row, lane i direction i (the cells x0 .. x0 + 63 of the row of
// x - c_i; the one cell of a shifted pair outside them lies in a neighbouring tile's lines). A
// prefetch is a hint: it reads nothing into registers and cannot fault on these in-buffer rows.
template <class L, int S, int TY, int TZ>
__device__ __forceinline__ void hydro2_prefetch(const KParams &P, const typename Store<S>::T *src, int bx, int by,
                                                int bz) {
  using T = typename Store<S>::T;
  const int i = threadIdx.x;
  const int y = by * TY + threadIdx.y, z = bz * TZ + threadIdx.z, x0 = bx * 64;
  if (i >= L::Q || y >= P.ny || z >= P.nz) return;
  constexpr unsigned long long c0 = row_codes<L>(0), c1 = row_codes<L>(1);
  const int code = (int)((i < 16 ? c0 >> (4 * i) : c1 >> (4 * (i - 16))) & 15ull);
  const int Y = wrapn(y - ((code & 3) - 1), P.ny), Z = wrapn(z - ((code >> 2) - 1), P.nz);
  const T *row = src + ((unsigned)i * (unsigned)P.N + (unsigned)(P.nx * (Y + P.ny * Z) + x0));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(row));
  constexpr int PER_LINE = 128 / (int)sizeof(T);
  if (PER_LINE < 64 && x0 + PER_LINE < P.nx) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + PER_LINE));
}

// listed == nullptr: every cell. Otherwise the split step's first part: only the halves whose
// near-contact tile is not listed (a block with both halves listed returns at once). prefetch: the
// block asks L2 for its population rows before it waits for the previous kernel (D3Q19: 0.9 % off
// the FP32 step and 1.3 % off the FP16 one on 256 x 128 x 128; D3Q27 measured 2.3 % slower with it,
// and a prefetch of the tile one resident wave ahead 16 % slower).
template <class L, int S, int MODE>
__global__ void __launch_bounds__(256, L::Q >= 27 ? 2 : LBM_HYDRO2_MINB)
k_hydro2(const KParams P, const typename Store<S>::T *__restrict__ src, typename Store<S>::T *__restrict__ dst,
         const int32_t *__restrict__ phi, const float4 *__restrict__ frep, float *__restrict__ u_out,
         float *__restrict__ ps_out, const int *__restrict__ listed, const bool prefetch) {
  // the rows were written by an earlier step's hydrodynamic kernel, which has completed; a prefetch
  // only moves lines into L2, the coherence point of every SM
  if (prefetch) hydro2_prefetch<L, S, 4, 2>(P, src, blockIdx.x, blockIdx.y, blockIdx.z);
  pdl_enter();
  unsigned halves = 3u;
  if (listed) {
    const int2 t = nci_tiles_of_pair(P, blockIdx.x, blockIdx.y, blockIdx.z);
    halves = (listed[t.x] ? 0u : 1u) | (t.y >= 0 && listed[t.y] ? 0u : 2u);
    if (halves == 0u) return;  // block-uniform
  }
  hydro2_tile<L, S, MODE, 4, 2>(P, src, dst, phi, frep, u_out, ps_out, blockIdx.x, blockIdx.y, blockIdx.z, halves);
}

// The split step's second part: the cells of the listed near-contact tiles. Item i of 4 n covers
// the paired tile (tx / 2, 2 ty + (i & 1), 2 tz + (i >> 1 & 1)) of listed tile i / 4 = (tx, ty, tz);
// when both near-contact tiles of a pair are listed, the even one's items update both halves and
// the odd one's items are skipped, so every cell is written once.
template <class L, int S>
__global__ void __launch_bounds__(256, L::Q >= 27 ? 2 : LBM_HYDRO2_MINB)
k_hydro2_listed(const KParams P, const typename Store<S>::T *__restrict__ src, typename Store<S>::T *__restrict__ dst,
                const int32_t *__restrict__ phi, const float4 *__restrict__ frep, float *__restrict__ u_out,
                const int *__restrict__ tiles, const int *__restrict__ ntiles, const int *__restrict__ listed) {
  pdl_enter();
  const int n4 = 4 * *ntiles;
  const int gtx = (P.nx + 31) >> 5, gty = (P.ny + 7) >> 3;
  for (int it = blockIdx.x; it < n4; it += gridDim.x) {
    const int tile = tiles[it >> 2];
    const int tx = tile % gtx, tyz = tile / gtx;
    const int ty = tyz % gty, tz = tyz / gty;
    if ((tx & 1) && listed[tile - 1]) continue;  // block-uniform: the even tile's items cover it
    const int bx = tx >> 1, by = 2 * ty + (it & 1), bz = 2 * tz + ((it >> 1) & 1);
    if (4 * by >= P.ny || 2 * bz >= P.nz) continue;
    const unsigned halves = (tx & 1) ? 2u : (1u | (tx + 1 < gtx && listed[tile + 1] ? 2u : 0u));
    hydro2_tile<L, S, kStep, 4, 2>(P, src, dst, phi, frep, u_out, nullptr, bx, by, bz, halves);
    __syncthreads();  // the staged phi of this item is no longer read
  }
}

template <class L, int S>
cudaError_t launch_hydro_t(int mode, const KParams &P, const void *src, void *dst, const int32_t *phi,
                           const float4 *frep, float *u, float *pstar, cudaStream_t s) {
  using TT = Tile<L::D>;
  using T = typename Store<S>::T;
  dim3 block(TT::X, TT::Y, TT::Z);
  dim3 grid((P.nx + TT::X - 1) / TT::X, (P.ny + TT::Y - 1) / TT::Y, (P.nz + TT::Z - 1) / TT::Z);
  const bool i32 = (long long)L::Q * P.N <= (1LL << 32);  // largest offset Q N - 1 fits an unsigned
  const T *a = (const T *)src;
  T *b = (T *)dst;
  const int *all = nullptr;
  if constexpr (L::D == 3 && S != kStoreRecord) {
    if (i32 && P.nx % 2 == 0) {
      dim3 g2((P.nx + 63) / 64, (P.ny + 3) / 4, (P.nz + 1) / 2);
      constexpr bool pf = L::Q == 19;
      return mode == kStep
                 ? launch_pdl(k_hydro2<L, S, kStep>, g2, block, 0, s, P, a, b, phi, frep, u, pstar, all, pf)
                 : launch_pdl(k_hydro2<L, S, kMoments>, g2, block, 0, s, P, a, b, phi, frep, u, pstar, all, false);
    }
  }
  if (mode == kStep)
    return i32 ? launch_pdl(k_hydro<L, S, kStep, true>, grid, block, 0, s, P, a, b, phi, frep, u, pstar)
               : launch_pdl(k_hydro<L, S, kStep, false>, grid, block, 0, s, P, a, b, phi, frep, u, pstar);
  return i32 ? launch_pdl(k_hydro<L, S, kMoments, true>, grid, block, 0, s, P, a, b, phi, frep, u, pstar)
             : launch_pdl(k_hydro<L, S, kMoments, false>, grid, block, 0, s, P, a, b, phi, frep, u, pstar);
}

template <class L>
cudaError_t launch_hydro_lattice(int store, int mode, const KParams &P, const void *src, void *dst,
                                 const int32_t *phi, const float4 *frep, float *u, float *pstar, cudaStream_t s) {
  switch (store) {
    case 0: return launch_hydro_t<L, 0>(mode, P, src, dst, phi, frep, u, pstar, s);
    case 1: return launch_hydro_t<L, 1>(mode, P, src, dst, phi, frep, u, pstar, s);
    case 2: return launch_hydro_t<L, 2>(mode, P, src, dst, phi, frep, u, pstar, s);
    case kStoreRecord:
      if constexpr (L::D == 3) return launch_hydro_t<L, kStoreRecord>(mode, P, src, dst, phi, frep, u, pstar, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <class L, int S>
cudaError_t launch_split_t(int part, const KParams &P, const void *src, void *dst, const int32_t *phi,
                           const float4 *frep, float *u, const TileList &listed, int blocks, cudaStream_t s) {
  using T = typename Store<S>::T;
  const T *a = (const T *)src;
  T *b = (T *)dst;
  if (part == 0) {
    dim3 g2((P.nx + 63) / 64, (P.ny + 3) / 4, (P.nz + 1) / 2);
    return launch_pdl(k_hydro2<L, S, kStep>, g2, dim3(32, 4, 2), 0, s, P, a, b, phi, frep, u, (float *)nullptr,
                      (const int *)listed.mark, L::Q == 19);
  }
  return launch_pdl(k_hydro2_listed<L, S>, dim3(blocks > 0 ? blocks : 1), dim3(32, 4, 2), 0, s, P, a, b, phi, frep,
                    u, (const int *)listed.tiles, (const int *)listed.count, (const int *)listed.mark);
}

template <class L>
cudaError_t launch_split_lattice(int part, int store, const KParams &P, const void *src, void *dst,
                                 const int32_t *phi, const float4 *frep, float *u, const TileList &listed,
                                 int blocks, cudaStream_t s) {
  switch (store) {
    case 0: return launch_split_t<L, 0>(part, P, src, dst, phi, frep, u, listed, blocks, s);
    case 1: return launch_split_t<L, 1>(part, P, src, dst, phi, frep, u, listed, blocks, s);
    case 2: return launch_split_t<L, 2>(part, P, src, dst, phi, frep, u, listed, blocks, s);
    default: return cudaErrorInvalidValue;  // the paired kernel stores populations
  }
}

}  // namespace lbm
