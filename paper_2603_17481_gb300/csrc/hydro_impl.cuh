// hydro_impl.cuh -- the hydrodynamic half of a time step (Sec. 2.1): pull streaming, macroscopic
// moments (Eqs. 6-7), mixture properties (Eqs. 8-10), the force split (Eqs. 18-21) and the
// recursive-regularized collision with Guo forcing (Eqs. 3, 11, 14, 16, 17).
//
// Layout: populations are structure-of-arrays, buf[i * N + n]. The buffer read at step t holds
// post-collision populations of step t-1 at their source cell, so the pre-collision population
// of direction i at cell x is src[i][x - c_i] (pull); the kernel writes dst[i][x] = f_post_i(x).
// One thread per cell; phi of the tile + 1 halo is staged in shared memory as fixed-point
// integers so that every stencil difference is exact before conversion to FP32.
//
// The collision is evaluated from moments rather than by summing over tensors: with the
// fourth-order isotropy of D2Q9/D3Q19/D3Q27, sum f_eq c c = p* cs^2 I + u u and sum S c c =
// u F' + F' u, hence A2 = M2 - p* cs^2 I - u u + (u F' + F' u) / 2 with M2 = sum f c c, and the
// per-direction Hermite contractions reduce to
//   H2 : T   = c.T.c - cs^2 tr T,
//   H3 : uuu = (c.u)^3 - 3 cs^2 |u|^2 (c.u),
//   H3 : A3  = 3 (c.u)(c.A2.c) - 3 cs^2 [ (c.u) tr A2 + 2 c.A2.u ]   (A3 of Eq. 16).
#pragma once

#include "launch.h"

namespace lbm {

template <class L, int S, int MODE>
__global__ void __launch_bounds__(Tile<L::D>::X * Tile<L::D>::Y * Tile<L::D>::Z)
k_hydro(const KParams P, const typename Store<S>::T *__restrict__ src, typename Store<S>::T *__restrict__ dst,
        const int32_t *__restrict__ phi, const float4 *__restrict__ frep, float *__restrict__ u_out,
        float *__restrict__ ps_out) {
  constexpr int DIM = L::D;
  using SL = typename StencilOf<DIM>::type;
  using TT = Tile<DIM>;
  constexpr int HX = TT::X + 2, HY = TT::Y + 2, HZ = DIM == 3 ? TT::Z + 2 : 1;
  constexpr int NB = HX * HY * HZ, NT = TT::X * TT::Y * TT::Z;
  __shared__ int32_t s_phi[NB];

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + TT::X * (ty + TT::Y * tz);
  const int x0 = blockIdx.x * TT::X, y0 = blockIdx.y * TT::Y, z0 = blockIdx.z * TT::Z;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  for (int t = tid; t < NB; t += NT) {
    int bx = t % HX, by = (t / HX) % HY, bz = t / (HX * HY);
    int X = wrapi(x0 + bx - 1, nx), Y = wrapi(y0 + by - 1, ny), Z = DIM == 3 ? wrapi(z0 + bz - 1, nz) : 0;
    s_phi[t] = phi[(long long)X + (long long)nx * (Y + (long long)ny * Z)];
  }
  __syncthreads();

  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  if (x >= nx || y >= ny || z >= nz) return;
  const long long N = P.N;
  const long long idx = (long long)x + (long long)nx * (y + (long long)ny * z);

  // pull: f_i(x) = src_i(x - c_i), periodic
  float f[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    int sx = x - L::c(i, 0), sy = y - L::c(i, 1), sz = z - L::c(i, 2);
    sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
    sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
    if (DIM == 3) sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
    const long long sidx = (long long)sx + (long long)nx * (sy + (long long)ny * sz);
    f[i] = Store<S>::ld(src + (long long)i * N + sidx, L::w(i));
  }

  // isotropic gradient and Laplacian of phi (Eqs. 22-23) on exact fixed-point differences
  const int b = (DIM == 3 ? (tz + 1) * HX * HY : 0) + (ty + 1) * HX + tx + 1;
  const int32_t v = s_phi[b];
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, lap = 0.f;
#pragma unroll
  for (int i = 1; i < SL::Q; i++) {
    if (!positive<SL>(i)) continue;
    const int o = SL::c(i, 0) + HX * (SL::c(i, 1) + HY * SL::c(i, 2));
    const int32_t vp = s_phi[b + o], vm = s_phi[b - o];
    const float d = SL::w(i) * dphi_of(vp, vm);
    g0 += SL::c(i, 0) * d;
    g1 += SL::c(i, 1) * d;
    if (DIM == 3) g2 += SL::c(i, 2) * d;
    lap += SL::w(i) * (dphi_of(vp, v) + dphi_of(vm, v));
  }
  g0 *= 3.0f; g1 *= 3.0f; g2 *= 3.0f;  // 1 / cs^2
  lap *= 6.0f;                          // 2 / cs^2
  const float ph = phi_of(v);

  // mixture properties, Eqs. 8-10 (linear rho and mu)
  const float rho = P.rho_g + P.drho * ph;
  const float inv_rho = 1.0f / rho;
  const float gr0 = P.drho * g0, gr1 = P.drho * g1, gr2 = P.drho * g2;
  const float nu = (P.mu_g + P.dmu * ph) * inv_rho;
  const float omega = 1.0f / (0.5f + 3.0f * nu);

  // capillary force, Eq. 19
  const float muphi = P.beta4 * ph * (ph - 1.0f) * (ph - 0.5f) - P.kap * lap;
  float F0 = muphi * g0, F1 = muphi * g1, F2 = muphi * g2;

  // near-contact force where the near-contact kernel wrote one (same gate)
  if (P.nci_on && q_gate_value(v) >= P.q_th) {
    const float4 fr = __ldg(frep + idx);
    F0 += fr.x; F1 += fr.y; F2 += fr.z;
  }

  // moments, Eqs. 6-7
  float ps = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
  float m00 = 0.f, m11 = 0.f, m22 = 0.f, m01 = 0.f, m02 = 0.f, m12 = 0.f;
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    const float fi = f[i];
    ps += fi;
    const int c0 = L::c(i, 0), c1 = L::c(i, 1), c2 = L::c(i, 2);
    if (c0) { j0 += c0 * fi; m00 += fi; }
    if (c1) { j1 += c1 * fi; m11 += fi; }
    if (c2) { j2 += c2 * fi; m22 += fi; }
    if (c0 && c1) m01 += c0 * c1 * fi;
    if (c0 && c2) m02 += c0 * c2 * fi;
    if (c1 && c2) m12 += c1 * c2 * fi;
  }

  // pressure correction (Eq. 20) and buoyancy
  const float pc = -ps * kCs2;
  F0 += pc * gr0 + (rho - P.rho_bar) * P.g[0];
  F1 += pc * gr1 + (rho - P.rho_bar) * P.g[1];
  F2 += pc * gr2 + (rho - P.rho_bar) * P.g[2];

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
    u_out[N + idx] = u1;
    u_out[2 * N + idx] = u2;
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

#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    const int c0 = L::c(i, 0), c1 = L::c(i, 1), c2 = L::c(i, 2);
    const float cu = c0 * u0 + c1 * u1 + c2 * u2;
    const float cr = c0 * r0 + c1 * r1 + c2 * r2;
    const float cAc = c0 * c0 * A00 + c1 * c1 * A11 + c2 * c2 * A22 +
                      2.0f * (c0 * c1 * A01 + c0 * c2 * A02 + c1 * c2 * A12);
    const float cAu = c0 * Au0 + c1 * Au1 + c2 * Au2;
    // Eq. 11 (1/(2 cs^4) = 1/(6 cs^6) = 4.5; 3 cs^2 = 1)
    const float feq = ps + 3.0f * cu + 4.5f * (cu * cu - kCs2 * uu) + 4.5f * (cu * cu * cu - uu * cu);
    // Eq. 14 with A3 of Eq. 16
    const float reg = 4.5f * (cAc - kCs2 * trA) + 4.5f * (3.0f * cu * cAc - cu * trA - 2.0f * cAu);
    // Eq. 17 (1/cs^2 = 3, 1/cs^4 = 9)
    const float src_i = 3.0f * (cr - ur) + 9.0f * cu * cr;
    const float fpost = L::w(i) * (feq + om1 * reg + 0.5f * src_i);
    Store<S>::st(dst + (long long)i * N + idx, fpost, L::w(i));
  }
  u_out[idx] = u0;
  u_out[N + idx] = u1;
  if (DIM == 3) u_out[2 * N + idx] = u2;
}

template <class L, int S>
cudaError_t launch_hydro_t(int mode, const KParams &P, const void *src, void *dst, const int32_t *phi,
                           const float4 *frep, float *u, float *pstar, cudaStream_t s) {
  using TT = Tile<L::D>;
  using T = typename Store<S>::T;
  dim3 block(TT::X, TT::Y, TT::Z);
  dim3 grid((P.nx + TT::X - 1) / TT::X, (P.ny + TT::Y - 1) / TT::Y, (P.nz + TT::Z - 1) / TT::Z);
  if (mode == kStep)
    k_hydro<L, S, kStep><<<grid, block, 0, s>>>(P, (const T *)src, (T *)dst, phi, frep, u, pstar);
  else
    k_hydro<L, S, kMoments><<<grid, block, 0, s>>>(P, (const T *)src, (T *)dst, phi, frep, u, pstar);
  return cudaGetLastError();
}

template <class L>
cudaError_t launch_hydro_lattice(int store, int mode, const KParams &P, const void *src, void *dst,
                                 const int32_t *phi, const float4 *frep, float *u, float *pstar, cudaStream_t s) {
  switch (store) {
    case 0: return launch_hydro_t<L, 0>(mode, P, src, dst, phi, frep, u, pstar, s);
    case 1: return launch_hydro_t<L, 1>(mode, P, src, dst, phi, frep, u, pstar, s);
    default: return launch_hydro_t<L, 2>(mode, P, src, dst, phi, frep, u, pstar, s);
  }
}

}  // namespace lbm
