// kernels_phase.cu -- the phase-field half of a time step (Sec. 2.1.1): Eq. 28,
//   phi^{n+1} = phi^n - div_h(u phi) + D lap_h(phi) + S_comp,
// with MUSCL-minmod face fluxes (Eqs. 29-34), the isotropic Laplacian (Eq. 23) and the
// isotropic compressive divergence S_comp = -(kappa / cs^2) sum_i w_i c_i . a(x + c_i),
// a = phi (1 - phi) n, kappa = 4 D / eps (Eqs. 26, 35).
//
// Every term is regrouped as a transfer across the links of the D2Q9 / D3Q27 stencil: since
// sum_i w_i c_i = 0 and sum_{i != 0} w_i = 1 - w_0,
//   D lap_h(phi)(x) = sum_{i != 0} D (2/cs^2) w_i (phi(x + c_i) - phi(x)),
//   S_comp(x)       = sum_{i != 0} -(kappa/cs^2) w_i c_i . (a(x) + a(x + c_i)),
// and the MUSCL flux difference is the difference of the two axis-face fluxes. The transfer of
// each link y -> y + c is computed by one function of the link's own data, rounded once to the
// 2^-30 phi grid and applied with opposite signs at its two ends, so sum(phi) is conserved
// exactly. Both cells of a link evaluate the same rounded value because the function uses
// explicitly rounded operations (no contraction) on identical inputs.
#include "launch.h"

namespace lbm {

template <int DIM> struct PhaseGeom {
  static constexpr int TX = PhaseTile<DIM>::X, TY = PhaseTile<DIM>::Y, TZ = PhaseTile<DIM>::Z;
  static constexpr int HX = TX + 4, HY = TY + 4, HZ = DIM == 3 ? TZ + 4 : 1;  // phi, halo 2
  static constexpr int AX = TX + 2, AY = TY + 2, AZ = DIM == 3 ? TZ + 2 : 1;  // a, halo 1
  static constexpr int NB = HX * HY * HZ, NA = AX * AY * AZ, NT = TX * TY * TZ;
};

__device__ __forceinline__ int32_t minmod_i(int32_t a, int32_t b) {
  if ((a > 0 && b > 0)) return a < b ? a : b;
  if ((a < 0 && b < 0)) return a > b ? a : b;
  return 0;
}

template <int DIM>
__global__ void __launch_bounds__(PhaseGeom<DIM>::NT)
k_phase(const KParams P, const int32_t *__restrict__ phi, const float *__restrict__ u,
        int32_t *__restrict__ phi_out) {
  using G = PhaseGeom<DIM>;
  using SL = typename StencilOf<DIM>::type;
  __shared__ int32_t s_phi[G::NB];
  __shared__ float s_a[3][G::NA];

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + G::TX * (ty + G::TY * tz);
  const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * G::TY, z0 = blockIdx.z * G::TZ;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  for (int t = tid; t < G::NB; t += G::NT) {
    int bx = t % G::HX, by = (t / G::HX) % G::HY, bz = t / (G::HX * G::HY);
    int X = wrapi(x0 + bx - 2, nx), Y = wrapi(y0 + by - 2, ny), Z = DIM == 3 ? wrapi(z0 + bz - 2, nz) : 0;
    s_phi[t] = phi[(long long)X + (long long)nx * (Y + (long long)ny * Z)];
  }
  __syncthreads();

  // compressive vector a = phi (1 - phi) grad(phi) / (|grad(phi)| + eps_n) on the tile + 1 halo
  for (int t = tid; t < G::NA; t += G::NT) {
    int ax = t % G::AX, ay = (t / G::AX) % G::AY, az = t / (G::AX * G::AY);
    int b = (DIM == 3 ? (az + 1) * G::HX * G::HY : 0) + (ay + 1) * G::HX + ax + 1;
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
    s_a[0][t] = g0 * s;
    s_a[1][t] = g1 * s;
    s_a[2][t] = g2 * s;
  }
  __syncthreads();

  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  if (x >= nx || y >= ny || z >= nz) return;
  const long long N = P.N;
  const int b = (DIM == 3 ? (tz + 2) * G::HX * G::HY : 0) + (ty + 2) * G::HX + tx + 2;
  const int ab = (DIM == 3 ? (tz + 1) * G::AX * G::AY : 0) + (ty + 1) * G::AX + tx + 1;
  const int xyz[3] = {x, y, z};
  const int nn[3] = {nx, ny, nz};

  int32_t acc = 0;
#pragma unroll
  for (int i = 1; i < SL::Q; i++) {
    if (!positive<SL>(i)) continue;
    const int c0 = SL::c(i, 0), c1 = SL::c(i, 1), c2 = SL::c(i, 2);
    const int o = c0 + G::HX * (c1 + G::HY * c2);
    const int oa = c0 + G::AX * (c1 + G::AY * c2);
    const float wl = SL::w(i);
    const int axis = (c0 != 0) + (c1 != 0) + (c2 != 0) == 1 ? (c0 ? 0 : (c1 ? 1 : 2)) : -1;
    // side 0: link x -> x + c (outgoing); side 1: link x - c -> x (incoming)
#pragma unroll
    for (int side = 0; side < 2; side++) {
      const int yb = b - side * o, ya = ab - side * oa;   // tail of the link
      const int32_t vy = s_phi[yb], vz = s_phi[yb + o];
      // Laplacian transfer D (2/cs^2) w (phi_y - phi_z)
      float tau = __fmul_rn(__fmul_rn(P.Dlap, wl), dphi_of(vy, vz));
      // compressive transfer (kappa/cs^2) w c . (a_y + a_z)
      float cd = 0.f;
      if (c0) cd = __fadd_rn(cd, c0 * __fadd_rn(s_a[0][ya], s_a[0][ya + oa]));
      if (c1) cd = __fadd_rn(cd, c1 * __fadd_rn(s_a[1][ya], s_a[1][ya + oa]));
      if (c2) cd = __fadd_rn(cd, c2 * __fadd_rn(s_a[2][ya], s_a[2][ya + oa]));
      tau = __fadd_rn(tau, __fmul_rn(__fmul_rn(P.kc, wl), cd));
      if (axis >= 0) {
        // MUSCL face flux u_f phi_up (Eqs. 30-34), face between y and z = y + e_axis
        const int32_t vym = s_phi[yb - o], vzp = s_phi[yb + 2 * o];
        const int32_t sy = minmod_i(vy - vym, vz - vy);
        const int32_t sz = minmod_i(vz - vy, vzp - vz);
        int p[3] = {xyz[0], xyz[1], xyz[2]};
        int pz[3] = {xyz[0], xyz[1], xyz[2]};
        if (side == 1) p[axis] = p[axis] == 0 ? nn[axis] - 1 : p[axis] - 1;
        else pz[axis] = pz[axis] == nn[axis] - 1 ? 0 : pz[axis] + 1;
        const long long iy = (long long)p[0] + (long long)nx * (p[1] + (long long)ny * p[2]);
        const long long iz = (long long)pz[0] + (long long)nx * (pz[1] + (long long)ny * pz[2]);
        const float uy = __ldg(u + axis * N + (side == 1 ? iy : (long long)x + (long long)nx * (y + (long long)ny * z)));
        const float uz = __ldg(u + axis * N + (side == 1 ? (long long)x + (long long)nx * (y + (long long)ny * z) : iz));
        const float uf = __fmul_rn(0.5f, __fadd_rn(uy, uz));
        // reconstructed states, exact in 64-bit fixed point with one extra fractional bit
        const long long up2 = uf >= 0.0f ? 2LL * vy + sy : 2LL * vz - sz;
        const float pup = __ll2float_rn(up2) * (0.5f * kInvQ30);
        tau = __fadd_rn(tau, __fmul_rn(uf, pup));
      }
      const int32_t r = __float2int_rn(__fmul_rn(tau, kQ30));
      acc += side == 0 ? -r : r;
    }
  }
  phi_out[(long long)x + (long long)nx * (y + (long long)ny * z)] = s_phi[b] + acc;
}

template <int DIM>
static cudaError_t launch_phase_dim(const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out,
                                    cudaStream_t s) {
  using G = PhaseGeom<DIM>;
  dim3 block(G::TX, G::TY, G::TZ);
  dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, (P.nz + G::TZ - 1) / G::TZ);
  k_phase<DIM><<<grid, block, 0, s>>>(P, phi, u, phi_out);
  return cudaGetLastError();
}

cudaError_t launch_phase(int dim, const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out,
                         cudaStream_t s) {
  return dim == 2 ? launch_phase_dim<2>(P, phi, u, phi_out, s) : launch_phase_dim<3>(P, phi, u, phi_out, s);
}

}  // namespace lbm
