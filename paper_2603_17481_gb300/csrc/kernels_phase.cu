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
// This file holds the 2D kernel (one block per tile, shared-memory face transfers) and the
// launchers; the 3D update is the register march of phase3_march.cuh.
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

template <int DIM>
static cudaError_t launch_phase_dim(const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out,
                                    int *tiles, int *ntiles, cudaStream_t s) {
  using G = PhaseGeom<DIM>;
  dim3 block(G::TX, G::TY, G::TZ);
  dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, (P.nz + G::TZ - 1) / G::TZ);
  return launch_pdl(k_phase<DIM>, grid, block, 0, s, P, phi, u, phi_out, tiles, ntiles);
}

// Records once, at context creation, how many k_phase3m blocks the device holds at once (SMs x
// resident blocks), so that the launches make no non-stream CUDA call (they may be captured).
static int g_march_slots = 0;
#ifndef LBM_MARCH_ROWS
#define LBM_MARCH_ROWS 4
#endif
constexpr int kMarchRows = LBM_MARCH_ROWS;  // rows in y per thread of k_phase3m (2 or 4)

cudaError_t phase_prepare(int dim) {
  static bool done = false;
  if (dim != 3 || done) return cudaSuccess;
  int dev = 0, sms = 0, perm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perm, k_phase3m<kMarchRows>, March3::NT, 0);
  if (e == cudaSuccess) {
    g_march_slots = sms * (perm > 0 ? perm : 1);
    done = true;
  }
  return e;
}

static cudaError_t launch_phase3(const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out,
                                 const TileList &next, const TileList &prev, cudaStream_t s) {
  const cudaError_t e = phase_prepare(3);
  if (e != cudaSuccess) return e;
  // one resident wave of warps sharing the (column, plane) units equally, at least MIN_RUN planes each
  constexpr int M = kMarchRows;
  const int ncx = (P.nx + March3::OUT - 1) / March3::OUT, ncy = (P.ny + M - 1) / M;
  const long long units = (long long)ncx * ncy * P.nz;
  const long long want = (units + March3::MIN_RUN - 1) / March3::MIN_RUN;
  long long blocks = (want + March3::WARPS - 1) / March3::WARPS;
  if (blocks > g_march_slots) blocks = g_march_slots;
  if (blocks < 1) blocks = 1;
  const TileList none{};
  return launch_pdl(k_phase3m<M>, dim3((unsigned)blocks), dim3(March3::NT), 0, s, P, phi, u, phi_out,
                    next.tiles ? next : none, next.tiles ? prev : none, ncx, units);
}

cudaError_t launch_phase(int dim, const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out,
                         const TileList &next, const TileList &prev, cudaStream_t s) {
  return dim == 2 ? launch_phase_dim<2>(P, phi, u, phi_out, next.tiles, next.count, s)
                  : launch_phase3(P, phi, u, phi_out, next, prev, s);
}

// Lists the tiles holding an interfacial cell of phi (used after the state is set from the host).
template <int DIM>
__global__ void __launch_bounds__(PhaseGeom<DIM>::NT)
k_gate_tiles(const KParams P, const int32_t *__restrict__ phi, int *__restrict__ tiles, int *__restrict__ ntiles,
             int *__restrict__ mark) {
  using G = PhaseGeom<DIM>;
  const int x = blockIdx.x * G::TX + threadIdx.x, y = blockIdx.y * G::TY + threadIdx.y,
            z = blockIdx.z * G::TZ + threadIdx.z;
  bool gated = false;
  if (x < P.nx && y < P.ny && z < P.nz)
    gated = q_gate_value(phi[(long long)x + (long long)P.nx * (y + (long long)P.ny * z)]) >= P.q_th;
  const int any = __syncthreads_or(gated);
  if (any && threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    const int tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    tiles[atomicAdd(ntiles, 1)] = tile;
    if (mark) mark[tile] = 1;
  }
}

cudaError_t launch_gate_tiles(int dim, const KParams &P, const int32_t *phi, const TileList &list, cudaStream_t s) {
  if (dim == 2) {
    using G = PhaseGeom<2>;
    dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, 1);
    k_gate_tiles<2><<<grid, dim3(G::TX, G::TY, G::TZ), 0, s>>>(P, phi, list.tiles, list.count, nullptr);
  } else {
    using G = PhaseGeom<3>;
    dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, (P.nz + G::TZ - 1) / G::TZ);
    k_gate_tiles<3><<<grid, dim3(G::TX, G::TY, G::TZ), 0, s>>>(P, phi, list.tiles, list.count, list.mark);
  }
  return cudaGetLastError();
}

}  // namespace lbm
