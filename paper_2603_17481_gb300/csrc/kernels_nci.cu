// kernels_nci.cu -- near-contact interaction (Sec. 2.3): interfacial gate (Eqs. 58-59), bounded
// window pairing (Eqs. 60-65), closed-form proximity indicator and repulsive force (Eqs. 66-73).
//
// A block handles one tile: its phi plus a halo of 4 cells (window radius <= 3 plus the gradient
// stencil) is staged in shared memory, normals are computed only at gated cells of the tile + 3
// halo, and the gated cells of the tile are compacted into a list that the warps share out: one
// warp per gated cell, 32 window offsets per iteration in (|r|^2, canonical index) order, stopping
// after the first shell that holds an accepted candidate. Only tiles listed as holding a gated
// cell are visited in a time step. The force is written only at gated cells; the hydrodynamic
// kernel reads it exactly there (same gate function).
#include "launch.h"

namespace lbm {

template <int DIM> struct NciGeom {
  static constexpr int TX = NciTile<DIM>::X, TY = NciTile<DIM>::Y, TZ = NciTile<DIM>::Z;
  static constexpr int H = 4;  // phi halo
  static constexpr int HX = TX + 2 * H, HY = TY + 2 * H, HZ = DIM == 3 ? TZ + 2 * H : 1;
  static constexpr int NB = HX * HY * HZ;
  static constexpr int GX = TX + 2 * (H - 1), GY = TY + 2 * (H - 1), GZ = DIM == 3 ? TZ + 2 * (H - 1) : 1;
  static constexpr int NG = GX * GY * GZ;
  static constexpr int NT = TX * TY * TZ;
  static constexpr size_t smem = sizeof(int32_t) * NB + sizeof(float) * 3 * NG + sizeof(int) * (NT + 1);
};

// One tile of the near-contact pass. All threads of the block call it with the same tile.
template <int DIM>
__device__ __forceinline__ void nci_tile(const KParams &P, const NciTable &T, const int32_t *__restrict__ phi,
                                         float4 *__restrict__ frep, int32_t *__restrict__ partner, int debug,
                                         int bx, int by, int bz, int32_t *s_phi, float *s_n) {
  using G = NciGeom<DIM>;
  using SL = typename StencilOf<DIM>::type;
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + G::TX * (ty + G::TY * tz);
  const int x0 = bx * G::TX, y0 = by * G::TY, z0 = bz * G::TZ;
  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  const bool inb = x < P.nx && y < P.ny && z < P.nz;
  const long long idx = inb ? (long long)x + (long long)P.nx * (y + (long long)P.ny * z) : 0;

  const int32_t v = inb ? phi[idx] : 0;
  const float qx = q_gate_value(v);
  const bool gated = inb && (qx >= P.q_th);
  if (!__syncthreads_or(gated) && !debug) return;

  // phi box with periodic wrap, loaded row by row (rows of HX = TX + 8 values)
  {
    const int xl = wrapn(x0 - G::H + tx, P.nx);
    const int xr = wrapn(x0 - G::H + 32 + (tx & 7), P.nx);
    constexpr int NROWS = G::HY * G::HZ, NW = G::TY * G::TZ;
    for (int r = ty + G::TY * tz; r < NROWS; r += NW) {
      const int ry = r % G::HY, rz = r / G::HY;
      const int Y = wrapn(y0 + ry - G::H, P.ny);
      const int Z = DIM == 3 ? wrapn(z0 + rz - G::H, P.nz) : 0;
      const int32_t *row = phi + (long long)P.nx * (Y + (long long)P.ny * Z);
      s_phi[r * G::HX + tx] = row[xl];
      if (tx < 8) s_phi[r * G::HX + 32 + tx] = row[xr];
    }
  }
  __syncthreads();

  // normals (Eq. 57, isotropic gradient of Eq. 22) at gated cells of the tile + 3 halo
  for (int t = tid; t < G::NG; t += G::NT) {
    int gx = t % G::GX, gy = (t / G::GX) % G::GY, gz = t / (G::GX * G::GY);
    int b = (DIM == 3 ? (gz + 1) * G::HX * G::HY : 0) + (gy + 1) * G::HX + gx + 1;
    int32_t vc = s_phi[b];
    if (q_gate_value(vc) >= P.q_th) {
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
      const float inv = 1.0f / (sqrtf(g0 * g0 + g1 * g1 + g2 * g2) + P.eps_n);
      s_n[t] = g0 * inv;
      s_n[G::NG + t] = g1 * inv;
      s_n[2 * G::NG + t] = g2 * inv;
    }
  }
  // compact list of the tile's gated cells (tile-local linear index)
  int *s_list = reinterpret_cast<int *>(s_n + 3 * G::NG);
  int *s_count = s_list + G::NT;
  if (tid == 0) *s_count = 0;
  __syncthreads();
  {
    const unsigned m = __ballot_sync(0xffffffffu, gated);
    const int lane = tid & 31;
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(s_count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (gated) s_list[base + __popc(m & ((1u << lane) - 1u))] = tid;
  }
  __syncthreads();

  // one warp per gated cell: the 32 lanes test 32 window offsets at a time, in (|r|^2, canonical
  // index) order; the candidate criteria are Eqs. 59, 61 and 62, and the winner is the nearest
  // accepted candidate, then the largest facing score, then the first in table order (the
  // packed key below orders exactly that way).
  const int lane = tid & 31, warp = tid >> 5;
  const int ncell = *s_count;
  for (int k = warp; k < ncell; k += G::NT / 32) {
    const int c = s_list[k];
    const int cx = c % G::TX, cy = (c / G::TX) % G::TY, cz = c / (G::TX * G::TY);
    const int ob = (DIM == 3 ? (cz + G::H) * G::HX * G::HY : 0) + (cy + G::H) * G::HX + cx + G::H;
    const int on = (DIM == 3 ? (cz + G::H - 1) * G::GX * G::GY : 0) + (cy + G::H - 1) * G::GX + cx + G::H - 1;
    const int32_t vx = s_phi[ob];
    const float qxc = q_gate_value(vx);
    const float n0 = s_n[on], n1 = s_n[G::NG + on], n2 = s_n[2 * G::NG + on];
    const float sim = __fmul_rn(P.eta, fmaxf(qxc, P.eps_q));
    unsigned long long best = ~0ull;
    for (int j0 = 0; j0 < T.count; j0 += 32) {
      // stop once a candidate is held and this chunk starts beyond its shell
      if (best != ~0ull && (int)T.o[j0].d2 > (int)(best >> 40)) break;
      const int j = j0 + lane;
      unsigned long long key = ~0ull;
      if (j < T.count) {
        const NciOffset o = T.o[j];
        const int32_t vy = s_phi[ob + o.dx + G::HX * (o.dy + G::HY * o.dz)];
        const float qy = q_gate_value(vy);
        if (qy >= P.q_th && fabsf(__fsub_rn(qy, qxc)) <= sim) {
          const int yn = on + o.dx + G::GX * (o.dy + G::GY * o.dz);
          const float dot = __fadd_rn(__fadd_rn(__fmul_rn(n0, s_n[yn]), __fmul_rn(n1, s_n[G::NG + yn])),
                                      __fmul_rn(n2, s_n[2 * G::NG + yn]));
          if (dot <= P.cos_opp) {
            const float ff = fmaxf(-dot, 0.0f);
            key = ((unsigned long long)o.d2 << 40) | ((unsigned long long)(0x7fffffffu - __float_as_uint(ff)) << 9) |
                  (unsigned long long)j;
          }
        }
      }
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, sh);
        key = other < key ? other : key;
      }
      best = key < best ? key : best;
    }
    if (lane != 0) continue;
    const long long gidx = (long long)(x0 + cx) + (long long)P.nx * ((y0 + cy) + (long long)P.ny * (z0 + cz));
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (best != ~0ull) {
      const int bj = (int)(best & 511ull);
      const NciOffset o = T.o[bj];
      const float ff = __uint_as_float(0x7fffffffu - (unsigned)((best >> 9) & 0x7fffffffull));
      const int32_t vy = s_phi[ob + o.dx + G::HX * (o.dy + G::HY * o.dz)];
      const int yn = on + o.dx + G::GX * (o.dy + G::GY * o.dz);
      const float m0 = s_n[yn], m1 = s_n[G::NG + yn], m2 = s_n[2 * G::NG + yn];
      const float qy = q_gate_value(vy);
      // paired indicator and clamp, Eqs. 66-67
      const float qpair = 0.5f * (qxc + qy);
      const float qcl = fminf(fmaxf(qpair, P.eps_q), 0.25f - P.eps_q);
      // proximity indicator, Eq. 70, as eps * artanh(sqrt(1 - 4 q)): the same value, and
      // 1 - 4 q_pair = ((1 - 2 phi_x)^2 + (1 - 2 phi_y)^2) / 2 has no cancellation
      float mm;
      if (qcl == qpair) {
        const float ax = 1.0f - 2.0f * fminf(fmaxf(phi_of(vx), 0.f), 1.f);
        const float ay = 1.0f - 2.0f * fminf(fmaxf(phi_of(vy), 0.f), 1.f);
        mm = 0.5f * (ax * ax + ay * ay);
      } else {
        mm = 1.0f - 4.0f * qcl;
      }
      const float h = P.eps * atanhf(sqrtf(mm));
      const float t = h / P.h0;
      const float tp = (P.p == 4.0f) ? (t * t) * (t * t) : powf(t, P.p);
      const float wh = 1.0f / (1.0f + tp);  // Eq. 71
      // symmetric normal, Eq. 69, line-of-centres fallback, oriented toward the partner
      const float rn = sqrtf((float)o.d2);
      const float r0 = o.dx / rn, r1 = o.dy / rn, r2 = o.dz / rn;
      float s0 = n0 - m0, s1 = n1 - m1, s2 = n2 - m2;
      const float sn = sqrtf(s0 * s0 + s1 * s1 + s2 * s2);
      if (sn < 1e-8f) {
        s0 = r0; s1 = r1; s2 = r2;
      } else {
        const float is = 1.0f / (sn + P.eps_n);
        s0 *= is; s1 *= is; s2 *= is;
      }
      if (r0 * s0 + r1 * s1 + r2 * s2 < 0.0f) {
        s0 = -s0; s1 = -s1; s2 = -s2;
      }
      // flux and force density with the facing factor of Eq. 68, Eqs. 72-73
      const float rho = P.rho_g + P.drho * phi_of(vx);
      const float amp = rho * P.A_rep * qcl * wh * ff;
      out = make_float4(amp * s0, amp * s1, DIM == 3 ? amp * s2 : 0.0f, 1.0f);
      if (partner) {
        partner[3 * gidx] = o.dx;
        partner[3 * gidx + 1] = o.dy;
        partner[3 * gidx + 2] = o.dz;
      }
    } else if (partner) {
      partner[3 * gidx] = partner[3 * gidx + 1] = partner[3 * gidx + 2] = INT32_MIN;
    }
    frep[gidx] = out;
  }
  // debug read-back: every non-gated cell reports no partner and zero force
  if (debug && inb && !gated) {
    frep[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (partner) partner[3 * idx] = partner[3 * idx + 1] = partner[3 * idx + 2] = INT32_MIN;
  }
}

// Every tile of the grid (used for the diagnostic read-back, where every cell reports).
template <int DIM>
__global__ void __launch_bounds__(NciGeom<DIM>::NT)
k_nci_full(const KParams P, const NciTable T, const int32_t *__restrict__ phi, float4 *__restrict__ frep,
           int32_t *__restrict__ partner, int debug) {
  using G = NciGeom<DIM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t *s_phi = reinterpret_cast<int32_t *>(smem_raw);
  float *s_n = reinterpret_cast<float *>(smem_raw + sizeof(int32_t) * G::NB);
  nci_tile<DIM>(P, T, phi, frep, partner, debug, blockIdx.x, blockIdx.y, blockIdx.z, s_phi, s_n);
}

// Only the tiles listed by the phase-field kernel (those holding an interfacial cell); a grid of
// resident blocks walks the list.
template <int DIM>
__global__ void __launch_bounds__(NciGeom<DIM>::NT)
k_nci_list(const KParams P, const NciTable T, const int32_t *__restrict__ phi, float4 *__restrict__ frep,
           const int *__restrict__ tiles, const int *__restrict__ ntiles, int gtx, int gty) {
  using G = NciGeom<DIM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t *s_phi = reinterpret_cast<int32_t *>(smem_raw);
  float *s_n = reinterpret_cast<float *>(smem_raw + sizeof(int32_t) * G::NB);
  const int n = *ntiles;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int tile = tiles[t];
    const int bx = tile % gtx, by = (tile / gtx) % gty, bz = tile / (gtx * gty);
    nci_tile<DIM>(P, T, phi, frep, nullptr, 0, bx, by, bz, s_phi, s_n);
    __syncthreads();
  }
}

template <int DIM>
static cudaError_t nci_attr() {
  using G = NciGeom<DIM>;
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_nci_full<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_nci_list<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int DIM>
static cudaError_t launch_nci_dim(const KParams &P, const NciTable &T, const int32_t *phi, float4 *frep,
                                  int32_t *partner, int debug, const int *tiles, const int *ntiles, int list_blocks,
                                  cudaStream_t s) {
  using G = NciGeom<DIM>;
  cudaError_t e = nci_attr<DIM>();
  if (e != cudaSuccess) return e;
  dim3 block(G::TX, G::TY, G::TZ);
  dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, (P.nz + G::TZ - 1) / G::TZ);
  if (tiles)
    k_nci_list<DIM><<<list_blocks, block, G::smem, s>>>(P, T, phi, frep, tiles, ntiles, grid.x, grid.y);
  else
    k_nci_full<DIM><<<grid, block, G::smem, s>>>(P, T, phi, frep, partner, debug);
  return cudaGetLastError();
}

cudaError_t launch_nci(int dim, const KParams &P, const NciTable &T, const int32_t *phi, float4 *frep,
                       int32_t *partner, int debug, const int *tiles, const int *ntiles, int list_blocks,
                       cudaStream_t s) {
  return dim == 2 ? launch_nci_dim<2>(P, T, phi, frep, partner, debug, tiles, ntiles, list_blocks, s)
                  : launch_nci_dim<3>(P, T, phi, frep, partner, debug, tiles, ntiles, list_blocks, s);
}

int nci_list_blocks(int dim) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dim == 2) {
    if (nci_attr<2>() != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_nci_list<2>, NciGeom<2>::NT, NciGeom<2>::smem);
  } else {
    if (nci_attr<3>() != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_nci_list<3>, NciGeom<3>::NT, NciGeom<3>::smem);
  }
  return sms * (per > 0 ? per : 1);
}

}  // namespace lbm
