// kernels_nci.cu -- near-contact interaction (Sec. 2.3): interfacial gate (Eqs. 58-59), bounded
// window pairing (Eqs. 60-65), closed-form proximity indicator and repulsive force (Eqs. 66-73).
//
// One thread per cell of a tile. The tile's phi plus a halo of 4 cells (window radius <= 3 plus
// the gradient stencil) is staged in shared memory; normals are computed only at gated cells of
// the tile + 3 halo; each gated cell scans the window offsets in (|r|^2, canonical index) order
// and stops after the first shell that holds an accepted candidate. Tiles without a gated cell
// exit after one coalesced read of their phi. The force is written only at gated cells; the
// hydrodynamic kernel reads it exactly there (same gate function).
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
  static constexpr size_t smem = sizeof(int32_t) * NB + sizeof(float) * 3 * NG;
};

template <int DIM>
__global__ void __launch_bounds__(NciGeom<DIM>::NT)
k_nci(const KParams P, const NciTable T, const int32_t *__restrict__ phi, float4 *__restrict__ frep,
      int32_t *__restrict__ partner, int debug) {
  using G = NciGeom<DIM>;
  using SL = typename StencilOf<DIM>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t *s_phi = reinterpret_cast<int32_t *>(smem_raw);
  float *s_n = reinterpret_cast<float *>(smem_raw + sizeof(int32_t) * G::NB);

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + G::TX * (ty + G::TY * tz);
  const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * G::TY, z0 = blockIdx.z * G::TZ;
  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  const bool inb = x < P.nx && y < P.ny && z < P.nz;
  const long long idx = inb ? (long long)x + (long long)P.nx * (y + (long long)P.ny * z) : 0;

  const int32_t v = inb ? phi[idx] : 0;
  const float qx = q_gate_value(v);
  const bool gated = inb && (qx >= P.q_th);
  if (!__syncthreads_or(gated) && !debug) return;

  // phi box with periodic wrap
  for (int t = tid; t < G::NB; t += G::NT) {
    int bx = t % G::HX, by = (t / G::HX) % G::HY, bz = t / (G::HX * G::HY);
    int X = wrapi(x0 + bx - G::H, P.nx), Y = wrapi(y0 + by - G::H, P.ny);
    int Z = DIM == 3 ? wrapi(z0 + bz - G::H, P.nz) : 0;
    s_phi[t] = phi[(long long)X + (long long)P.nx * (Y + (long long)P.ny * Z)];
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
  __syncthreads();
  if (!inb) return;

  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  int best = -1;
  if (gated) {
    const int ob = (DIM == 3 ? (tz + G::H) * G::HX * G::HY : 0) + (ty + G::H) * G::HX + tx + G::H;
    const int on = (DIM == 3 ? (tz + G::H - 1) * G::GX * G::GY : 0) + (ty + G::H - 1) * G::GX + tx + G::H - 1;
    const float n0 = s_n[on], n1 = s_n[G::NG + on], n2 = s_n[2 * G::NG + on];
    const float sim = __fmul_rn(P.eta, fmaxf(qx, P.eps_q));
    int bd2 = 1 << 30;
    float bff = 0.f;
    // candidate criteria Eqs. 59, 61, 62; nearest first, then largest facing score, then the
    // smallest canonical index (the table is sorted that way)
    for (int k = 0; k < T.count; k++) {
      const NciOffset o = T.o[k];
      if (o.d2 > bd2) break;
      const int32_t vy = s_phi[ob + o.dx + G::HX * (o.dy + G::HY * o.dz)];
      const float qy = q_gate_value(vy);
      if (!(qy >= P.q_th)) continue;
      if (!(fabsf(__fsub_rn(qy, qx)) <= sim)) continue;
      const int yn = on + o.dx + G::GX * (o.dy + G::GY * o.dz);
      const float dot = __fadd_rn(__fadd_rn(__fmul_rn(n0, s_n[yn]), __fmul_rn(n1, s_n[G::NG + yn])),
                                  __fmul_rn(n2, s_n[2 * G::NG + yn]));
      if (!(dot <= P.cos_opp)) continue;
      const float ff = fmaxf(-dot, 0.0f);
      if (best < 0 || ff > bff) {
        best = k;
        bd2 = o.d2;
        bff = ff;
      }
    }
    if (best >= 0) {
      const NciOffset o = T.o[best];
      const int32_t vy = s_phi[ob + o.dx + G::HX * (o.dy + G::HY * o.dz)];
      const int yn = on + o.dx + G::GX * (o.dy + G::GY * o.dz);
      const float m0 = s_n[yn], m1 = s_n[G::NG + yn], m2 = s_n[2 * G::NG + yn];
      const float qy = q_gate_value(vy);
      // paired indicator and clamp, Eqs. 66-67
      const float qpair = 0.5f * (qx + qy);
      const float qcl = fminf(fmaxf(qpair, P.eps_q), 0.25f - P.eps_q);
      // proximity indicator, Eq. 70, as eps * artanh(sqrt(1 - 4 q)): the same value, and
      // 1 - 4 q_pair = ((1 - 2 phi_x)^2 + (1 - 2 phi_y)^2) / 2 has no cancellation
      float mm;
      if (qcl == qpair) {
        const float ax = 1.0f - 2.0f * fminf(fmaxf(phi_of(v), 0.f), 1.f);
        const float ay = 1.0f - 2.0f * fminf(fmaxf(phi_of(vy), 0.f), 1.f);
        mm = 0.5f * (ax * ax + ay * ay);
      } else {
        mm = 1.0f - 4.0f * qcl;
      }
      const float h = P.eps * atanhf(sqrtf(mm));
      const float t = h / P.h0;
      const float tp = (P.p == 4.0f) ? (t * t) * (t * t) : powf(t, P.p);
      const float wh = 1.0f / (1.0f + tp);  // Eq. 71
      // facing factor, Eq. 68 (the score of the chosen candidate)
      const float ff = bff;
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
      // flux and force density, Eqs. 72-73
      const float rho = P.rho_g + P.drho * phi_of(v);
      const float amp = rho * P.A_rep * qcl * wh * ff;
      out = make_float4(amp * s0, amp * s1, DIM == 3 ? amp * s2 : 0.0f, 1.0f);
    }
    frep[idx] = out;
  } else if (debug) {
    frep[idx] = out;
  }
  if (partner) {
    if (best >= 0) {
      const NciOffset o = T.o[best];
      partner[3 * idx] = o.dx;
      partner[3 * idx + 1] = o.dy;
      partner[3 * idx + 2] = o.dz;
    } else {
      partner[3 * idx] = partner[3 * idx + 1] = partner[3 * idx + 2] = INT32_MIN;
    }
  }
}

template <int DIM>
static cudaError_t launch_nci_dim(const KParams &P, const NciTable &T, const int32_t *phi, float4 *frep,
                                  int32_t *partner, int debug, cudaStream_t s) {
  using G = NciGeom<DIM>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_nci<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  dim3 block(G::TX, G::TY, G::TZ);
  dim3 grid((P.nx + G::TX - 1) / G::TX, (P.ny + G::TY - 1) / G::TY, (P.nz + G::TZ - 1) / G::TZ);
  k_nci<DIM><<<grid, block, G::smem, s>>>(P, T, phi, frep, partner, debug);
  return cudaGetLastError();
}

cudaError_t launch_nci(int dim, const KParams &P, const NciTable &T, const int32_t *phi, float4 *frep,
                       int32_t *partner, int debug, cudaStream_t s) {
  return dim == 2 ? launch_nci_dim<2>(P, T, phi, frep, partner, debug, s)
                  : launch_nci_dim<3>(P, T, phi, frep, partner, debug, s);
}

}  // namespace lbm
