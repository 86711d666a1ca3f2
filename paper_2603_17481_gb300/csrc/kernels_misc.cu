// kernels_misc.cu -- conversions between the FP64 host layout and the device state, equilibrium
// initialisation, and the FP64 / exact-integer reductions of the periodic conservation check.
#include "launch.h"

namespace lbm {

cudaError_t launch_hydro_q9(int, int, const KParams &, const void *, void *, const int32_t *, const float4 *,
                            float *, float *, cudaStream_t);
cudaError_t launch_hydro_q19(int, int, const KParams &, const void *, void *, const int32_t *, const float4 *,
                             float *, float *, cudaStream_t);
cudaError_t launch_hydro_q27(int, int, const KParams &, const void *, void *, const int32_t *, const float4 *,
                             float *, float *, cudaStream_t);
cudaError_t launch_split_q19(int, int, const KParams &, const void *, void *, const int32_t *, const float4 *,
                             float *, const TileList &, int, cudaStream_t);
cudaError_t launch_split_q27(int, int, const KParams &, const void *, void *, const int32_t *, const float4 *,
                             float *, const TileList &, int, cudaStream_t);

cudaError_t launch_hydro(int Q, int store, int mode, const KParams &P, const void *src, void *dst,
                         const int32_t *phi, const float4 *frep, float *u, float *pstar, cudaStream_t s) {
  switch (Q) {
    case 9: return launch_hydro_q9(store, mode, P, src, dst, phi, frep, u, pstar, s);
    case 19: return launch_hydro_q19(store, mode, P, src, dst, phi, frep, u, pstar, s);
    default: return launch_hydro_q27(store, mode, P, src, dst, phi, frep, u, pstar, s);
  }
}

bool hydro_split_applies(int Q, const KParams &P) {
  return (Q == 19 || Q == 27) && P.nx % 2 == 0 && (long long)Q * P.N <= (1LL << 32);
}

cudaError_t launch_hydro_split(int part, int Q, int store, const KParams &P, const void *src, void *dst,
                               const int32_t *phi, const float4 *frep, float *u, const TileList &listed, int blocks,
                               cudaStream_t s) {
  if (!hydro_split_applies(Q, P)) return cudaErrorInvalidValue;
  return Q == 19 ? launch_split_q19(part, store, P, src, dst, phi, frep, u, listed, blocks, s)
                 : launch_split_q27(part, store, P, src, dst, phi, frep, u, listed, blocks, s);
}

int tile_count(int dim, const KParams &P) {
  using T2 = PhaseTile<2>;
  using T3 = PhaseTile<3>;
  if (dim == 2) return ((P.nx + T2::X - 1) / T2::X) * ((P.ny + T2::Y - 1) / T2::Y);
  return ((P.nx + T3::X - 1) / T3::X) * ((P.ny + T3::Y - 1) / T3::Y) * ((P.nz + T3::Z - 1) / T3::Z);
}

static inline dim3 grid1d(long long n, int bs) {
  long long g = (n + bs - 1) / bs;
  return dim3((unsigned)(g < 1 ? 1 : g));
}

// phi (FP64) -> signed 2.30 fixed point, round to nearest, saturating
__global__ void k_phi_in(long long N, const double *__restrict__ in, int32_t *__restrict__ out) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  double v = in[n] * 1073741824.0;
  v = fmin(fmax(v, -2147483648.0), 2147483647.0);
  out[n] = (int32_t)__double2ll_rn(v);
}
__global__ void k_phi_out(long long N, const int32_t *__restrict__ in, double *__restrict__ out) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  out[n] = (double)in[n] * (1.0 / 1073741824.0);
}
__global__ void k_f32_out(long long n_, const float *__restrict__ in, double *__restrict__ out) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= n_) return;
  out[n] = (double)in[n];
}

cudaError_t launch_phi_in(const KParams &P, const double *phi64, int32_t *phi, cudaStream_t s) {
  k_phi_in<<<grid1d(P.N, 256), 256, 0, s>>>(P.N, phi64, phi);
  return cudaGetLastError();
}
cudaError_t launch_phi_out(const KParams &P, const int32_t *phi, double *phi64, cudaStream_t s) {
  k_phi_out<<<grid1d(P.N, 256), 256, 0, s>>>(P.N, phi, phi64);
  return cudaGetLastError();
}
cudaError_t launch_f32_out(long long n, const float *src, double *dst, cudaStream_t s) {
  k_f32_out<<<grid1d(n, 256), 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}

__device__ __forceinline__ long long cell_shift(const KParams &P, int x, int y, int z, int cx, int cy, int cz,
                                                int dim) {
  int X = x + cx, Y = y + cy, Z = z + cz;
  X = X < 0 ? X + P.nx : (X >= P.nx ? X - P.nx : X);
  Y = Y < 0 ? Y + P.ny : (Y >= P.ny ? Y - P.ny : Y);
  if (dim == 3) Z = Z < 0 ? Z + P.nz : (Z >= P.nz ? Z - P.nz : Z);
  else Z = 0;
  return (long long)X + (long long)P.nx * (Y + (long long)P.ny * Z);
}

// Initial populations f_eq(p*, u) (Eq. 11), stored for the pull scheme: buffer cell y holds the
// population that streams to y + c_i, i.e. f_eq_i at y + c_i. The thread of cell m evaluates its
// own f_eq_i and writes it to m - c_i (each cell's fields are read once). The equilibrium is
// evaluated in FP32, the precision of every later update, in its even / odd split over the pair
// (c, -c): with A = p* - 1.5 |u|^2 and B = 3 - 4.5 |u|^2,
//   f_eq(+-c) / w = E +- O,  E = A + 4.5 (c.u)^2,  O = (c.u)(B + 4.5 (c.u)^2),
// which is the third-order polynomial of Eq. 11 regrouped (cs^2 = 1/3); each c.u is a sum of
// signed velocity components. GB300 runs FP64 at a small fraction of its FP32 rate: the same
// polynomial in FP64 took as long as seven time steps of the grid.
template <class L, int S>
__global__ void k_init_pops(const KParams P, const double *__restrict__ u64, const double *__restrict__ ps64,
                            typename Store<S>::T *__restrict__ pops) {
  long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= P.N) return;
  int x = (int)(m % P.nx), y = (int)((m / P.nx) % P.ny), z = (int)(m / ((long long)P.nx * P.ny));
  const float u[3] = {(float)u64[m], (float)u64[P.N + m], L::D == 3 ? (float)u64[2 * P.N + m] : 0.0f};
  const float ps = ps64 ? (float)ps64[m] : 0.0f;
  const float uu = __fmaf_rn(u[0], u[0], __fmaf_rn(u[1], u[1], __fmul_rn(u[2], u[2])));
  const float A = __fmaf_rn(-1.5f, uu, ps), B = __fmaf_rn(-4.5f, uu, 3.0f);
  auto put = [&](int i, float g) {
    const long long n = cell_shift(P, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2), L::D);
    Store<S>::st_w(pops + (long long)i * P.N + n, g, L::w(i));
  };
  put(0, A);
#pragma unroll
  for (int i = 1; i < L::Q; i++) {
    if (L::opp(i) < i) continue;  // each pair once, through its lower index
    float cu = 0.0f;
#pragma unroll
    for (int a = 0; a < L::D; a++) {
      if (L::c(i, a) > 0) cu = __fadd_rn(cu, u[a]);
      if (L::c(i, a) < 0) cu = __fsub_rn(cu, u[a]);
    }
    const float s = __fmul_rn(cu, cu);
    const float E = __fmaf_rn(4.5f, s, A), O = __fmul_rn(cu, __fmaf_rn(4.5f, s, B));
    put(i, __fadd_rn(E, O));
    put(L::opp(i), __fsub_rn(E, O));
  }
}

// Host pre-collision populations f[i][x] -> pull storage buf[i][x - c_i] = f[i][x].
template <class L, int S>
__global__ void k_set_pops(const KParams P, const double *__restrict__ f64, typename Store<S>::T *__restrict__ pops) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= P.N) return;
  int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / ((long long)P.nx * P.ny));
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    long long m = cell_shift(P, x, y, z, L::c(i, 0), L::c(i, 1), L::c(i, 2), L::D);
    Store<S>::st(pops + (long long)i * P.N + n, (float)f64[(long long)i * P.N + m], L::w(i));
  }
}

template <class L, int S>
__global__ void k_get_pops(const KParams P, const typename Store<S>::T *__restrict__ pops, double *__restrict__ f64) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= P.N) return;
  int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / ((long long)P.nx * P.ny));
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    long long m = cell_shift(P, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2), L::D);
    f64[(long long)i * P.N + n] = (double)Store<S>::ld(pops + (long long)i * P.N + m, L::w(i));
  }
}

// Moment-record storage: the record of the equilibrium f_eq(p*, u) at every cell (B = 0, r = 0),
// so that cell x pulls f_eq_i of x - c_i at the first step.
__global__ void k_init_record(const KParams P, const double *__restrict__ u64, const double *__restrict__ ps64,
                              float4 *__restrict__ rec) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= P.N) return;
  const double u0 = u64[n], u1 = u64[P.N + n], u2 = u64[2 * P.N + n];
  const double ps = ps64 ? ps64[n] : 0.0;
  const double uu = u0 * u0 + u1 * u1 + u2 * u2;
  rec[n] = make_float4((float)(ps - 1.5 * uu), (float)(3.0 - 4.5 * uu), (float)u0, (float)u1);
  rec[P.N + n] = make_float4((float)u2, 0.f, 0.f, 0.f);
  rec[2 * P.N + n] = make_float4(0.f, 0.f, 0.f, 0.f);
  rec[3 * P.N + n] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Pre-collision populations f[i][x] of the moment-record state: direction i of the record of x - c_i.
template <class L>
__global__ void k_get_record(const KParams P, const float4 *__restrict__ rec, double *__restrict__ f64) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= P.N) return;
  int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / ((long long)P.nx * P.ny));
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    const float4 *q = rec + cell_shift(P, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2), L::D);
    f64[(long long)i * P.N + n] = (double)(L::w(i) * record_f_over_w<L>(i, q[0], q[P.N], q[2 * P.N], q[3 * P.N]));
  }
}

template <class L>
static cudaError_t pops_dispatch_l(int what, int store, const KParams &P, const double *a, const double *b,
                                   void *pops, double *out, cudaStream_t s) {
  dim3 g = grid1d(P.N, 128);
  if (store == kStoreRecord) {  // 3D only; populations cannot be set in record form
    if (L::D != 3 || what == 1) return cudaErrorInvalidValue;
    if (what == 0) k_init_record<<<g, 128, 0, s>>>(P, a, b, (float4 *)pops);
    else k_get_record<L><<<g, 128, 0, s>>>(P, (const float4 *)pops, out);
    return cudaGetLastError();
  }
#define LBM_POPS_CASE(SV)                                                                              \
  case SV: {                                                                                           \
    using T = typename Store<SV>::T;                                                                   \
    if (what == 0) k_init_pops<L, SV><<<g, 128, 0, s>>>(P, a, b, (T *)pops);                           \
    else if (what == 1) k_set_pops<L, SV><<<g, 128, 0, s>>>(P, a, (T *)pops);                          \
    else k_get_pops<L, SV><<<g, 128, 0, s>>>(P, (const T *)pops, out);                                 \
    break;                                                                                             \
  }
  switch (store) {
    LBM_POPS_CASE(0)
    LBM_POPS_CASE(1)
    LBM_POPS_CASE(2)
    default: return cudaErrorInvalidValue;
  }
#undef LBM_POPS_CASE
  return cudaGetLastError();
}

static cudaError_t pops_dispatch(int Q, int what, int store, const KParams &P, const double *a, const double *b,
                                 void *pops, double *out, cudaStream_t s) {
  switch (Q) {
    case 9: return pops_dispatch_l<D2Q9>(what, store, P, a, b, pops, out, s);
    case 19: return pops_dispatch_l<D3Q19>(what, store, P, a, b, pops, out, s);
    default: return pops_dispatch_l<D3Q27>(what, store, P, a, b, pops, out, s);
  }
}

cudaError_t launch_init_pops(int Q, int store, const KParams &P, const double *u64, const double *ps64, void *pops,
                             cudaStream_t s) {
  return pops_dispatch(Q, 0, store, P, u64, ps64, pops, nullptr, s);
}
cudaError_t launch_set_pops(int Q, int store, const KParams &P, const double *f64, void *pops, cudaStream_t s) {
  return pops_dispatch(Q, 1, store, P, f64, nullptr, pops, nullptr, s);
}
cudaError_t launch_get_pops(int Q, int store, const KParams &P, const void *pops, double *f64, cudaStream_t s) {
  return pops_dispatch(Q, 2, store, P, nullptr, nullptr, const_cast<void *>(pops), f64, s);
}

__global__ void k_frep_out(long long N, int dim, const float4 *__restrict__ frep, double *__restrict__ out) {
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  float4 f = frep[n];
  out[n] = f.x;
  out[N + n] = f.y;
  out[2 * N + n] = dim == 3 ? f.z : 0.0;
}
cudaError_t launch_partner_frep_out(const KParams &P, int dim, const float4 *frep, double *frep64, cudaStream_t s) {
  k_frep_out<<<grid1d(P.N, 256), 256, 0, s>>>(P.N, dim, frep, frep64);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Reductions: fixed grid, fixed per-thread strides and a fixed tree, so the FP64 results are
// reproducible run to run; the phi sum is an exact 64-bit integer sum of the fixed-point field.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kReduceThreads = 256;

// MOM = false leaves out the FP64 momentum sums (GB300's FP64 rate makes them the cost of this
// kernel): the phi sum and, when u is given, the non-finite count only.
template <bool MOM>
__global__ void __launch_bounds__(kReduceThreads)
k_reduce_partial(const KParams P, const int32_t *__restrict__ phi, const float *__restrict__ u,
                 ReduceOut *__restrict__ partials) {
  long long sphi = 0, nonfin = 0;
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += stride) {
    const int32_t v = phi[n];
    sphi += v;
    if (!MOM && !u) continue;
    const float a = u[n], b = u[P.N + n], c = u[2 * P.N + n];
    if (!isfinite(a) || !isfinite(b) || !isfinite(c)) nonfin++;
    if constexpr (MOM) {
      const double rho = P.rho_g64 + P.drho64 * ((double)v * (1.0 / 1073741824.0));
      m0 += rho * a;
      m1 += rho * b;
      m2 += rho * c;
    }
  }
  __shared__ double sm[3][kReduceThreads / 32];
  __shared__ long long sl[2][kReduceThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  m0 = warp_sum(m0); m1 = warp_sum(m1); m2 = warp_sum(m2);
  sphi = warp_sum_ll(sphi); nonfin = warp_sum_ll(nonfin);
  if (lane == 0) {
    sm[0][wid] = m0; sm[1][wid] = m1; sm[2][wid] = m2;
    sl[0][wid] = sphi; sl[1][wid] = nonfin;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ReduceOut r{0, {0.0, 0.0, 0.0}, 0};
    for (int k = 0; k < kReduceThreads / 32; k++) {
      r.mom[0] += sm[0][k]; r.mom[1] += sm[1][k]; r.mom[2] += sm[2][k];
      r.phi_q30 += sl[0][k]; r.nonfinite += sl[1][k];
    }
    partials[blockIdx.x] = r;
  }
}

// One warp: lane l sums partials l, l + 32, ... in order, then a fixed shuffle tree.
__global__ void k_reduce_final(const ReduceOut *__restrict__ partials, int n, ReduceOut *__restrict__ out) {
  if (blockIdx.x != 0) return;
  const int lane = threadIdx.x;
  long long sphi = 0, nonfin = 0;
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  for (int k = lane; k < n; k += 32) {
    sphi += partials[k].phi_q30;
    nonfin += partials[k].nonfinite;
    m0 += partials[k].mom[0];
    m1 += partials[k].mom[1];
    m2 += partials[k].mom[2];
  }
  m0 = warp_sum(m0); m1 = warp_sum(m1); m2 = warp_sum(m2);
  sphi = warp_sum_ll(sphi); nonfin = warp_sum_ll(nonfin);
  if (lane == 0) {
    ReduceOut r;
    r.phi_q30 = sphi;
    r.nonfinite = nonfin;
    r.mom[0] = m0; r.mom[1] = m1; r.mom[2] = m2;
    *out = r;
  }
}

cudaError_t launch_reduce_n(const KParams &P, const int32_t *phi, const float *u, ReduceOut *partials, int nblocks,
                            ReduceOut *out, cudaStream_t s) {
  k_reduce_partial<true><<<nblocks, kReduceThreads, 0, s>>>(P, phi, u, partials);
  k_reduce_final<<<1, 32, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const KParams &P, const int32_t *phi, const float *u, ReduceOut *partials, ReduceOut *out,
                          cudaStream_t s, bool mom) {
  if (mom) k_reduce_partial<true><<<kReduceBlocks, kReduceThreads, 0, s>>>(P, phi, u, partials);
  else k_reduce_partial<false><<<kReduceBlocks, kReduceThreads, 0, s>>>(P, phi, u, partials);
  k_reduce_final<<<1, 32, 0, s>>>(partials, kReduceBlocks, out);
  return cudaGetLastError();
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Film statistics of Sec. 3.3 (Eq. 74): per film cell, n = grad(phi) / (|grad(phi)| + eps_n) and
// F_cap = mu_phi grad(phi) from the isotropic stencils (Eqs. 19, 22, 23), in FP32 as in the hydro
// kernel; sums in FP64 over a fixed grid, then a fixed tree.
template <int DIM>
__global__ void __launch_bounds__(kReduceThreads)
k_nci_diag_partial(const KParams P, const int32_t *__restrict__ phi, const float4 *__restrict__ frep,
                   DiagOut *__restrict__ partials) {
  using SL = typename StencilOf<DIM>::type;
  double vf = 0.0, srn = 0.0, scn = 0.0, fmx = 0.0, sab = 0.0;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += stride) {
    const int32_t v = phi[n];
    if (!(q_gate_value(v) >= P.q_th)) continue;
    const float4 fr = frep[n];
    if (!(fr.w > 0.5f)) continue;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
    const float ph = phi_of(v);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, lap = 0.f;
#pragma unroll
    for (int i = 1; i < SL::Q; i++) {
      if (!positive<SL>(i)) continue;
      const int c0 = SL::c(i, 0), c1 = SL::c(i, 1), c2 = SL::c(i, 2);
      const long long ip = wrapn(x + c0, nx) + (long long)nx * (wrapn(y + c1, ny) + (long long)ny * wrapn(z + c2, nz));
      const long long im = wrapn(x - c0, nx) + (long long)nx * (wrapn(y - c1, ny) + (long long)ny * wrapn(z - c2, nz));
      const float vp = phi_of(phi[ip]), vm = phi_of(phi[im]);
      const float d = SL::w(i) * (vp - vm);
      g0 += c0 * d;
      g1 += c1 * d;
      g2 += c2 * d;
      lap += SL::w(i) * ((vp - ph) + (vm - ph));
    }
    g0 *= 3.0f; g1 *= 3.0f; g2 *= 3.0f;
    lap *= 6.0f;
    const float muphi = P.beta4 * ph * (ph - 1.0f) * (ph - 0.5f) - P.kap * lap;
    const float gg = g0 * g0 + g1 * g1 + g2 * g2;
    const float inv = 1.0f / (sqrtf(gg) + P.eps_n);
    const double rn = (double)((fr.x * g0 + fr.y * g1 + fr.z * g2) * inv);
    const double cn = (double)(muphi * gg * inv);
    const double fa = sqrt((double)fr.x * fr.x + (double)fr.y * fr.y + (double)fr.z * fr.z);
    vf += 1.0;
    srn += fabs(rn);
    scn += fabs(cn);
    sab += fa;
    fmx = fmax(fmx, fa);
  }
  __shared__ double sm[5][kReduceThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  vf = warp_sum(vf); srn = warp_sum(srn); scn = warp_sum(scn); sab = warp_sum(sab); fmx = warp_max(fmx);
  if (lane == 0) {
    sm[0][wid] = vf; sm[1][wid] = srn; sm[2][wid] = scn; sm[3][wid] = fmx; sm[4][wid] = sab;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    DiagOut r{{0.0, 0.0, 0.0, 0.0, 0.0}};
    for (int k = 0; k < kReduceThreads / 32; k++) {
      r.v[0] += sm[0][k]; r.v[1] += sm[1][k]; r.v[2] += sm[2][k]; r.v[4] += sm[4][k];
      r.v[3] = fmax(r.v[3], sm[3][k]);
    }
    partials[blockIdx.x] = r;
  }
}

__global__ void k_nci_diag_final(const DiagOut *__restrict__ partials, int n, DiagOut *__restrict__ out) {
  if (blockIdx.x != 0) return;
  const int lane = threadIdx.x;
  double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int k = lane; k < n; k += 32) {
#pragma unroll
    for (int j = 0; j < 5; j++) a[j] = j == 3 ? fmax(a[j], partials[k].v[j]) : a[j] + partials[k].v[j];
  }
#pragma unroll
  for (int j = 0; j < 5; j++) a[j] = j == 3 ? warp_max(a[j]) : warp_sum(a[j]);
  if (lane == 0) {
    DiagOut r;
#pragma unroll
    for (int j = 0; j < 5; j++) r.v[j] = a[j];
    *out = r;
  }
}

cudaError_t launch_nci_diag(int dim, const KParams &P, const int32_t *phi, const float4 *frep, DiagOut *partials,
                            DiagOut *out, cudaStream_t s) {
  if (dim == 2)
    k_nci_diag_partial<2><<<kReduceBlocks, kReduceThreads, 0, s>>>(P, phi, frep, partials);
  else
    k_nci_diag_partial<3><<<kReduceBlocks, kReduceThreads, 0, s>>>(P, phi, frep, partials);
  k_nci_diag_final<<<1, 32, 0, s>>>(partials, kReduceBlocks, out);
  return cudaGetLastError();
}

// Normals n = grad(phi) / (|grad(phi)| + eps_n) (Eqs. 22, 57) of every cell.
template <int DIM>
__global__ void __launch_bounds__(kReduceThreads)
k_normals_all(const KParams P, const int32_t *__restrict__ phi, float4 *__restrict__ nrm) {
  using SL = typename StencilOf<DIM>::type;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += stride) {
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int i = 1; i < SL::Q; i++) {
      if (!positive<SL>(i)) continue;
      const int c0 = SL::c(i, 0), c1 = SL::c(i, 1), c2 = SL::c(i, 2);
      const long long ip = wrapn(x + c0, nx) + (long long)nx * (wrapn(y + c1, ny) + (long long)ny * wrapn(z + c2, nz));
      const long long im = wrapn(x - c0, nx) + (long long)nx * (wrapn(y - c1, ny) + (long long)ny * wrapn(z - c2, nz));
      const float d = SL::w(i) * dphi_of(phi[ip], phi[im]);
      g0 += c0 * d;
      g1 += c1 * d;
      g2 += c2 * d;
    }
    g0 *= 3.0f; g1 *= 3.0f; g2 *= 3.0f;
    const float inv = 1.0f / (sqrtf(g0 * g0 + g1 * g1 + g2 * g2) + P.eps_n);
    nrm[n] = make_float4(g0 * inv, g1 * inv, g2 * inv, 0.0f);
  }
}

// kappa = div n by the isotropic stencil (Eq. 22 on each component) at the band cells; a block
// histogram in shared memory flushed with integer atomics, and the count and sum per block.
template <int DIM>
__global__ void __launch_bounds__(kReduceThreads)
k_curv_partial(const KParams P, const int32_t *__restrict__ phi, const float4 *__restrict__ nrm, float kmin,
               float kmax, int nbins, unsigned long long *__restrict__ hist, double *__restrict__ partials) {
  using SL = typename StencilOf<DIM>::type;
  __shared__ unsigned int sh[kMaxCurvBins];
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) sh[k] = 0u;
  __syncthreads();
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const float scale = (float)nbins / (kmax - kmin);
  double cnt = 0.0, sum = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < P.N; n += stride) {
    if (!(q_gate_value(phi[n]) >= P.q_th)) continue;
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
    float k = 0.f;
#pragma unroll
    for (int i = 1; i < SL::Q; i++) {
      if (!positive<SL>(i)) continue;
      const int c0 = SL::c(i, 0), c1 = SL::c(i, 1), c2 = SL::c(i, 2);
      const long long ip = wrapn(x + c0, nx) + (long long)nx * (wrapn(y + c1, ny) + (long long)ny * wrapn(z + c2, nz));
      const long long im = wrapn(x - c0, nx) + (long long)nx * (wrapn(y - c1, ny) + (long long)ny * wrapn(z - c2, nz));
      const float4 a = nrm[ip], b = nrm[im];
      k += SL::w(i) * (c0 * (a.x - b.x) + c1 * (a.y - b.y) + c2 * (a.z - b.z));
    }
    k *= 3.0f;
    cnt += 1.0;
    sum += (double)k;
    if (k >= kmin && k < kmax) {
      int bin = (int)((k - kmin) * scale);
      bin = bin < nbins ? bin : nbins - 1;
      atomicAdd(&sh[bin], 1u);
    }
  }
  __shared__ double sm[2][kReduceThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  cnt = warp_sum(cnt);
  sum = warp_sum(sum);
  if (lane == 0) {
    sm[0][wid] = cnt;
    sm[1][wid] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double c = 0.0, t = 0.0;
    for (int w = 0; w < kReduceThreads / 32; w++) {
      c += sm[0][w];
      t += sm[1][w];
    }
    partials[2 * blockIdx.x] = c;
    partials[2 * blockIdx.x + 1] = t;
  }
  for (int k = threadIdx.x; k < nbins; k += blockDim.x)
    if (sh[k]) atomicAdd(&hist[k], (unsigned long long)sh[k]);
}

__global__ void k_curv_final(const double *__restrict__ partials, int n, double *__restrict__ out) {
  if (blockIdx.x != 0) return;
  double c = 0.0, t = 0.0;
  for (int k = threadIdx.x; k < n; k += 32) {
    c += partials[2 * k];
    t += partials[2 * k + 1];
  }
  c = warp_sum(c);
  t = warp_sum(t);
  if (threadIdx.x == 0) {
    out[0] = c;
    out[1] = t;
  }
}

cudaError_t launch_curvature(int dim, const KParams &P, const int32_t *phi, float4 *nrm, float kmin, float kmax,
                             int nbins, unsigned long long *hist, double *partials, double *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * nbins, s);
  if (e != cudaSuccess) return e;
  if (dim == 2) {
    k_normals_all<2><<<kReduceBlocks, kReduceThreads, 0, s>>>(P, phi, nrm);
    k_curv_partial<2><<<kReduceBlocks, kReduceThreads, 0, s>>>(P, phi, nrm, kmin, kmax, nbins, hist, partials);
  } else {
    k_normals_all<3><<<kReduceBlocks, kReduceThreads, 0, s>>>(P, phi, nrm);
    k_curv_partial<3><<<kReduceBlocks, kReduceThreads, 0, s>>>(P, phi, nrm, kmin, kmax, nbins, hist, partials);
  }
  k_curv_final<<<1, 32, 0, s>>>(partials, kReduceBlocks, out);
  return cudaGetLastError();
}

}  // namespace lbm
