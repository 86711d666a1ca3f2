// kernels_nci.cu -- near-contact interaction (Sec. 2.3): interfacial gate (Eqs. 58-59), bounded
// window pairing (Eqs. 60-65), closed-form proximity indicator and repulsive force (Eqs. 66-73).
//
// Passes over the tiles that hold an interfacial (gated) cell, as listed by the phase-field kernel
// of the previous step (or over every tile for the diagnostic read-back):
//   k_nci_normals3 / k_nci_normals2  the normal n = grad(phi) / (|grad(phi)| + eps_n) of every gated
//                  cell (Eq. 57, isotropic gradient of Eq. 22), computed once and stored as a float4;
//                  in 3D also zero force at every gated cell and the normal ranges of each 4x4x4 brick;
//   k_nci_prefilter (3D, sides multiples of 4) per listed tile, a lower bound of n(x).n(y) from the
//                  brick ranges; only tiles where the facing gate can hold go on to the scan;
//   k_nci_scan     per tile: phi and the gated normals of the tile + 3 halo staged in shared memory,
//                  the gated cells of the tile compacted into a list, then one warp per gated cell
//                  tests 32 window offsets per iteration in (|r|^2, canonical index) order and
//                  stops after the first shell holding an accepted candidate.
// Before scanning, a cell bounds n(x).n(y) from below by the component ranges [lo_a, hi_a] of the
// gated normals around it: sum_a min(n_a lo_a, n_a hi_a) <= n(x).n(y). A cell whose bound exceeds
// the facing threshold cannot have a candidate (Eq. 62) and skips the scan; this is exact (a
// rounding margin of 1e-5 is kept). The ranges are taken first over the whole halo box of the
// tile, and where that does not decide, over the cell's own 7^3 window: separable sliding min/max
// filters (z, then y, then x) of the three components, with non-gated cells as NaN (which fminf
// and fmaxf skip), kept as halves rounded outward (lo down, hi up) so the bound stays a lower
// bound. A curved interface of radius R turns its normal by about 5/R inside a window, so on
// isolated drops and bubbles only cells facing another interface within 3 cells are scanned.
// The force is written only at gated cells; the hydrodynamic kernel reads it exactly there (same
// gate function).
#include "launch.h"

namespace lbm {

template <int DIM> struct NciGeom {
  static constexpr int TX = NciTile<DIM>::X, TY = NciTile<DIM>::Y, TZ = NciTile<DIM>::Z;
  static constexpr int H = 3;  // window radius bound
  static constexpr int HX = TX + 2 * H, HY = TY + 2 * H, HZ = DIM == 3 ? TZ + 2 * H : 1;
  static constexpr int NB = HX * HY * HZ;
  static constexpr int NT = TX * TY * TZ, NW = NT / 32;
  static constexpr int NZR = HX * HY * TZ;  // z-filtered planes (3D)
  static constexpr int NYR = HX * TY * TZ;  // z- and y-filtered rows
  static constexpr size_t smem = sizeof(int32_t) * NB + sizeof(float) * 3 * NB + sizeof(int) * (NT + 1) +
                                 sizeof(float) * (6 * (NW + 1) + 1) + sizeof(long long) * (HY * HZ + 1) +
                                 sizeof(int) * HX + sizeof(__half) * 6 * ((DIM == 3 ? NZR : 0) + NYR) +
                                 sizeof(float) * NB;
};

// The eight windows [o, o + 6], o = 0..7, of fourteen values: the suffix extremes of [0, 6] and the
// prefix extremes of [7, 13] (van Herk / Gil-Werman), 18 operations instead of 48.
template <bool MAX>
__device__ __forceinline__ void win7x8(const float *v, float *out) {
  auto op = [](float a, float b) { return MAX ? fmaxf(a, b) : fminf(a, b); };
  float suf[7], pre[7];
  suf[6] = v[6];
#pragma unroll
  for (int i = 5; i >= 0; i--) suf[i] = op(v[i], suf[i + 1]);
  pre[0] = v[7];
#pragma unroll
  for (int j = 1; j < 7; j++) pre[j] = op(pre[j - 1], v[7 + j]);
  out[0] = suf[0];
#pragma unroll
  for (int o = 1; o < 7; o++) out[o] = op(suf[o], pre[o - 1]);
  out[7] = pre[6];
}

// The four windows [o, o + 6], o = 0..3, of ten values share the core [3, 6] and the pairs (1, 2)
// and (7, 8): 13 min (or max) operations instead of 24.
template <bool MAX>
__device__ __forceinline__ void win7x4(const float *v, float *out) {
  auto op = [](float a, float b) { return MAX ? fmaxf(a, b) : fminf(a, b); };
  const float core = op(op(v[3], v[4]), op(v[5], v[6]));
  const float p12 = op(v[1], v[2]), q78 = op(v[7], v[8]);
  out[0] = op(core, op(v[0], p12));
  out[1] = op(core, op(p12, v[7]));
  out[2] = op(core, op(v[2], q78));
  out[3] = op(core, op(q78, v[9]));
}

template <int DIM>
__device__ __forceinline__ void tile_of(int tile, int gtx, int gty, int &bx, int &by, int &bz) {
  bx = tile % gtx;
  by = (tile / gtx) % gty;
  bz = tile / (gtx * gty);
}

// Normals of the gated cells of the listed tiles (or of every tile when tiles == nullptr), 2D.
__global__ void __launch_bounds__(NciGeom<2>::NT)
k_nci_normals2(const KParams P, const int32_t *__restrict__ phi, float4 *__restrict__ nrm,
               const int *__restrict__ tiles, const int *__restrict__ ntiles, int total, int gtx, int gty,
               int *__restrict__ reset_other) {
  pdl_enter();
  if (reset_other && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) *reset_other = 0;
  using G = NciGeom<2>;
  using SL = StencilOf<2>::type;
  const int n = tiles ? *ntiles : total;
  const int nx = P.nx, ny = P.ny;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    int bx, by, bz;
    tile_of<2>(tiles ? tiles[t] : t, gtx, gty, bx, by, bz);
    const int x = bx * G::TX + threadIdx.x, y = by * G::TY + threadIdx.y;
    if (x >= nx || y >= ny) continue;
    const int X[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
    const int Y[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
    const long long idx = (long long)x + (long long)nx * y;
    if (!(q_gate_value(phi[idx]) >= P.q_th)) continue;
    float g0 = 0.f, g1 = 0.f;
#pragma unroll
    for (int i = 1; i < SL::Q; i++) {
      if (!positive<SL>(i)) continue;
      const int c0 = SL::c(i, 0), c1 = SL::c(i, 1);
      const float d = SL::w(i) * dphi_of(__ldg(phi + X[1 + c0] + (long long)nx * Y[1 + c1]),
                                         __ldg(phi + X[1 - c0] + (long long)nx * Y[1 - c1]));
      g0 += c0 * d;
      g1 += c1 * d;
    }
    g0 *= 3.0f; g1 *= 3.0f;
    const float inv = 1.0f / (sqrtf(g0 * g0 + g1 * g1) + P.eps_n);
    nrm[idx] = make_float4(g0 * inv, g1 * inv, 0.0f, 0.0f);
  }
}

// Normals of the gated cells of the listed tiles (or of every tile when tiles == nullptr), 3D.
// One 128-thread block per half tile (32 x 4 x 4 cells, eight 4x4x4 bricks side by side in x):
// phi of the half tile + 1 halo (34 x 6 x 6) is staged in shared memory, then warp w takes the 4
// rows of plane z0 + w. The gradient is the isotropic D3Q27 one of Eq. 22, summed over the 13
// links in the same order as everywhere else.
// With the prefilter (listed tiles): every gated cell's force is set to zero here (the scan
// overwrites it where a partner is found), the tile's flag is set, and the component ranges of
// the gated normals of each brick are stored (empty bricks as [+inf, -inf]).
constexpr int kNrmThreads = 128;
struct NrmBox {
  static constexpr int X = 34, Y = 6, Z = 6, ROWS = Y * Z;  // warp w stages rows w, w + 4, ...
};

__global__ void __launch_bounds__(kNrmThreads)
k_nci_normals3(const KParams P, const int32_t *__restrict__ phi, float4 *__restrict__ nrm, float4 *__restrict__ frep,
               const int *__restrict__ tiles, const int *__restrict__ ntiles, int total, int gtx, int gty,
               const NciAux aux, int *__restrict__ reset_other) {
  pdl_enter();
  if (reset_other && blockIdx.x == 0 && threadIdx.x == 0) *reset_other = 0;
  using G = NciGeom<3>;
  using SL = StencilOf<3>::type;
  using B = NrmBox;
  static_assert(G::TX == 32 && G::TY == 8 && G::TZ == 4, "two 32 x 4 x 4 halves per tile");
  __shared__ int32_t s_box[B::ROWS * B::X];
  __shared__ float s_part[4][8][6];  // [warp][brick][lo0..hi2]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool bricks = aux.bricks != nullptr;  // uniform over the grid
  if (bricks && blockIdx.x == 0 && threadIdx.x == 0) *aux.nscan = 0;
  const int n = tiles ? *ntiles : total;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const float inf = __int_as_float(0x7f800000);
  for (int item = blockIdx.x; item < 2 * n; item += gridDim.x) {
    const int tile = tiles ? tiles[item >> 1] : (item >> 1);
    const int half = item & 1;
    int bx, by, bz;
    tile_of<3>(tile, gtx, gty, bx, by, bz);
    if (bricks && half == 0 && threadIdx.x == 0) aux.flags[tile] = 1;
    const int x0 = bx * G::TX, y0 = by * G::TY + 4 * half, z0 = bz * G::TZ;
    {
      const int xa = wrapn(x0 - 1 + lane, nx), xb = wrapn(x0 + 31 + (lane & 1), nx);
      int32_t va[9], vb[9];
#pragma unroll
      for (int j = 0; j < 9; j++) {
        const int r = warp + 4 * j, ry = r % B::Y, rz = r / B::Y;
        const long long row = (long long)nx * (wrapn(y0 - 1 + ry, ny) + (long long)ny * wrapn(z0 - 1 + rz, nz));
        va[j] = phi[row + xa];
        if (lane < 2) vb[j] = phi[row + xb];
      }
#pragma unroll
      for (int j = 0; j < 9; j++) {
        const int r = warp + 4 * j;
        s_box[r * B::X + lane] = va[j];
        if (lane < 2) s_box[r * B::X + 32 + lane] = vb[j];
      }
    }
    __syncthreads();
    const int x = x0 + lane, z = z0 + warp;
    const bool xin = x < nx && z < nz;
    float lo0 = inf, lo1 = inf, lo2 = inf, hi0 = -inf, hi1 = -inf, hi2 = -inf;
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const int y = y0 + r;
      const int o = ((warp + 1) * B::Y + r + 1) * B::X + lane + 1;
      if (!(xin && y < ny && q_gate_value(s_box[o]) >= P.q_th)) continue;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
      for (int i = 1; i < SL::Q; i++) {
        if (!positive<SL>(i)) continue;
        const int c0 = SL::c(i, 0), c1 = SL::c(i, 1), c2 = SL::c(i, 2);
        const int off = c0 + B::X * (c1 + B::Y * c2);
        const float d = SL::w(i) * dphi_of(s_box[o + off], s_box[o - off]);
        g0 += c0 * d;
        g1 += c1 * d;
        g2 += c2 * d;
      }
      g0 *= 3.0f; g1 *= 3.0f; g2 *= 3.0f;
      const float inv = 1.0f / (sqrtf(g0 * g0 + g1 * g1 + g2 * g2) + P.eps_n);
      g0 *= inv; g1 *= inv; g2 *= inv;
      const long long idx = (long long)x + (long long)nx * (y + (long long)ny * z);
      nrm[idx] = make_float4(g0, g1, g2, 0.0f);
      if (bricks) {
        frep[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
        lo0 = fminf(lo0, g0); lo1 = fminf(lo1, g1); lo2 = fminf(lo2, g2);
        hi0 = fmaxf(hi0, g0); hi1 = fmaxf(hi1, g1); hi2 = fmaxf(hi2, g2);
      }
    }
    if (bricks) {  // lanes 4k..4k+3 of each warp share brick k; the four planes meet in shared memory
#pragma unroll
      for (int sh = 1; sh <= 2; sh <<= 1) {
        lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, sh));
        lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, sh));
        lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, sh));
        hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, sh));
        hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, sh));
        hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, sh));
      }
      if ((lane & 3) == 0) {
        float *sp = s_part[warp][lane >> 2];
        sp[0] = lo0; sp[1] = lo1; sp[2] = lo2; sp[3] = hi0; sp[4] = hi1; sp[5] = hi2;
      }
    }
    __syncthreads();  // s_part complete; s_box and s_part are free for the next item after this
    if (bricks) {
      const int k = threadIdx.x;
      const int gbx = 8 * bx + k, gby = 2 * by + half;
      if (k < 8 && gbx < (nx >> 2) && gby < (ny >> 2)) {
        float v[6];
#pragma unroll
        for (int c = 0; c < 6; c++) {
          v[c] = s_part[0][k][c];
#pragma unroll
          for (int w = 1; w < 4; w++) v[c] = c < 3 ? fminf(v[c], s_part[w][k][c]) : fmaxf(v[c], s_part[w][k][c]);
        }
        const auto h = [](__half q) { return (unsigned)__half_as_ushort(q); };
        uint4 o;
        o.x = h(__float2half_rd(v[0])) | (h(__float2half_rd(v[1])) << 16);
        o.y = h(__float2half_rd(v[2]));
        o.z = h(__float2half_ru(v[3])) | (h(__float2half_ru(v[4])) << 16);
        o.w = h(__float2half_ru(v[5]));
        aux.bricks[(long long)gbx + (long long)(nx >> 2) * (gby + (long long)(ny >> 2) * bz)] = o;
      }
    }
  }
}

// One 128-thread block per listed tile (3D). The tile's sixteen bricks are tested against the
// union of the normal ranges of their 27 neighbouring bricks, a 10x4x3 box of bricks; a brick of a
// tile that is not listed holds no gated cell and counts as empty. Every window offset of the scan
// (each component |r_a| <= 3) stays inside those 27 bricks, so for a cell x of a brick with ranges
// [lo, hi] and every gated y in its window,
//   n(x).n(y) >= sum_a min(lo_a L_a, lo_a H_a, hi_a L_a, hi_a H_a),
// [L, H] being the union (the product is bilinear, so its minimum over the two boxes is at a
// corner). Where that bound exceeds cos_opp + 1e-5 for all sixteen bricks, no cell of the tile
// can meet the facing gate (Eq. 62) and the tile keeps the zero force written by the normals
// pass; otherwise the tile goes to the scan list.
__global__ void __launch_bounds__(128)
k_nci_prefilter(const KParams P, const uint4 *__restrict__ bricks, const unsigned char *__restrict__ flags,
                const int *__restrict__ tiles, const int *__restrict__ ntiles, int *__restrict__ scan_tiles,
                int *__restrict__ nscan, int gtx, int gty) {
  pdl_enter();
  constexpr int RX = 10, RY = 4, RZ = 3, NR = RX * RY * RZ;
  __shared__ float s_r[6][NR];
  __shared__ float s_b[48];
  const int tid = threadIdx.x;
  const int n = *ntiles;
  const int nbx = P.nx >> 2, nby = P.ny >> 2, nbz = P.nz >> 2;
  const float inf = __int_as_float(0x7f800000);
  const float thr = P.cos_opp + 1e-5f;
  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    const int tile = tiles[t];
    int bx, by, bz;
    tile_of<3>(tile, gtx, gty, bx, by, bz);
    if (tid < NR) {
      const int rx = tid % RX, ry = (tid / RX) % RY, rz = tid / (RX * RY);
      const int gbx = wrapn(8 * bx - 1 + rx, nbx), gby = wrapn(2 * by - 1 + ry, nby), gbz = wrapn(bz - 1 + rz, nbz);
      float v[6] = {inf, inf, inf, -inf, -inf, -inf};
      if (flags[(gbx >> 3) + gtx * ((gby >> 1) + gty * gbz)]) {
        const uint4 w = bricks[(long long)gbx + (long long)nbx * (gby + (long long)nby * gbz)];
        v[0] = __half2float(__ushort_as_half((unsigned short)(w.x & 0xffffu)));
        v[1] = __half2float(__ushort_as_half((unsigned short)(w.x >> 16)));
        v[2] = __half2float(__ushort_as_half((unsigned short)(w.y & 0xffffu)));
        v[3] = __half2float(__ushort_as_half((unsigned short)(w.z & 0xffffu)));
        v[4] = __half2float(__ushort_as_half((unsigned short)(w.z >> 16)));
        v[5] = __half2float(__ushort_as_half((unsigned short)(w.w & 0xffffu)));
      }
#pragma unroll
      for (int c = 0; c < 6; c++) s_r[c][tid] = v[c];
    }
    __syncthreads();
    if (tid < 48) {
      const int b = tid & 15, a = tid >> 4;
      const int cx = b & 7, cy = b >> 3;
      float L = inf, H = -inf;
#pragma unroll
      for (int dz = 0; dz < 3; dz++)
#pragma unroll
        for (int dy = 0; dy < 3; dy++)
#pragma unroll
          for (int dx = 0; dx < 3; dx++) {
            const int r = (cx + dx) + RX * ((cy + dy) + RY * dz);
            L = fminf(L, s_r[a][r]);
            H = fmaxf(H, s_r[3 + a][r]);
          }
      const int rc = (cx + 1) + RX * ((cy + 1) + RY);
      const float lo = s_r[a][rc], hi = s_r[3 + a][rc];
      s_b[tid] = fminf(fminf(lo * L, lo * H), fminf(hi * L, hi * H));
    }
    __syncthreads();
    bool need = false;
    if (tid < 16) {
      const int cx = tid & 7, cy = tid >> 3;
      const int rc = (cx + 1) + RX * ((cy + 1) + RY);
      const bool has = 8 * bx + cx < nbx && 2 * by + cy < nby && s_r[0][rc] <= s_r[3][rc];
      need = has && s_b[tid] + s_b[16 + tid] + s_b[32 + tid] <= thr;
    }
    if (__syncthreads_or(need) && tid == 0) scan_tiles[atomicAdd(nscan, 1)] = tile;
  }
}

template <int DIM>
__global__ void __launch_bounds__(NciGeom<DIM>::NT, NciGeom<DIM>::NT >= 1024 ? 1 : 2)
k_nci_scan(const KParams P, const NciTable T, const int32_t *__restrict__ phi, const float4 *__restrict__ nrm,
           float4 *__restrict__ frep, int32_t *__restrict__ partner, int debug, const int *__restrict__ tiles,
           const int *__restrict__ ntiles, int total, int gtx, int gty, unsigned char *__restrict__ flags,
           const int *__restrict__ listed, const int *__restrict__ nlisted) {
  pdl_enter();
  using G = NciGeom<DIM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t *s_phi = reinterpret_cast<int32_t *>(smem_raw);
  float *s_n = reinterpret_cast<float *>(s_phi + G::NB);
  int *s_list = reinterpret_cast<int *>(s_n + 3 * G::NB);
  int *s_count = s_list + G::NT;
  float *s_rng = reinterpret_cast<float *>(s_count + 1);  // [NW + 1][6]
  long long *s_row = reinterpret_cast<long long *>(s_rng + 6 * (G::NW + 1) + 1);  // [HY * HZ], 8-aligned
  int *s_col = reinterpret_cast<int *>(s_row + G::HY * G::HZ);                   // [HX]
  __half *s_yr = reinterpret_cast<__half *>(s_col + G::HX);                        // [6][NYR]
  __half *s_zr = s_yr + 6 * G::NYR;                                                // [6][NZR] (3D)
  // q = phi (1 - phi) of the staged box (phi clamped, binary32 as the gate takes it), computed once
  float *s_q = reinterpret_cast<float *>(s_zr + 6 * (DIM == 3 ? G::NZR : 0));        // [NB]

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + G::TX * (ty + G::TY * tz), lane = tid & 31, warp = tid >> 5;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int n = tiles ? *ntiles : total;
  if (flags) {  // the prefilter has read the flags of this step's listed tiles: clear them
    const int m = *nlisted;
    for (int i = blockIdx.x * G::NT + tid; i < m; i += gridDim.x * G::NT) flags[listed[i]] = 0;
  }

  for (int t = blockIdx.x; t < n; t += gridDim.x) {
    int bx, by, bz;
    tile_of<DIM>(tiles ? tiles[t] : t, gtx, gty, bx, by, bz);
    const int x0 = bx * G::TX, y0 = by * G::TY, z0 = bz * G::TZ;
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    const bool inb = x < nx && y < ny && z < nz;
    const long long idx = inb ? (long long)x + (long long)nx * (y + (long long)ny * z) : 0;
    bool gated = false;
    if (!tiles) {  // every tile is visited: skip those without an interfacial cell
      gated = inb && (q_gate_value(phi[idx]) >= P.q_th);
      if (!__syncthreads_or(gated)) {
        if (debug && inb) {
          frep[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (partner) partner[3 * idx] = partner[3 * idx + 1] = partner[3 * idx + 2] = INT32_MIN;
        }
        continue;  // uniform over the block
      }
    }

    // Stage phi and the gated normals (written once per step by k_nci_normals) of the tile + 3
    // halo, row by row (rows of HX = TX + 6 values): every row's phi loads are issued before any is
    // stored; each warp then gates its own rows and loads the normals of their gated cells.
    // Non-gated cells hold NaN normals, which fminf / fmaxf skip.
    float lo0 = 1e30f, lo1 = 1e30f, lo2 = 1e30f, hi0 = -1e30f, hi1 = -1e30f, hi2 = -1e30f;
    {
      constexpr int NROWS = G::HY * G::HZ, RPW = (NROWS + G::NW - 1) / G::NW;
      const int xl = wrapn(x0 - G::H + tx, nx);
      const int xr = wrapn(x0 - G::H + 32 + (tx & 7), nx);
      const bool xtra = lane < G::HX - 32;
      int32_t va[RPW], vb[RPW];
#pragma unroll
      for (int h = 0; h < RPW; h++) {
        const int r = warp + h * G::NW;
        if (r < NROWS) {
          const int ry = r % G::HY, rz = r / G::HY;
          const long long row = (long long)nx * (wrapn(y0 + ry - G::H, ny) +
                                                 (long long)ny * (DIM == 3 ? wrapn(z0 + rz - G::H, nz) : 0));
          if (lane == 0) s_row[r] = row;
          va[h] = phi[row + xl];
          if (xtra) vb[h] = phi[row + xr];
        }
      }
#pragma unroll
      for (int h = 0; h < RPW; h++) {
        const int r = warp + h * G::NW;
        if (r < NROWS) {
          s_phi[r * G::HX + lane] = va[h];
          s_q[r * G::HX + lane] = q_gate_value(va[h]);
          if (xtra) {
            s_phi[r * G::HX + 32 + lane] = vb[h];
            s_q[r * G::HX + 32 + lane] = q_gate_value(vb[h]);
          }
        }
      }
      __syncwarp();  // this warp's rows of s_phi and s_row
      const float qnan = __int_as_float(0x7fffffff);
#pragma unroll 2
      for (int h = 0; h < RPW; h++) {
        const int r = warp + h * G::NW;
        if (r >= NROWS) break;
        const int b = r * G::HX + lane;
        const bool ga = s_q[b] >= P.q_th;
        const bool gb = xtra && s_q[b + 32] >= P.q_th;
        float4 na, nb;
        if (ga || gb) {
          const long long row = s_row[r];
          if (ga) na = __ldg(nrm + row + xl);
          if (gb) nb = __ldg(nrm + row + xr);
        }
        if (ga) {
          s_n[b] = na.x; s_n[G::NB + b] = na.y; s_n[2 * G::NB + b] = na.z;
          lo0 = fminf(lo0, na.x); lo1 = fminf(lo1, na.y); lo2 = fminf(lo2, na.z);
          hi0 = fmaxf(hi0, na.x); hi1 = fmaxf(hi1, na.y); hi2 = fmaxf(hi2, na.z);
        } else {
          s_n[b] = s_n[G::NB + b] = s_n[2 * G::NB + b] = qnan;
        }
        if (xtra) {
          if (gb) {
            s_n[b + 32] = nb.x; s_n[G::NB + b + 32] = nb.y; s_n[2 * G::NB + b + 32] = nb.z;
            lo0 = fminf(lo0, nb.x); lo1 = fminf(lo1, nb.y); lo2 = fminf(lo2, nb.z);
            hi0 = fmaxf(hi0, nb.x); hi1 = fmaxf(hi1, nb.y); hi2 = fmaxf(hi2, nb.z);
          } else {
            s_n[b + 32] = s_n[G::NB + b + 32] = s_n[2 * G::NB + b + 32] = qnan;
          }
        }
      }
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
      lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, sh));
      lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, sh));
      lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, sh));
      hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, sh));
      hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, sh));
      hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, sh));
    }
    if (lane == 0) {
      float *rw = s_rng + 6 * warp;
      rw[0] = lo0; rw[1] = lo1; rw[2] = lo2; rw[3] = hi0; rw[4] = hi1; rw[5] = hi2;
    }
    if (tid == 0) *s_count = 0;
    __syncthreads();
    if (tid < 6) {
      float a = s_rng[tid];
      for (int w = 1; w < G::NW; w++) a = tid < 3 ? fminf(a, s_rng[6 * w + tid]) : fmaxf(a, s_rng[6 * w + tid]);
      s_rng[6 * G::NW + tid] = a;
    }
    __syncthreads();
    const float rlo0 = s_rng[6 * G::NW], rlo1 = s_rng[6 * G::NW + 1], rlo2 = s_rng[6 * G::NW + 2];
    const float rhi0 = s_rng[6 * G::NW + 3], rhi1 = s_rng[6 * G::NW + 4], rhi2 = s_rng[6 * G::NW + 5];
    const float thr = P.cos_opp + 1e-5f;
    const int ob0 = (DIM == 3 ? (tz + G::H) * G::HX * G::HY : 0) + (ty + G::H) * G::HX + tx + G::H;
    if (tiles) gated = inb && s_q[ob0] >= P.q_th;
    bool scan = false;
    if (gated) {
      const float n0 = s_n[ob0], n1 = s_n[G::NB + ob0], n2 = s_n[2 * G::NB + ob0];
      scan = fminf(n0 * rlo0, n0 * rhi0) + fminf(n1 * rlo1, n1 * rhi1) + fminf(n2 * rlo2, n2 * rhi2) <= thr;
    }
    if (__syncthreads_or(scan)) {
      // window ranges: z pass (3D) over the box columns, y pass, then x per cell
      if constexpr (DIM == 3) {
        for (int col = tid; col < G::HX * G::HY; col += G::NT) {
#pragma unroll
          for (int a = 0; a < 3; a++) {
            float v[G::HZ];
#pragma unroll
            for (int k = 0; k < G::HZ; k++) v[k] = s_n[a * G::NB + k * G::HX * G::HY + col];
            static_assert(G::HZ == 10 && G::TZ == 4, "window filter of four outputs over ten planes");
            float lo[4], hi[4];
            win7x4<false>(v, lo);
            win7x4<true>(v, hi);
#pragma unroll
            for (int o = 0; o < G::TZ; o++) {
              s_zr[(2 * a) * G::NZR + o * G::HX * G::HY + col] = __float2half_rd(lo[o]);
              s_zr[(2 * a + 1) * G::NZR + o * G::HX * G::HY + col] = __float2half_ru(hi[o]);
            }
          }
        }
        __syncthreads();
      }
      for (int col = tid; col < G::HX * G::TZ; col += G::NT) {
        const int cx = col % G::HX, cz = col / G::HX;
#pragma unroll
        for (int c = 0; c < 6; c++) {
          float v[G::HY];
#pragma unroll
          for (int k = 0; k < G::HY; k++) {
            if constexpr (DIM == 3) {
              v[k] = __half2float(s_zr[c * G::NZR + (cz * G::HY + k) * G::HX + cx]);
            } else {
              v[k] = s_n[(c >> 1) * G::NB + k * G::HX + cx];
            }
          }
          if constexpr (G::HY == 10 && G::TY == 4) {
            float r[4];
            if (c & 1) win7x4<true>(v, r); else win7x4<false>(v, r);
#pragma unroll
            for (int o = 0; o < G::TY; o++)
              s_yr[c * G::NYR + (cz * G::TY + o) * G::HX + cx] = (c & 1) ? __float2half_ru(r[o]) : __float2half_rd(r[o]);
          } else if constexpr (G::HY == 14 && G::TY == 8) {
            float r[8];
            if (c & 1) win7x8<true>(v, r); else win7x8<false>(v, r);
#pragma unroll
            for (int o = 0; o < G::TY; o++)
              s_yr[c * G::NYR + (cz * G::TY + o) * G::HX + cx] = (c & 1) ? __float2half_ru(r[o]) : __float2half_rd(r[o]);
          } else {
#pragma unroll
            for (int o = 0; o < G::TY; o++) {
              float r = v[o];
#pragma unroll
              for (int k = 1; k <= 2 * G::H; k++) r = (c & 1) ? fmaxf(r, v[o + k]) : fminf(r, v[o + k]);
              s_yr[c * G::NYR + (cz * G::TY + o) * G::HX + cx] = (c & 1) ? __float2half_ru(r) : __float2half_rd(r);
            }
          }
        }
      }
      __syncthreads();
      if (scan) {
        const __half *row = s_yr + (tz * G::TY + ty) * G::HX + tx;
        float b = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; a++) {
          float lo = __half2float(row[(2 * a) * G::NYR]), hi = __half2float(row[(2 * a + 1) * G::NYR]);
#pragma unroll
          for (int k = 1; k <= 2 * G::H; k++) {
            lo = fminf(lo, __half2float(row[(2 * a) * G::NYR + k]));
            hi = fmaxf(hi, __half2float(row[(2 * a + 1) * G::NYR + k]));
          }
          const float na = s_n[a * G::NB + ob0];
          b += fminf(na * lo, na * hi);
        }
        scan = b <= thr;
      }
    }
    if (gated && !scan) {  // no candidate can face this cell: no force
      frep[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (partner) partner[3 * idx] = partner[3 * idx + 1] = partner[3 * idx + 2] = INT32_MIN;
    }
    {  // compact the cells to scan
      const unsigned m = __ballot_sync(0xffffffffu, scan);
      int base = 0;
      if (lane == 0 && m) base = atomicAdd(s_count, __popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (scan) s_list[base + __popc(m & ((1u << lane) - 1u))] = tid;
    }
    if (debug && inb && !gated) {
      frep[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (partner) partner[3 * idx] = partner[3 * idx + 1] = partner[3 * idx + 2] = INT32_MIN;
    }
    __syncthreads();

    // one warp per gated cell; candidate criteria Eqs. 59, 61, 62; the winner is the nearest
    // accepted candidate, then the largest facing score, then the first in table order (the
    // packed key orders exactly that way)
    const int ncell = *s_count;
    for (int k = warp; k < ncell; k += G::NW) {
      const int c = s_list[k];
      const int cx = c % G::TX, cy = (c / G::TX) % G::TY, cz = c / (G::TX * G::TY);
      const int ob = (DIM == 3 ? (cz + G::H) * G::HX * G::HY : 0) + (cy + G::H) * G::HX + cx + G::H;
      const int32_t vx = s_phi[ob];
      const float qxc = s_q[ob];
      const float n0 = s_n[ob], n1 = s_n[G::NB + ob], n2 = s_n[2 * G::NB + ob];
      unsigned long long best = ~0ull;
      {
        const float sim = __fmul_rn(P.eta, fmaxf(qxc, P.eps_q));
        for (int j0 = 0; j0 < T.count; j0 += 32) {
          // stop once a candidate is held and this chunk starts beyond its shell
          if (best != ~0ull && (int)T.o[j0].d2 > (int)(best >> 40)) break;
          const int j = j0 + lane;
          unsigned long long key = ~0ull;
          if (j < T.count) {
            const NciOffset o = T.o[j];
            const int yb = ob + o.dx + G::HX * (o.dy + G::HY * o.dz);
            const float qy = s_q[yb];
            if (qy >= P.q_th && fabsf(__fsub_rn(qy, qxc)) <= sim) {
              const float dot = __fadd_rn(__fadd_rn(__fmul_rn(n0, s_n[yb]), __fmul_rn(n1, s_n[G::NB + yb])),
                                          __fmul_rn(n2, s_n[2 * G::NB + yb]));
              if (dot <= P.cos_opp) {
                const float ff = fmaxf(-dot, 0.0f);
                key = ((unsigned long long)o.d2 << 40) |
                      ((unsigned long long)(0x7fffffffu - __float_as_uint(ff)) << 9) | (unsigned long long)j;
              }
            }
          }
          if (__any_sync(0xffffffffu, key != ~0ull)) {
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1) {
              const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, sh);
              key = other < key ? other : key;
            }
            best = key < best ? key : best;
          }
        }
      }
      if (lane != 0) continue;
      const long long gidx = (long long)(x0 + cx) + (long long)nx * ((y0 + cy) + (long long)ny * (z0 + cz));
      float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
      if (best != ~0ull) {
        const int bj = (int)(best & 511ull);
        const NciOffset o = T.o[bj];
        const float ff = __uint_as_float(0x7fffffffu - (unsigned)((best >> 9) & 0x7fffffffull));
        const int yb = ob + o.dx + G::HX * (o.dy + G::HY * o.dz);
        const int32_t vy = s_phi[yb];
        const float m0 = s_n[yb], m1 = s_n[G::NB + yb], m2 = s_n[2 * G::NB + yb];
        const float qy = s_q[yb];
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
        const float tt = h / P.h0;
        const float tp = (P.p == 4.0f) ? (tt * tt) * (tt * tt) : powf(tt, P.p);
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
    __syncthreads();  // the next tile reuses the shared buffers
  }
}

template <int DIM>
static cudaError_t nci_attr() {
  using G = NciGeom<DIM>;
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_nci_scan<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int DIM>
static cudaError_t launch_nci_dim(const KParams &P, const NciTable &T, const int32_t *phi, float4 *nrm, float4 *frep,
                                  int32_t *partner, int debug, const int *tiles, const int *ntiles, int list_blocks,
                                  cudaStream_t s, const NciAux *aux, int *reset_other) {
  using G = NciGeom<DIM>;
  cudaError_t e = nci_attr<DIM>();
  if (e != cudaSuccess) return e;
  const int gtx = (P.nx + G::TX - 1) / G::TX, gty = (P.ny + G::TY - 1) / G::TY, gtz = (P.nz + G::TZ - 1) / G::TZ;
  const int total = gtx * gty * gtz;
  // resident blocks walk the list; a small grid has fewer tiles than that
  const int blocks = tiles ? (total < list_blocks ? total : list_blocks) : (total < list_blocks * 4 ? total : list_blocks * 4);
  dim3 block(G::TX, G::TY, G::TZ);
  const bool pre = DIM == 3 && aux && tiles && aux->bricks && nci_aux_applies(DIM, P);
  const NciAux none{};
  if constexpr (DIM == 2) {
    cudaError_t e2 = launch_pdl(k_nci_normals2, dim3(blocks), block, 0, s, P, phi, nrm, tiles, ntiles, total, gtx, gty,
                                tiles ? reset_other : nullptr);
    if (e2 != cudaSuccess) return e2;
  } else {
    // one block per half tile, at most 16 blocks per resident scan block (grid-stride beyond)
    const int nb = 2 * total < 16 * list_blocks ? 2 * total : 16 * list_blocks;
    cudaError_t e3 = launch_pdl(k_nci_normals3, dim3(nb), dim3(kNrmThreads), 0, s, P, phi, nrm, frep, tiles, ntiles, total,
                                gtx, gty, pre ? *aux : none, tiles ? reset_other : nullptr);
    if (e3 != cudaSuccess) return e3;
  }
  if (!pre) {
    return launch_pdl(k_nci_scan<DIM>, dim3(blocks), block, G::smem, s, P, T, phi, nrm, frep, partner, debug, tiles,
                      ntiles, total, gtx, gty, nullptr, nullptr, nullptr);
  }
  e = launch_pdl(k_nci_prefilter, dim3(total < 16 * list_blocks ? total : 16 * list_blocks), dim3(128), 0, s, P,
                 (const uint4 *)aux->bricks,
                 (const unsigned char *)aux->flags, tiles, ntiles, aux->scan_tiles, aux->nscan, gtx, gty);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_nci_scan<DIM>, dim3(blocks), block, G::smem, s, P, T, phi, nrm, frep, partner, debug,
                    (const int *)aux->scan_tiles, (const int *)aux->nscan, total, gtx, gty, aux->flags, tiles, ntiles);
}

cudaError_t launch_nci(int dim, const KParams &P, const NciTable &T, const int32_t *phi, float4 *nrm, float4 *frep,
                       int32_t *partner, int debug, const int *tiles, const int *ntiles, int list_blocks,
                       cudaStream_t s, const NciAux *aux, int *reset_other) {
  return dim == 2 ? launch_nci_dim<2>(P, T, phi, nrm, frep, partner, debug, tiles, ntiles, list_blocks, s, aux,
                                      reset_other)
                  : launch_nci_dim<3>(P, T, phi, nrm, frep, partner, debug, tiles, ntiles, list_blocks, s, aux,
                                      reset_other);
}

bool nci_aux_applies(int dim, const KParams &P) {
  return dim == 3 && P.nx % 4 == 0 && P.ny % 4 == 0 && P.nz % 4 == 0;
}

size_t nci_brick_count(const KParams &P) { return (size_t)(P.nx / 4) * (size_t)(P.ny / 4) * (size_t)(P.nz / 4); }

int nci_list_blocks(int dim) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dim == 2) {
    if (nci_attr<2>() != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_nci_scan<2>, NciGeom<2>::NT, NciGeom<2>::smem);
  } else {
    if (nci_attr<3>() != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_nci_scan<3>, NciGeom<3>::NT, NciGeom<3>::smem);
  }
  return sms * (per > 0 ? per : 1);
}

}  // namespace lbm
