// launch.h -- host-side launchers of the liblbm kernels (internal to the library).
#pragma once

#include <utility>

#include "lbm_device.cuh"

namespace lbm {

// Launches a step kernel with programmatic stream serialization (see pdl_enter).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Window offsets of the near-contact search, sorted by (|r|^2, canonical index), passed by value.
struct NciTable {
  NciOffset o[kMaxOffsets];
  int count;
};

// Kernel modes of the hydrodynamic kernel.
enum HydroMode { kStep = 0, kMoments = 1 };

// Buffers of the near-contact prefilter (3D grids whose sides are multiples of 4): the component
// ranges of the gated normals of every 4x4x4 brick, as halves lo0 lo1 lo2 - hi0 hi1 hi2 - (lo
// rounded down, hi up); a flag per tile, set while the tile is listed for the current phi (zero
// between steps); the listed tiles that may hold a facing pair, and their count.
struct NciAux {
  uint4 *bricks = nullptr;
  unsigned char *flags = nullptr;
  int *scan_tiles = nullptr;
  int *nscan = nullptr;
};
bool nci_aux_applies(int dim, const KParams &P);
size_t nci_brick_count(const KParams &P);

// Normals of the gated cells into nrm, then the window scan writing frep at gated cells.
// tiles == nullptr: every tile (debug = 1 also writes zero force / no partner at every cell);
// otherwise only the ntiles listed tiles, walked by list_blocks resident blocks. With aux (listed
// tiles only), the normals pass also writes zero force at every gated cell and the brick ranges,
// a prefilter keeps the tiles whose bricks may face another interface, and only those are scanned.
// reset_other (listed tiles, may be null): the count of the other phi buffer's list, whose tiles
// were consumed by the previous step; the normals pass sets it to zero, so that the phase pass of
// this step starts that buffer's list empty.
cudaError_t launch_nci(int dim, const KParams &P, const NciTable &T, const int32_t *phi, float4 *nrm, float4 *frep,
                       int32_t *partner, int debug, const int *tiles, const int *ntiles, int list_blocks,
                       cudaStream_t s, const NciAux *aux = nullptr, int *reset_other = nullptr);
int nci_list_blocks(int dim);
cudaError_t phase_prepare(int dim);

// src/dst are population buffers of the store type; MODE kStep writes dst and u, kMoments writes
// u and pstar only.
cudaError_t launch_hydro(int Q, int store, int mode, const KParams &P, const void *src, void *dst,
                         const int32_t *phi, const float4 *frep, float *u, float *pstar, cudaStream_t s);

// Resident k_hydro2 blocks per SM its registers are sized for (D3Q19; D3Q27 takes 2).
#ifndef LBM_HYDRO2_MINB
#define LBM_HYDRO2_MINB 3
#endif

// The near-contact list of one phi buffer: the 32 x 8 x 4 tiles (3D; 32 x 8 in 2D) holding a
// gated cell, their count, and one mark per tile of the grid (3D), set while the tile is listed.
struct TileList {
  int *tiles = nullptr;
  int *count = nullptr;
  int *mark = nullptr;
};

// The hydrodynamic step split in two launches around the near-contact pass (3D, nx even,
// Q N <= 2^32: the paired kernel). part 0 updates every 64 x 4 x 2 tile half whose near-contact
// tile is not marked in `listed` (those cells are not gated, so they never read frep, and it may
// run while the near-contact pass writes frep); part 1 walks the listed tiles on `blocks`
// resident blocks and updates the rest, after the near-contact pass. Each cell is written by
// exactly one part, with the arithmetic of launch_hydro.
bool hydro_split_applies(int Q, const KParams &P);
cudaError_t launch_hydro_split(int part, int Q, int store, const KParams &P, const void *src, void *dst,
                               const int32_t *phi, const float4 *frep, float *u, const TileList &listed, int blocks,
                               cudaStream_t s);

// Also builds `next` (if its tiles are not null): appends the tiles of phi_out that hold an
// interfacial cell, using next.mark (all zero on entry) in 3D so that each is appended once.
// In 3D the marks of `prev` (the list of phi, consumed by this step's near-contact and
// hydrodynamic passes) are cleared, so that buffer's marks are zero when its list is built again.
cudaError_t launch_phase(int dim, const KParams &P, const int32_t *phi, const float *u, int32_t *phi_out,
                         const TileList &next, const TileList &prev, cudaStream_t s);
// Lists (and in 3D marks) the tiles holding an interfacial cell of phi (after the state is set
// from the host); the count and the marks are zero on entry.
cudaError_t launch_gate_tiles(int dim, const KParams &P, const int32_t *phi, const TileList &list, cudaStream_t s);
int tile_count(int dim, const KParams &P);

// Geometry of the 3D phase-field register march (phase3_march.cuh).
struct March3 {
  static constexpr int OUT = 28;       // output columns per warp
  static constexpr int WARPS = 4;      // warps per block
  static constexpr int NT = 32 * WARPS;
  static constexpr int MIN_RUN = 8;    // fewest planes per warp before the grid is shrunk
};

// Batched passes over many independent cases (the sweep of uneven collision cases). One
// BatchCase per case and buffer parity: where the pass reads and writes, and its tile grids.
struct __align__(16) BatchCase {
  KParams P;
  const void *src;      // populations of the current state
  void *dst;            // populations of the next state
  const int32_t *phi;   // phi^n
  int32_t *phi_out;     // phi^{n+1}
  const float4 *frep;   // near-contact force at the gated cells of phi^n
  float *u;             // velocity, written by the hydrodynamic pass, read by the phase pass
  TileList next;        // near-contact list of phi^{n+1}, built by the phase pass (tiles null: none)
  TileList prev;        // near-contact list of phi^n, whose marks the phase pass clears
  int ncx;              // x segments of the phase march
};
// The paired hydrodynamic kernel over a list of (case, bx, by, bz) tile items of 64 x ty x tz cells
// (ty x tz = 8; all cases D3Q19 or D3Q27 per Q, one store type, nx even, Q N <= 2^32), on a grid of
// `blocks` resident blocks walking the list.
cudaError_t launch_hydro_batch(int Q, int store, int ty, const BatchCase *cases, const int4 *items, int nitems,
                               int blocks, cudaStream_t s);
int hydro_batch_blocks(int Q, int store, int ty);  // resident blocks of the device (SMs x per SM)
// The phase march over the concatenated (column, plane) units of every case (uoff: ncases + 1
// prefix offsets); rows = 2 or 4 rows of y per thread.
cudaError_t launch_phase_batch(int rows, const BatchCase *cases, const long long *uoff, int ncases, int blocks,
                               cudaStream_t s);
int phase_batch_blocks(int rows);

// Conversions between host-layout FP64 staging buffers and the device state.
cudaError_t launch_phi_in(const KParams &P, const double *phi64, int32_t *phi, cudaStream_t s);
cudaError_t launch_phi_out(const KParams &P, const int32_t *phi, double *phi64, cudaStream_t s);
cudaError_t launch_f32_out(long long n, const float *src, double *dst, cudaStream_t s);
cudaError_t launch_init_pops(int Q, int store, const KParams &P, const double *u64, const double *ps64,
                             void *pops, cudaStream_t s);
cudaError_t launch_set_pops(int Q, int store, const KParams &P, const double *f64, void *pops, cudaStream_t s);
cudaError_t launch_get_pops(int Q, int store, const KParams &P, const void *pops, double *f64, cudaStream_t s);
cudaError_t launch_partner_frep_out(const KParams &P, int dim, const float4 *frep, double *frep64,
                                    cudaStream_t s);

// FP64 / exact-integer reductions over the current fields.
struct ReduceOut {
  long long phi_q30;  // exact sum of the fixed-point phi
  double mom[3];      // sum of rho(phi) u
  long long nonfinite;
};
constexpr int kReduceBlocks = 608;  // 4 per SM of a 152-SM GB300
// The phi sum (exact), the non-finite count of u (u may be null when mom is false) and, with mom,
// the FP64 momentum sum of rho(phi) u.
cudaError_t launch_reduce(const KParams &P, const int32_t *phi, const float *u, ReduceOut *partials,
                          ReduceOut *out, cudaStream_t s, bool mom = true);
// The same reduction on a grid of nblocks blocks (nblocks partial slots).
cudaError_t launch_reduce_n(const KParams &P, const int32_t *phi, const float *u, ReduceOut *partials,
                            int nblocks, ReduceOut *out, cudaStream_t s);

// Near-contact film statistics (Sec. 3.3): over the cells with a partner (frep.w = 1 at gated
// cells), V_film, sum |F_rep.n|, sum |F_cap.n|, max |F_rep|, sum |F_rep| in FP64, fixed order.
struct DiagOut {
  double v[5];
};
cudaError_t launch_nci_diag(int dim, const KParams &P, const int32_t *phi, const float4 *frep, DiagOut *partials,
                            DiagOut *out, cudaStream_t s);

// Interfacial mean curvature kappa = div n (Sec. 3.4, Eq. 78): normals of every cell into nrm, then
// over the band q >= q_th a histogram of kappa on [kmin, kmax) (nbins <= kMaxCurvBins, integer
// counts) and the band's cell count and sum of kappa (FP64, fixed order): out = {count, sum}.
constexpr int kMaxCurvBins = 4096;

// Carrier-phase kinetic-energy spectrum (Sec. 3.4) of the velocity u (3N) into E_dev (nshells
// doubles on the device), synchronous on s. Returns 0, 1 (bad nshells), 2 (CUDA error or out of
// memory) or 3 (cuFFT failure). Allocates about 8N bytes plus the transform's workspace per call.
constexpr int kMaxSpectrumShells = 1024;
int spectrum_compute(const KParams &P, const int32_t *phi, const float *u, int nshells, double *E_dev,
                     cudaStream_t s);
cudaError_t launch_curvature(int dim, const KParams &P, const int32_t *phi, float4 *nrm, float kmin, float kmax,
                             int nbins, unsigned long long *hist, double *partials, double *out, cudaStream_t s);

}  // namespace lbm
