// batch_kernels.cu -- the hydrodynamic and phase-field passes of a step over many independent
// cases in one launch each (the batched sweep of uneven collision cases; the paper runs one case
// at a time). A persistent grid of resident blocks (hydro) or warps (phase) walks a work list that
// concatenates every case: (case, tile) items for the hydrodynamic tiles, and the (column, plane)
// units of the phase march split evenly over the warps. Each item runs the same tile or march code
// as the single-case kernels, with that case's parameters and buffers (BatchCase).
#include "hydro_impl.cuh"
#include "phase3_march.cuh"

namespace lbm {

// The case record of the next item is copied into shared memory (double-buffered) while the
// current item computes, so an item starts without a chain of dependent global loads, and its
// parameters are read from shared memory.
template <class L, int S, int TY>
__global__ void __launch_bounds__(256, L::Q >= 27 ? 2 : LBM_HYDRO2_MINB)
k_hydro2_batch(const BatchCase *__restrict__ cases, const int4 *__restrict__ items, const int nitems) {
  pdl_enter();
  constexpr int TZ = 8 / TY;
  constexpr int WORDS = sizeof(BatchCase) / sizeof(uint4);
  static_assert(sizeof(BatchCase) % sizeof(uint4) == 0, "case record in 16-byte words");
  __shared__ uint4 s_case[2][WORDS];
  __shared__ int4 s_item[2];
  using T = typename Store<S>::T;
  const int tid = threadIdx.x + 32 * (threadIdx.y + TY * threadIdx.z);
  auto fetch = [&](int it, int buf) {  // warp 0 copies item it and its case record
    if (tid < 32 && it < nitems) {
      const int4 w = items[it];
      const uint4 *src = reinterpret_cast<const uint4 *>(cases + w.x);
      for (int k = tid; k < WORDS; k += 32) s_case[buf][k] = src[k];
      if (tid == 0) s_item[buf] = w;
    }
  };
  int buf = 0;
  fetch(blockIdx.x, 0);
  __syncthreads();
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    fetch(it + gridDim.x, buf ^ 1);  // in flight during this item
    const BatchCase &C = *reinterpret_cast<const BatchCase *>(s_case[buf]);
    const int4 w = s_item[buf];
    hydro2_tile<L, S, kStep, TY, TZ>(C.P, (const T *)C.src, (T *)C.dst, C.phi, C.frep, C.u, nullptr, w.y, w.z, w.w);
    __syncthreads();  // this item's staged phi and case record are no longer read
    buf ^= 1;
  }
}

template <int M>
__global__ void __launch_bounds__(March3::NT, LBM_MARCH_MINB)
k_phase3m_batch(const BatchCase *__restrict__ cases, const long long *__restrict__ uoff, const int ncases) {
  pdl_enter();
  // the marks of the lists of phi^n: block b clears those of cases b, b + grid, ...
  for (int c = blockIdx.x; c < ncases; c += gridDim.x) clear_marks(cases[c].prev, threadIdx.x, March3::NT);
  const long long units = uoff[ncases];
  const long long nwarps = (long long)gridDim.x * March3::WARPS;
  const long long wid = (long long)blockIdx.x * March3::WARPS + (threadIdx.x >> 5);
  long long ub = units * wid / nwarps;
  const long long ue = units * (wid + 1) / nwarps;
  if (ub >= ue) return;
  int c = 0;  // the case holding unit ub: largest c with uoff[c] <= ub
  {
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (uoff[mid] <= ub) lo = mid; else hi = mid - 1;
    }
    c = lo;
  }
  while (ub < ue) {
    while (uoff[c + 1] <= ub) c++;
    const BatchCase &C = cases[c];
    const int nz = C.P.nz;
    const long long lu = ub - uoff[c];
    const long long col = lu / nz;
    const int z0 = (int)(lu - col * nz);
    const long long end = min(ue, uoff[c + 1]);
    const int z1 = (int)min((long long)nz, (long long)z0 + (end - ub));
    ub += z1 - z0;
    march_run<M>(C.P, C.phi, C.u, C.phi_out, C.next.tiles, C.next.count, C.next.mark, C.ncx, col, z0, z1);
  }
}

namespace {
template <class K> int resident(K kernel, int threads) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess) return 0;
  return sms * (per > 0 ? per : 1);
}

template <class L, int S>
cudaError_t hydro_batch_ty(int ty, const BatchCase *cases, const int4 *items, int nitems, int blocks, cudaStream_t s) {
  switch (ty) {
    case 2: return launch_pdl(k_hydro2_batch<L, S, 2>, dim3(blocks), dim3(32, 2, 4), 0, s, cases, items, nitems);
    case 8: return launch_pdl(k_hydro2_batch<L, S, 8>, dim3(blocks), dim3(32, 8, 1), 0, s, cases, items, nitems);
    default: return launch_pdl(k_hydro2_batch<L, S, 4>, dim3(blocks), dim3(32, 4, 2), 0, s, cases, items, nitems);
  }
}
template <class L>
cudaError_t hydro_batch_store(int store, int ty, const BatchCase *cases, const int4 *items, int nitems, int blocks,
                              cudaStream_t s) {
  switch (store) {
    case 0: return hydro_batch_ty<L, 0>(ty, cases, items, nitems, blocks, s);
    case 1: return hydro_batch_ty<L, 1>(ty, cases, items, nitems, blocks, s);
    default: return hydro_batch_ty<L, 2>(ty, cases, items, nitems, blocks, s);
  }
}
}  // namespace

cudaError_t launch_hydro_batch(int Q, int store, int ty, const BatchCase *cases, const int4 *items, int nitems,
                               int blocks, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (blocks > nitems) blocks = nitems;
  return Q == 27 ? hydro_batch_store<D3Q27>(store, ty, cases, items, nitems, blocks, s)
                 : hydro_batch_store<D3Q19>(store, ty, cases, items, nitems, blocks, s);
}

int hydro_batch_blocks(int Q, int store, int ty) {
  // the resident count depends on the lattice (registers), not on the store or the tile shape
  (void)store; (void)ty;
  return Q == 27 ? resident(k_hydro2_batch<D3Q27, 0, 4>, 256) : resident(k_hydro2_batch<D3Q19, 0, 4>, 256);
}

cudaError_t launch_phase_batch(int rows, const BatchCase *cases, const long long *uoff, int ncases, int blocks,
                               cudaStream_t s) {
  if (ncases <= 0) return cudaSuccess;
  return rows == 2 ? launch_pdl(k_phase3m_batch<2>, dim3(blocks), dim3(March3::NT), 0, s, cases, uoff, ncases)
                   : launch_pdl(k_phase3m_batch<4>, dim3(blocks), dim3(March3::NT), 0, s, cases, uoff, ncases);
}

int phase_batch_blocks(int rows) {
  return rows == 2 ? resident(k_phase3m_batch<2>, March3::NT) : resident(k_phase3m_batch<4>, March3::NT);
}

}  // namespace lbm
