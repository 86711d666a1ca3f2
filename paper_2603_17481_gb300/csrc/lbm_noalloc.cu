// lbm_noalloc.cu -- lbm_mass_noalloc: the FP64 integrals of lbm_mass computed without allocating
// any device memory.
//
// Some callers cannot allocate device memory at the moment they need the integrals: processes
// whose device memory is already reserved by another allocator (a framework's caching allocator
// that owns nearly all of HBM, where a raw cudaMalloc would fail or fragment it), and latency-
// critical loops in which cudaMalloc's implicit device-wide synchronisation is not acceptable.
// lbm_mass allocates its moment buffer on first use; this variant instead keeps the reduction
// scratch (one partial slot per block of 4096 cells, plus the result) in a file-scope static
// device array of fixed size, which every GPU that loads the library holds until the process exits.
#include <mutex>

#include "ctx.h"

using namespace lbm;

namespace {

constexpr int kCellsPerBlock = 4096;  // 256 threads x 16 cells per thread
constexpr int kMaxBlocks = 4096;      // => at most 16,777,216 cells
constexpr int kMaxDevices = 64;

// Shared by every call on a device; a call overwrites every slot it reads, so nothing needs to be
// cleared between calls.
static __device__ __align__(256) ReduceOut g_lbm_noalloc_scratch[kMaxBlocks + 1];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device, looked up once per device (the
// array's name is only a host-side stand-in, not a device address).
int scratch_for_current_device(ReduceOut **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lbm_noalloc_scratch) != cudaSuccess || !p) return LBM_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<ReduceOut *>(g_scratch_addr[dev]);
  return LBM_OK;
}

}  // namespace

// Called by lbm_create with the context's device current. With lazy module loading (the CUDA
// default), the module holding the static scratch is loaded, and its memory taken, on the first
// use of one of its symbols; looking the address up here makes that happen while the library is
// still allowed to allocate, not in the first lbm_mass_noalloc call.
int lbm_noalloc_prepare_device() {
  ReduceOut *scratch = nullptr;
  return scratch_for_current_device(&scratch);
}

extern "C" int lbm_mass_noalloc(lbm_ctx *c, double *phi_mass, double *mom) {
  if (!c) return LBM_ERR_ARG;
  const long long nblocks = (c->N + kCellsPerBlock - 1) / kCellsPerBlock;
  if (nblocks > kMaxBlocks) return LBM_ERR_ARG;  // more than 16,777,216 cells
  if (!c->initialised || !c->mom) return LBM_ERR_STATE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
  if (dev != c->device) return LBM_ERR_ARG;  // the context's device must be current
  ReduceOut *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;

  // moments of the current state (the near-contact and hydrodynamic kernels in moments mode, as in
  // lbm_mass), then the reduction into the static scratch
  cudaError_t e = cudaSuccess;
  if (c->P.nci_on)
    e = launch_nci(c->P.dim, c->K, c->T, c->phi[c->pcur], c->nrm, c->frep, nullptr, 0, c->tiles[c->pcur],
                   c->ntiles + c->pcur, c->nci_blocks, c->stream, nci_aux(c), c->ntiles + (c->pcur ^ 1));
  if (e == cudaSuccess)
    e = launch_hydro(c->P.Q, c->P.store, kMoments, c->K, c->pop[c->cur], nullptr, c->phi[c->pcur], c->frep,
                     c->mom, c->mom + 3 * c->N, c->stream);
  if (e == cudaSuccess)
    e = launch_reduce_n(c->K, c->phi[c->pcur], c->mom, scratch, (int)nblocks, scratch + kMaxBlocks, c->stream);
  ReduceOut r;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, scratch + kMaxBlocks, sizeof(r), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  if (phi_mass) *phi_mass = (double)r.phi_q30 / 1073741824.0;
  if (mom)
    for (int a = 0; a < 3; a++) mom[a] = r.mom[a];
  return LBM_OK;
}
