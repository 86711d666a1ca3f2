// lbm_api.cu -- the C ABI of include/lbm.h: context lifetime, device memory, host <-> device
// conversions, the per-step launch sequence, the periodic conservation check and the profiler.
//
// Device memory of a context (N cells, Q directions, store type T):
//   pop[2]   Q*N T        ping-pong population buffers (pull scheme, structure of arrays)
//   phi[2]   N int32      fixed-point phi, ping-pong
//   u        3*N float    velocity of the last hydrodynamic pass (advects phi)
//   frep     N float4     near-contact force, valid at gated cells only
//   nrm      N float4     interface normals, valid at gated cells only
//   mom      4*N float    u and p* of lbm_read_fields / lbm_mass (allocated on first use)
//   stage    k*N double   FP64 staging of host I/O (allocated on first use, grown as needed)
//   tiles[2] int          near-contact tiles holding an interfacial cell of phi[k] (+ 2 counts)
//   lflag    2 x int      per near-contact tile and phi buffer: the tile is in that buffer's list
//   red      reduction partials and result
#include <cuda.h>  // driver API types (CUpointer_attribute); no driver symbols are linked

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.h"

using namespace lbm;

namespace {

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  if (e == cudaErrorMemoryAllocation) return LBM_ERR_OOM;
  return LBM_ERR_CUDA;
}

cudaEvent_t take_event(lbm_ctx *c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Wraps one launch (on stream s, default the context stream) in a pair of events when the
// profiler is on.
template <class F> cudaError_t timed_on(lbm_ctx *c, cudaStream_t s, int kind, F &&launch, int kernels = 1) {
  if (!c->prof || !((c->prof_mask >> kind) & 1u)) return launch();
  if (c->prof_seen[kind]++ % c->prof_every != 0) return launch();  // a pass between samples
  cudaEvent_t a = take_event(c), b = take_event(c);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaEventRecord(a, s);
  cudaError_t e = launch();
  cudaEventRecord(b, s);
  c->pairs.push_back({kind, kernels, a, b});
  return e;
}
template <class F> cudaError_t timed(lbm_ctx *c, int kind, F &&launch, int kernels = 1) {
  return timed_on(c, c->stream, kind, launch, kernels);
}

int validate(const lbm_params *p) {
  if (!p) return LBM_ERR_ARG;
  if (p->dim != 2 && p->dim != 3) return LBM_ERR_ARG;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBM_ERR_ARG;
  if (p->dim == 2 && (p->nz != 1 || p->Q != 9)) return LBM_ERR_ARG;
  if (p->dim == 3 && p->Q != 19 && p->Q != 27) return LBM_ERR_ARG;
  if (p->store < LBM_STORE_F32 || p->store > LBM_STORE_MOMENTS) return LBM_ERR_ARG;
  if (p->store == LBM_STORE_MOMENTS && p->dim != 3) return LBM_ERR_ARG;
  long long N = (long long)p->nx * p->ny * p->nz;
  if (N > (long long)INT_MAX) return LBM_ERR_ARG;
  if (!(p->rho_l > 0) || !(p->rho_g > 0) || !(p->nu_l > 0) || !(p->nu_g > 0)) return LBM_ERR_ARG;
  if (!(p->eps > 0) || !(p->D >= 0) || !std::isfinite(p->sigma)) return LBM_ERR_ARG;
  if (p->nci_on) {
    if (p->w < 1 || p->w > 3) return LBM_ERR_ARG;
    if (!(p->h0 > 0) || !(p->p > 0) || !(p->q_th > 0) || !(p->q_th <= 0.25)) return LBM_ERR_ARG;
    if (!(p->eta >= 0) || !(p->eps_q > 0) || !std::isfinite(p->A_rep) || !std::isfinite(p->cos_opp))
      return LBM_ERR_ARG;
  }
  if (!(p->eps_n > 0)) return LBM_ERR_ARG;
  for (int a = 0; a < 3; a++)
    if (!std::isfinite(p->g[a])) return LBM_ERR_ARG;
  if (p->mass_check_every < 0 || !(p->mass_tol >= 0)) return LBM_ERR_ARG;
  return LBM_OK;
}

void derive_kparams(const lbm_params &p, KParams &K) {
  K.nx = p.nx; K.ny = p.ny; K.nz = p.nz;
  K.N = (long long)p.nx * p.ny * p.nz;
  K.rho_g = (float)p.rho_g;
  K.drho = (float)(p.rho_l - p.rho_g);
  K.mu_g = (float)(p.rho_g * p.nu_g);
  K.dmu = (float)(p.rho_l * p.nu_l - p.rho_g * p.nu_g);
  const double beta = 12.0 * p.sigma / p.eps, kap = 1.5 * p.sigma * p.eps;
  K.beta4 = (float)(4.0 * beta);
  K.kap = (float)kap;
  K.rho_bar = (float)p.rho_l;
  for (int a = 0; a < 3; a++) K.g[a] = (float)p.g[a];
  K.nci_on = p.nci_on;
  K.w = p.w;
  K.A_rep = (float)p.A_rep; K.h0 = (float)p.h0; K.p = (float)p.p; K.q_th = (float)p.q_th;
  K.eta = (float)p.eta; K.cos_opp = (float)p.cos_opp; K.eps_q = (float)p.eps_q; K.eps_n = (float)p.eps_n;
  K.eps = (float)p.eps;
  K.Dlap = (float)(p.D * 6.0);
  K.kc = (float)(3.0 * 4.0 * p.D / p.eps);
  K.rho_g64 = p.rho_g;
  K.drho64 = p.rho_l - p.rho_g;
}

// Window offsets of Eq. 60 sorted by |r|^2, then by the canonical index
// ((rz + w)(2w + 1) + (ry + w))(2w + 1) + (rx + w).
void build_table(int dim, int w, NciTable &T) {
  struct E { int d2, k, dx, dy, dz; };
  std::vector<E> v;
  const int W = 2 * w + 1, zr = dim == 3 ? w : 0;
  for (int rz = -zr; rz <= zr; rz++)
    for (int ry = -w; ry <= w; ry++)
      for (int rx = -w; rx <= w; rx++) {
        if (!rx && !ry && !rz) continue;
        v.push_back({rx * rx + ry * ry + rz * rz, ((rz + zr) * W + (ry + w)) * W + (rx + w), rx, ry, rz});
      }
  std::sort(v.begin(), v.end(), [](const E &a, const E &b) { return a.d2 != b.d2 ? a.d2 < b.d2 : a.k < b.k; });
  T.count = (int)v.size();
  for (int i = 0; i < T.count; i++)
    T.o[i] = NciOffset{(int8_t)v[i].dx, (int8_t)v[i].dy, (int8_t)v[i].dz, (int8_t)v[i].d2};
}

// bytes of one population buffer
size_t store_bytes(const lbm_params &p, long long N) {
  if (p.store == LBM_STORE_MOMENTS) return sizeof(float4) * kRecordWords * (size_t)N;
  return (size_t)p.Q * (size_t)N * (p.store == LBM_STORE_F32 ? 4 : 2);
}

int ensure_stage(lbm_ctx *c, size_t bytes) {
  if (c->stage_bytes >= bytes) return LBM_OK;
  if (c->stage) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&c->stage, bytes);
  if (e != cudaSuccess) {
    c->stage = nullptr;
    return from_cuda(e);
  }
  c->stage_bytes = bytes;
  return LBM_OK;
}

int ensure_mom(lbm_ctx *c) {
  if (c->mom) return LBM_OK;
  cudaError_t e = cudaMalloc(&c->mom, sizeof(float) * 4 * c->N);
  if (e != cudaSuccess) {
    c->mom = nullptr;
    return from_cuda(e);
  }
  return from_cuda(cudaMemsetAsync(c->mom, 0, sizeof(float) * 4 * c->N, c->stream));
}

int h2d(lbm_ctx *c, void *dst, const void *src, size_t bytes) {
  return from_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
}
int d2h(lbm_ctx *c, void *dst, const void *src, size_t bytes) {
  return from_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
}
int sync(lbm_ctx *c) { return from_cuda(cudaStreamSynchronize(c->stream)); }

// Device address of a caller's host array of `bytes` bytes when the whole array lies in one
// page-locked host allocation (cudaHostAlloc, cudaHostRegister): such memory is mapped into the
// device's address space, so the conversion kernels read or write it in place over the host link
// and the conversion hides under the transfer (the copy engines and the SMs reach the same link
// bandwidth). Null for any other memory, which goes through the staging buffer with one copy.
// The device's access to the memory at p as the driver reports it (CU_POINTER_ATTRIBUTE_ACCESS_FLAGS:
// 0 none, 1 read only, 3 read and write), or -1 when it cannot be asked. The driver call is looked
// up through the runtime, so the library does not link the driver library itself.
int device_access(const void *p) {
  using Fn = CUresult (*)(void *, CUpointer_attribute, CUdeviceptr);
  static const Fn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      return static_cast<Fn>(nullptr);
    }
    return reinterpret_cast<Fn>(f);
  }();
  if (!fn) return -1;
  unsigned long long v = 0;  // the driver writes a 4-byte enumerator into the low half
  if (fn(&v, CU_POINTER_ATTRIBUTE_ACCESS_FLAGS, reinterpret_cast<CUdeviceptr>(p)) != CUDA_SUCCESS) return -1;
  return (int)(v & 0xffffffffull);
}

// write: the kernels will store into the array, so memory registered read-only
// (cudaHostRegisterReadOnly) is staged instead; reads need read access.
template <class T>
T *mapped_view(T *p, size_t bytes, bool write) {
  if (!p || bytes == 0) return nullptr;
  const char *lo = reinterpret_cast<const char *>(p), *hi = lo + bytes - 1;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, lo) != cudaSuccess || cudaPointerGetAttributes(&b, hi) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
    return nullptr;
  // both ends map into one contiguous device range (one allocation, no gap)
  if (static_cast<const char *>(b.devicePointer) - static_cast<const char *>(a.devicePointer) != (ptrdiff_t)(bytes - 1))
    return nullptr;
  const int need = write ? CU_POINTER_ATTRIBUTE_ACCESS_FLAG_READWRITE : CU_POINTER_ATTRIBUTE_ACCESS_FLAG_READ;
  const int acc = device_access(a.devicePointer);
  if (acc < 0 || (acc & need) != need) return nullptr;
  return static_cast<T *>(a.devicePointer);
}

// rho_bar from the exact phi sum; also records the phi-mass reference of the conservation check
// and lists the near-contact tiles of the initial phi.
int finish_init(lbm_ctx *c) {
  int rc = from_cuda(cudaMemsetAsync(c->ntiles, 0, 2 * sizeof(int), c->stream));
  if (rc) return rc;
  rc = from_cuda(cudaMemsetAsync(c->lflag, 0, sizeof(int) * 2 * (size_t)c->ntile, c->stream));
  if (rc) return rc;
  rc = from_cuda(launch_gate_tiles(c->P.dim, c->K, c->phi[c->pcur], tile_list(c, c->pcur), c->stream));
  if (rc) return rc;
  rc = from_cuda(launch_reduce(c->K, c->phi[c->pcur], nullptr, c->red_part, c->red_out, c->stream, false));
  if (rc) return rc;
  ReduceOut r;
  if ((rc = d2h(c, &r, c->red_out, sizeof(r)))) return rc;
  if ((rc = sync(c))) return rc;
  const double mean_phi = (double)r.phi_q30 / 1073741824.0 / (double)c->N;
  c->K.rho_bar = (float)(c->P.rho_g + (c->P.rho_l - c->P.rho_g) * mean_phi);
  c->phi_q30_ref = r.phi_q30;
  c->initialised = true;
  c->steps = 0;
  return LBM_OK;
}

// Near-contact kernel + hydrodynamic kernel in moments mode on the current state -> c->mom.
int run_moments(lbm_ctx *c) {
  int rc = ensure_mom(c);
  if (rc) return rc;
  const int d = c->P.dim;
  if (c->P.nci_on) {
    rc = from_cuda(timed(c, LBM_K_NCI, [&] {
      return launch_nci(d, c->K, c->T, c->phi[c->pcur], c->nrm, c->frep, nullptr, 0, c->tiles[c->pcur],
                        c->ntiles + c->pcur, c->nci_blocks, c->stream, nci_aux(c), c->ntiles + (c->pcur ^ 1));
    }, nci_list_kernels(c)));
    if (rc) return rc;
  }
  return from_cuda(timed(c, LBM_K_HYDRO, [&] {
    return launch_hydro(c->P.Q, c->P.store, kMoments, c->K, c->pop[c->cur], nullptr, c->phi[c->pcur], c->frep,
                        c->mom, c->mom + 3 * c->N, c->stream);
  }));
}

}  // namespace

// One step's launches on stream s, from population buffer cur and phi buffer pcur, for a context
// whose state is set: the near-contact pass over the tiles listed for phi^n (it also empties the
// list of the other phi buffer, consumed by the previous step), the hydrodynamic pass, then the
// phase-field pass. With lists, the phase-field pass lists the tiles of phi^{n+1} and clears the
// marks of phi^n's list; without, the lists are left as they are (a dry step writes only the
// next-step buffers and per-step scratch). Makes no non-stream CUDA call (it may be captured).
int enqueue_step(lbm_ctx *c, int cur, int pcur, bool lists, cudaStream_t st) {
  const int d = c->P.dim, nxt = cur ^ 1, pn = pcur ^ 1;
  const bool nci = c->P.nci_on != 0;
  int rc;
  if (nci && c->overlap_blocks > 0 && c->side) {
    // split step: the near-contact pass, then the listed tiles' hydrodynamics, on the side stream,
    // while st updates every other tile (none of their cells is gated, so none reads frep)
    const TileList listed = tile_list(c, pcur);
    rc = from_cuda(cudaEventRecord(c->ev_fork, st));
    if (!rc) rc = from_cuda(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    if (rc) return rc;
    rc = from_cuda(timed_on(c, c->side, LBM_K_NCI, [&] {
      return launch_nci(d, c->K, c->T, c->phi[pcur], c->nrm, c->frep, nullptr, 0, c->tiles[pcur], c->ntiles + pcur,
                        c->overlap_blocks, c->side, nci_aux(c), c->ntiles + pn);
    }, nci_list_kernels(c)));
    if (rc) return rc;
    rc = from_cuda(launch_hydro_split(1, c->P.Q, c->P.store, c->K, c->pop[cur], c->pop[nxt], c->phi[pcur], c->frep,
                                      c->u, listed, c->split_blocks, c->side));
    if (!rc) rc = from_cuda(cudaEventRecord(c->ev_join, c->side));
    if (rc) return rc;
    // the hydrodynamic pass as timed: from its first launch to the join of both parts
    rc = from_cuda(timed_on(c, st, LBM_K_HYDRO, [&] {
      cudaError_t e = launch_hydro_split(0, c->P.Q, c->P.store, c->K, c->pop[cur], c->pop[nxt], c->phi[pcur],
                                         c->frep, c->u, listed, 0, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_join, 0);
      return e;
    }, 2));
    if (rc) return rc;
  } else {
    if (nci) {
      rc = from_cuda(timed_on(c, st, LBM_K_NCI, [&] {
        return launch_nci(d, c->K, c->T, c->phi[pcur], c->nrm, c->frep, nullptr, 0, c->tiles[pcur],
                          c->ntiles + pcur, c->nci_blocks, st, nci_aux(c), c->ntiles + pn);
      }, nci_list_kernels(c)));
      if (rc) return rc;
    }
    rc = from_cuda(timed_on(c, st, LBM_K_HYDRO, [&] {
      return launch_hydro(c->P.Q, c->P.store, kStep, c->K, c->pop[cur], c->pop[nxt], c->phi[pcur], c->frep, c->u,
                          nullptr, st);
    }));
    if (rc) return rc;
  }
  const bool upd = nci && lists;
  return from_cuda(timed_on(c, st, LBM_K_PHASE, [&] {
    return launch_phase(d, c->K, c->phi[pcur], c->u, c->phi[pn], upd ? tile_list(c, pn) : TileList{},
                        upd ? tile_list(c, pcur) : TileList{}, st);
  }));
}

extern "C" {

void lbm_params_default(lbm_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dim = 3; p->nx = p->ny = p->nz = 64; p->Q = 19; p->store = LBM_STORE_F32;
  p->rho_l = 1.0; p->rho_g = 1.0; p->nu_l = 0.005; p->nu_g = 0.05; p->sigma = 0.02;
  p->eps = 4.0; p->D = 0.1;
  p->nci_on = 1; p->w = 3; p->A_rep = 0.02; p->h0 = 1.0; p->p = 4.0;
  p->q_th = 0.125; p->eta = 0.1; p->cos_opp = -0.8; p->eps_q = 1e-12; p->eps_n = 1e-4;
  p->mass_check_every = 0; p->mass_tol = 1e-9;
}

int lbm_create(const lbm_params *p, lbm_ctx **out) {
  if (!out) return LBM_ERR_ARG;
  int rc = validate(p);
  if (rc) return rc;
  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_OOM;
  c->P = *p;
  derive_kparams(*p, c->K);
  build_table(p->dim, p->nci_on ? p->w : 1, c->T);
  c->N = c->K.N;
  c->pop_bytes = store_bytes(*p, c->N);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->pop[0], c->pop_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->pop[1], c->pop_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->phi[0], sizeof(int32_t) * c->N);
  if (e == cudaSuccess) e = cudaMalloc(&c->phi[1], sizeof(int32_t) * c->N);
  if (e == cudaSuccess) e = cudaMalloc(&c->u, sizeof(float) * 3 * c->N);
  if (e == cudaSuccess) e = cudaMalloc(&c->frep, sizeof(float4) * c->N);
  if (e == cudaSuccess) e = cudaMalloc(&c->nrm, sizeof(float4) * c->N);
  const int ntile = tile_count(p->dim, c->K);
  c->ntile = ntile;
  if (e == cudaSuccess) e = cudaMalloc(&c->tiles[0], sizeof(int) * ntile);
  if (e == cudaSuccess) e = cudaMalloc(&c->tiles[1], sizeof(int) * ntile);
  if (e == cudaSuccess) e = cudaMalloc(&c->ntiles, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->ntiles, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->lflag, sizeof(int) * 2 * (size_t)ntile);
  if (e == cudaSuccess) e = cudaMemset(c->lflag, 0, sizeof(int) * 2 * (size_t)ntile);
  if (e == cudaSuccess && p->nci_on && nci_aux_applies(p->dim, c->K)) {
    e = cudaMalloc(&c->aux.bricks, sizeof(uint4) * nci_brick_count(c->K));
    if (e == cudaSuccess) e = cudaMalloc(&c->aux.flags, (size_t)ntile);
    if (e == cudaSuccess) e = cudaMemset(c->aux.flags, 0, (size_t)ntile);
    if (e == cudaSuccess) e = cudaMalloc(&c->aux.scan_tiles, sizeof(int) * ntile);
    if (e == cudaSuccess) e = cudaMalloc(&c->aux.nscan, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->aux.nscan, 0, sizeof(int));
  }
  if (e == cudaSuccess) {
    c->nci_blocks = nci_list_blocks(p->dim);
    if (c->nci_blocks <= 0) e = cudaErrorInvalidConfiguration;
  }
  if (e == cudaSuccess && p->nci_on && p->store != LBM_STORE_MOMENTS && hydro_split_applies(p->Q, c->K)) {
    // the stream and events of the split step (lbm_set_overlap); it is off by default
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    c->overlap_blocks = 0;
    c->split_blocks = c->nci_blocks;
  }
  if (e == cudaSuccess) e = phase_prepare(p->dim);
  // the static scratch of lbm_mass_noalloc is taken here, once per device, while allocating is
  // allowed; a failure is not the context's (lbm_mass_noalloc repeats the look-up and reports it)
  if (e == cudaSuccess) (void)lbm_noalloc_prepare_device();
  if (e == cudaSuccess) e = cudaMalloc(&c->red_part, sizeof(ReduceOut) * kReduceBlocks);
  if (e == cudaSuccess) e = cudaMalloc(&c->red_out, sizeof(ReduceOut));
  if (e == cudaSuccess) e = cudaMemset(c->u, 0, sizeof(float) * 3 * c->N);
  if (e == cudaSuccess) e = cudaMemset(c->frep, 0, sizeof(float4) * c->N);
  if (e == cudaSuccess) e = cudaMemset(c->phi[0], 0, sizeof(int32_t) * c->N);
  if (e == cudaSuccess) e = cudaMemset(c->phi[1], 0, sizeof(int32_t) * c->N);
  if (e != cudaSuccess) {
    lbm_destroy(c);
    return from_cuda(e);
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);  // the stream must outlive the context
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (auto &pp : c->pairs) {
    cudaEventDestroy(pp.a);
    cudaEventDestroy(pp.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  cudaFree(c->pop[0]); cudaFree(c->pop[1]);
  cudaFree(c->phi[0]); cudaFree(c->phi[1]);
  cudaFree(c->u); cudaFree(c->frep); cudaFree(c->nrm); cudaFree(c->mom); cudaFree(c->stage);
  cudaFree(c->partner); cudaFree(c->red_part); cudaFree(c->red_out);
  cudaFree(c->diag_part); cudaFree(c->diag_out);
  cudaFree(c->curv_hist); cudaFree(c->curv_part);
  cudaFree(c->tiles[0]); cudaFree(c->tiles[1]); cudaFree(c->ntiles); cudaFree(c->lflag);
  cudaFree(c->aux.bricks); cudaFree(c->aux.flags); cudaFree(c->aux.scan_tiles); cudaFree(c->aux.nscan);
  delete c;
}

int lbm_set_stream(lbm_ctx *c, void *stream) {
  if (!c) return LBM_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return LBM_OK;
}

int lbm_init_fields(lbm_ctx *c, const double *phi, const double *u, const double *pstar) {
  if (!c || !phi || !u) return LBM_ERR_ARG;
  const long long N = c->N;
  const size_t bN = sizeof(double) * N;
  // page-locked inputs are read in place; the others are staged
  const double *d_phi = mapped_view(phi, bN, false), *d_u = mapped_view(u, 3 * bN, false),
               *d_ps = mapped_view(pstar, bN, false);
  int rc = LBM_OK;
  if ((!d_phi || !d_u || (pstar && !d_ps)) && (rc = ensure_stage(c, 5 * bN))) return rc;
  if (!d_phi) {
    if ((rc = h2d(c, c->stage, phi, bN))) return rc;
    d_phi = c->stage;
  }
  if (!d_u) {
    if ((rc = h2d(c, c->stage + N, u, 3 * bN))) return rc;
    d_u = c->stage + N;
  }
  if (pstar && !d_ps) {
    if ((rc = h2d(c, c->stage + 4 * N, pstar, bN))) return rc;
    d_ps = c->stage + 4 * N;
  }
  c->cur = 0;
  c->pcur = 0;
  rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_phi_in(c->K, d_phi, c->phi[0], c->stream); }));
  if (rc) return rc;
  rc = from_cuda(timed(c, LBM_K_CONVERT, [&] {
    return launch_init_pops(c->P.Q, c->P.store, c->K, d_u, d_ps, c->pop[0], c->stream);
  }));
  if (rc) return rc;
  return finish_init(c);
}

int lbm_set_state(lbm_ctx *c, const double *f, const double *phi) {
  if (!c || !f || !phi) return LBM_ERR_ARG;
  if (c->P.store == LBM_STORE_MOMENTS) return LBM_ERR_STATE;  // arbitrary f has no record form
  const long long N = c->N;
  const int Q = c->P.Q;
  int rc = ensure_stage(c, sizeof(double) * (size_t)(Q + 1) * N);
  if (rc) return rc;
  double *s_f = c->stage, *s_phi = c->stage + (size_t)Q * N;
  if ((rc = h2d(c, s_f, f, sizeof(double) * (size_t)Q * N))) return rc;
  if ((rc = h2d(c, s_phi, phi, sizeof(double) * N))) return rc;
  c->cur = 0;
  c->pcur = 0;
  rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_phi_in(c->K, s_phi, c->phi[0], c->stream); }));
  if (rc) return rc;
  rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_set_pops(Q, c->P.store, c->K, s_f, c->pop[0], c->stream); }));
  if (rc) return rc;
  return finish_init(c);
}

int lbm_get_state(lbm_ctx *c, double *f, double *phi) {
  if (!c) return LBM_ERR_ARG;
  if (!c->initialised) return LBM_ERR_STATE;
  const long long N = c->N;
  const int Q = c->P.Q;
  int rc = ensure_stage(c, sizeof(double) * (size_t)(Q + 1) * N);
  if (rc) return rc;
  double *s_f = c->stage, *s_phi = c->stage + (size_t)Q * N;
  if (f) {
    rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_get_pops(Q, c->P.store, c->K, c->pop[c->cur], s_f, c->stream); }));
    if (rc) return rc;
    if ((rc = d2h(c, f, s_f, sizeof(double) * (size_t)Q * N))) return rc;
  }
  if (phi) {
    rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_phi_out(c->K, c->phi[c->pcur], s_phi, c->stream); }));
    if (rc) return rc;
    if ((rc = d2h(c, phi, s_phi, sizeof(double) * N))) return rc;
  }
  return sync(c);
}

int lbm_set_overlap(lbm_ctx *c, int blocks) {
  if (!c || blocks < 0) return LBM_ERR_ARG;
  if (!c->side) return blocks == 0 ? LBM_OK : LBM_ERR_STATE;
  c->overlap_blocks = std::min(blocks, c->nci_blocks);
  return LBM_OK;
}

int lbm_get_overlap(const lbm_ctx *c, int *blocks) {
  if (!c || !blocks) return LBM_ERR_ARG;
  *blocks = c->side ? c->overlap_blocks : 0;
  return LBM_OK;
}

int lbm_step(lbm_ctx *c, int n) {
  if (!c || n < 0) return LBM_ERR_ARG;
  if (!c->initialised) return LBM_ERR_STATE;
  for (int s = 0; s < n; s++) {
    const int nxt = c->cur ^ 1, pn = c->pcur ^ 1;
    int rc = enqueue_step(c, c->cur, c->pcur, true, c->stream);
    if (rc) return rc;
    c->cur = nxt;
    c->pcur = pn;
    c->steps++;
    if (c->P.mass_check_every > 0 && c->steps % c->P.mass_check_every == 0) {
      rc = from_cuda(timed(c, LBM_K_REDUCE, [&] {
        return launch_reduce(c->K, c->phi[c->pcur], c->u, c->red_part, c->red_out, c->stream, false);
      }, 2));
      if (rc) return rc;
      ReduceOut r;
      if ((rc = d2h(c, &r, c->red_out, sizeof(r)))) return rc;
      if ((rc = sync(c))) return rc;
      const double ref = std::fabs((double)c->phi_q30_ref);
      const double drift = std::fabs((double)(r.phi_q30 - c->phi_q30_ref)) / (ref > 0 ? ref : 1.0);
      if (r.nonfinite > 0 || !(drift <= c->P.mass_tol)) return LBM_ERR_UNSTABLE;
    }
  }
  return LBM_OK;
}

int lbm_read_fields(lbm_ctx *c, double *phi, double *u, double *pstar) {
  if (!c) return LBM_ERR_ARG;
  if (!c->initialised) return LBM_ERR_STATE;
  const long long N = c->N;
  const size_t bN = sizeof(double) * N;
  // page-locked outputs are written in place; the others are staged
  double *o_phi = mapped_view(phi, bN, true), *o_u = mapped_view(u, 3 * bN, true),
         *o_ps = mapped_view(pstar, bN, true);
  int rc = LBM_OK;
  if (((phi && !o_phi) || (u && !o_u) || (pstar && !o_ps)) && (rc = ensure_stage(c, 5 * bN))) return rc;
  if (u || pstar) {
    if ((rc = run_moments(c))) return rc;
  }
  if (phi) {
    double *t = o_phi ? o_phi : c->stage;
    rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_phi_out(c->K, c->phi[c->pcur], t, c->stream); }));
    if (rc) return rc;
    if (!o_phi && (rc = d2h(c, phi, t, bN))) return rc;
  }
  if (u) {
    double *t = o_u ? o_u : c->stage + N;
    rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_f32_out(3 * N, c->mom, t, c->stream); }));
    if (rc) return rc;
    if (!o_u && (rc = d2h(c, u, t, 3 * bN))) return rc;
  }
  if (pstar) {
    double *t = o_ps ? o_ps : c->stage + 4 * N;
    rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_f32_out(N, c->mom + 3 * N, t, c->stream); }));
    if (rc) return rc;
    if (!o_ps && (rc = d2h(c, pstar, t, bN))) return rc;
  }
  return sync(c);
}

int lbm_mass(lbm_ctx *c, double *phi_mass, double *mom) {
  if (!c) return LBM_ERR_ARG;
  if (!c->initialised) return LBM_ERR_STATE;
  int rc = run_moments(c);
  if (rc) return rc;
  rc = from_cuda(timed(c, LBM_K_REDUCE, [&] {
    return launch_reduce(c->K, c->phi[c->pcur], c->mom, c->red_part, c->red_out, c->stream);
  }, 2));
  if (rc) return rc;
  ReduceOut r;
  if ((rc = d2h(c, &r, c->red_out, sizeof(r)))) return rc;
  if ((rc = sync(c))) return rc;
  if (phi_mass) *phi_mass = (double)r.phi_q30 / 1073741824.0;
  if (mom)
    for (int a = 0; a < 3; a++) mom[a] = r.mom[a];
  return LBM_OK;
}

int lbm_read_nci(lbm_ctx *c, int32_t *partner, double *frep) {
  if (!c) return LBM_ERR_ARG;
  if (!c->initialised) return LBM_ERR_STATE;
  const long long N = c->N;
  int rc;
  if (!c->partner) {
    cudaError_t e = cudaMalloc(&c->partner, sizeof(int32_t) * 3 * N);
    if (e != cudaSuccess) {
      c->partner = nullptr;
      return from_cuda(e);
    }
  }
  if ((rc = ensure_stage(c, sizeof(double) * 3 * N))) return rc;
  rc = from_cuda(timed(c, LBM_K_NCI, [&] {
    return launch_nci(c->P.dim, c->K, c->T, c->phi[c->pcur], c->nrm, c->frep, c->partner, 1, nullptr, nullptr,
                      c->nci_blocks, c->stream);
  }, 2));
  if (rc) return rc;
  if (partner && (rc = d2h(c, partner, c->partner, sizeof(int32_t) * 3 * N))) return rc;
  if (frep) {
    rc = from_cuda(timed(c, LBM_K_CONVERT, [&] { return launch_partner_frep_out(c->K, c->P.dim, c->frep, c->stage, c->stream); }));
    if (rc) return rc;
    if ((rc = d2h(c, frep, c->stage, sizeof(double) * 3 * N))) return rc;
  }
  return sync(c);
}

int lbm_nci_diagnostics(lbm_ctx *c, double *out) {
  if (!c || !out) return LBM_ERR_ARG;
  if (!c->initialised) return LBM_ERR_STATE;
  for (int k = 0; k < 7; k++) out[k] = 0.0;
  if (!c->P.nci_on) return LBM_OK;
  if (!c->diag_part) {
    cudaError_t e = cudaMalloc(&c->diag_part, sizeof(DiagOut) * kReduceBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&c->diag_out, sizeof(DiagOut));
    if (e != cudaSuccess) {
      cudaFree(c->diag_part);
      c->diag_part = nullptr;
      c->diag_out = nullptr;
      return from_cuda(e);
    }
  }
  // the near-contact pass over the tiles listed for the current phi (the list stays for the next step)
  int rc = from_cuda(timed(c, LBM_K_NCI, [&] {
    return launch_nci(c->P.dim, c->K, c->T, c->phi[c->pcur], c->nrm, c->frep, nullptr, 0, c->tiles[c->pcur],
                      c->ntiles + c->pcur, c->nci_blocks, c->stream, nci_aux(c), c->ntiles + (c->pcur ^ 1));
  }, nci_list_kernels(c)));
  if (rc) return rc;
  rc = from_cuda(timed(c, LBM_K_REDUCE, [&] {
    return launch_nci_diag(c->P.dim, c->K, c->phi[c->pcur], c->frep, c->diag_part, c->diag_out, c->stream);
  }, 2));
  if (rc) return rc;
  DiagOut d;
  if ((rc = d2h(c, &d, c->diag_out, sizeof(d)))) return rc;
  if ((rc = sync(c))) return rc;
  for (int k = 0; k < 5; k++) out[k] = d.v[k];
  out[5] = d.v[2] > 0.0 ? d.v[1] / d.v[2] : 0.0;
  out[6] = d.v[0] > 0.0 ? d.v[4] / d.v[0] : 0.0;
  return LBM_OK;
}

int lbm_curvature(lbm_ctx *c, double kmin, double kmax, int nbins, int64_t *hist, double *out) {
  if (!c || !out || (nbins > 0 && !hist)) return LBM_ERR_ARG;
  if (nbins < 0 || nbins > kMaxCurvBins || !(kmax > kmin)) return LBM_ERR_ARG;
  if (!c->initialised) return LBM_ERR_STATE;
  if (!c->curv_hist) {
    cudaError_t e = cudaMalloc(&c->curv_hist, sizeof(unsigned long long) * kMaxCurvBins);
    if (e == cudaSuccess) e = cudaMalloc(&c->curv_part, sizeof(double) * (2 * kReduceBlocks + 2));
    if (e != cudaSuccess) {
      cudaFree(c->curv_hist);
      c->curv_hist = nullptr;
      c->curv_part = nullptr;
      return from_cuda(e);
    }
  }
  double *res = c->curv_part + 2 * kReduceBlocks;
  int rc = from_cuda(timed(c, LBM_K_REDUCE, [&] {
    return launch_curvature(c->P.dim, c->K, c->phi[c->pcur], c->nrm, (float)kmin, (float)kmax, nbins > 0 ? nbins : 1,
                            c->curv_hist, c->curv_part, res, c->stream);
  }, 3));
  if (rc) return rc;
  double r[2];
  if ((rc = d2h(c, r, res, sizeof(r)))) return rc;
  if (nbins > 0 && (rc = d2h(c, hist, c->curv_hist, sizeof(int64_t) * nbins))) return rc;
  if ((rc = sync(c))) return rc;
  out[0] = r[0];
  out[1] = r[0] > 0.0 ? r[1] / r[0] : 0.0;
  return LBM_OK;
}

int lbm_energy_spectrum(lbm_ctx *c, int nshells, double *E) {
  if (!c || !E || nshells < 1 || nshells > kMaxSpectrumShells) return LBM_ERR_ARG;
  if (!c->initialised) return LBM_ERR_STATE;
  int rc = run_moments(c);
  if (rc) return rc;
  if ((rc = ensure_stage(c, sizeof(double) * nshells))) return rc;
  const int r = spectrum_compute(c->K, c->phi[c->pcur], c->mom, nshells, c->stage, c->stream);
  if (r == 1) return LBM_ERR_ARG;
  if (r) return LBM_ERR_CUDA;
  if ((rc = d2h(c, E, c->stage, sizeof(double) * nshells))) return rc;
  return sync(c);
}

int lbm_synchronize(lbm_ctx *c) {
  if (!c) return LBM_ERR_ARG;
  return sync(c);
}

int lbm_profile(lbm_ctx *c, int enable) { return lbm_profile_kinds(c, enable ? ~0u : 0u); }

int lbm_profile_kinds(lbm_ctx *c, unsigned mask) {
  if (!c) return LBM_ERR_ARG;
  int rc = sync(c);
  if (rc) return rc;
  for (auto &pp : c->pairs) {
    c->pool.push_back(pp.a);
    c->pool.push_back(pp.b);
  }
  c->pairs.clear();
  for (int k = 0; k < LBM_K_COUNT; k++) {
    c->prof_ms[k] = 0;
    c->prof_n[k] = 0;
    c->prof_seen[k] = 0;
  }
  c->prof_mask = mask & ((1u << LBM_K_COUNT) - 1u);
  c->prof = c->prof_mask != 0;
  return LBM_OK;
}

int lbm_profile_sample(lbm_ctx *c, int every) {
  if (!c || every < 1) return LBM_ERR_ARG;
  c->prof_every = every;
  return LBM_OK;
}

int lbm_profile_read(lbm_ctx *c, double *ms, int64_t *launches) {
  if (!c) return LBM_ERR_ARG;
  int rc = sync(c);
  if (rc) return rc;
  for (auto &pp : c->pairs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pp.a, pp.b) == cudaSuccess) c->prof_ms[pp.kind] += t;
    c->prof_n[pp.kind] += pp.kernels;
    c->pool.push_back(pp.a);
    c->pool.push_back(pp.b);
  }
  c->pairs.clear();
  for (int k = 0; k < LBM_K_COUNT; k++) {
    if (ms) ms[k] = c->prof_ms[k];
    if (launches) launches[k] = c->prof_n[k];
  }
  return LBM_OK;
}

int lbm_lattice(int dim, int Q, int *c, double *w) {
  if (!c || !w) return LBM_ERR_ARG;
  auto fill = [&](auto L) {
    using LT = decltype(L);
    for (int i = 0; i < LT::Q; i++) {
      for (int a = 0; a < 3; a++) c[3 * i + a] = LT::c(i, a);
      w[i] = LT::wd(i);
    }
  };
  if (dim == 2 && Q == 9) fill(D2Q9{});
  else if (dim == 3 && Q == 19) fill(D3Q19{});
  else if (dim == 3 && Q == 27) fill(D3Q27{});
  else return LBM_ERR_ARG;
  return LBM_OK;
}

const char *lbm_strerror(int s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "device out of memory";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_UNSTABLE: return "unstable: non-finite velocity or phi-mass drift above tolerance";
    case LBM_ERR_STATE: return "call out of order (no state initialised)";
    default: return "unknown status";
  }
}

const char *lbm_kernel_name(int kind) {
  switch (kind) {
    case LBM_K_NCI: return "nci";
    case LBM_K_HYDRO: return "hydro";
    case LBM_K_PHASE: return "phase";
    case LBM_K_REDUCE: return "reduce";
    case LBM_K_CONVERT: return "convert";
    default: return "unknown";
  }
}

}  // extern "C"
