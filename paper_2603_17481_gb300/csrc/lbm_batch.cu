// lbm_batch.cu -- many independent contexts advanced together (the sweep of uneven collision
// cases; the paper runs one case at a time).
//
// Two steps of every context are captured into one CUDA graph (two, because the population and
// phi buffers ping-pong and return to the same parity), launched on one stream. The graph holds,
// per step,
//   fused mode (every context 3D, one lattice and one store type, nx even, Q N <= 2^32):
//     the near-contact pass of every context on concurrent stream branches, then ONE launch of
//     the paired hydrodynamic kernel and ONE launch of the phase march, each a persistent grid
//     walking a work list that concatenates every case (batch_kernels.cu);
//   per-case mode (otherwise, or on request): every context's step on concurrent branches.
// When the batch can fuse, an autotuner picks, on the batch itself, the hydrodynamic tile shape
// (64 x ty x tz cells, ty in {4, 2, 8}) and the rows of y per thread of the phase march (4 or 2)
// by timing each candidate pass over the whole batch, then times one step of the tuned fused
// execution against one step of the per-case graph and keeps the faster. Everything it times
// writes only the next-step buffers and per-step scratch (near-contact list updates off), so the
// contexts' state is unchanged. The choices and the times are reported by lbm_batch_config.
//
// A graph bakes in the buffers of the parity it was captured from. An odd step count ends with one
// plain step per context, which flips every context's parity, so a second graph is captured from
// the flipped parity and each launch picks the graph whose parity the contexts hold.
#include <algorithm>
#include <vector>

#include "ctx.h"

using namespace lbm;

struct lbm_batch {
  std::vector<lbm_ctx *> ctxs;
  std::vector<cudaStream_t> branches;
  std::vector<cudaEvent_t> joins;
  cudaStream_t stream = nullptr;  // capture stream
  cudaStream_t launch = nullptr;  // graph launches go here (the caller's stream, else `stream`)
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};     // [0]: parity at creation, [1]: flipped
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::vector<int> cur0, pcur0;                  // each context's (cur, pcur) at creation
  // fused mode
  bool fused = false;
  int Q = 0, store = 0;
  BatchCase *d_cases = nullptr;  // [3][n]: parity 0, parity 1, tuning (no list updates)
  int4 *d_items = nullptr;
  int nitems = 0;
  long long *d_uoff = nullptr;
  int hydro_ty = 4, phase_rows = 4, hydro_blocks = 0, phase_blocks = 0;
  // tuner times: hydro ty 4, 2, 8 and phase rows 4, 2 (ms per pass); one dry step of the fused
  // candidate and of the per-case graph
  double tune_ms[7] = {0, 0, 0, 0, 0, 0, 0};
};

namespace {
constexpr double kFusedMargin = 0.97;  // the fused mode's dry step against the per-case graph's

int from_cuda_b(cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  if (e == cudaErrorMemoryAllocation) return LBM_ERR_OOM;
  return LBM_ERR_CUDA;
}

bool fusable(lbm_ctx *const *ctxs, int n) {
  const lbm_params &p0 = ctxs[0]->P;
  for (int i = 0; i < n; i++) {
    const lbm_params &p = ctxs[i]->P;
    if (p.dim != 3 || p.Q != p0.Q || p.store != p0.store || p.nx % 2 != 0) return false;
    if (p.store == LBM_STORE_MOMENTS) return false;  // the batched kernel stores populations
    if ((long long)p.Q * ctxs[i]->N > (1LL << 32)) return false;
  }
  return true;
}

// The near-contact pass of context c on phi[pc] (the list of that buffer), on stream s.
cudaError_t nci_pass(lbm_ctx *c, int pc, cudaStream_t s) {
  return launch_nci(c->P.dim, c->K, c->T, c->phi[pc], c->nrm, c->frep, nullptr, 0, c->tiles[pc], c->ntiles + pc,
                    c->nci_blocks, s, nci_aux(c), c->ntiles + (pc ^ 1));
}

// BatchCase of context c for a step from buffer parity (cur, pcur); lists = false leaves the
// near-contact lists untouched (tuning passes).
BatchCase batch_case(lbm_ctx *c, int cur, int pcur, bool lists) {
  BatchCase b{};
  b.P = c->K;
  b.src = c->pop[cur];
  b.dst = c->pop[cur ^ 1];
  b.phi = c->phi[pcur];
  b.phi_out = c->phi[pcur ^ 1];
  b.frep = c->frep;
  b.u = c->u;
  const bool nci = lists && c->P.nci_on;
  if (nci) {
    b.next = tile_list(c, pcur ^ 1);
    b.prev = tile_list(c, pcur);
  }
  b.ncx = (c->P.nx + March3::OUT - 1) / March3::OUT;
  return b;
}

int upload_cases(lbm_batch *b) {
  const int n = (int)b->ctxs.size();
  std::vector<BatchCase> h(3 * (size_t)n);
  for (int i = 0; i < n; i++) {
    lbm_ctx *c = b->ctxs[i];
    h[i] = batch_case(c, b->cur0[i], b->pcur0[i], true);
    h[n + i] = batch_case(c, b->cur0[i] ^ 1, b->pcur0[i] ^ 1, true);
    h[2 * n + i] = batch_case(c, b->cur0[i], b->pcur0[i], false);
  }
  return from_cuda_b(cudaMemcpy(b->d_cases, h.data(), sizeof(BatchCase) * h.size(), cudaMemcpyHostToDevice));
}

// (case, bx, by, bz) items of the hydrodynamic pass for tiles of 64 x ty x (8 / ty) cells
int upload_items(lbm_batch *b, int ty) {
  std::vector<int4> items;
  const int tz = 8 / ty;
  for (int i = 0; i < (int)b->ctxs.size(); i++) {
    const lbm_params &p = b->ctxs[i]->P;
    for (int bz = 0; bz < (p.nz + tz - 1) / tz; bz++)
      for (int by = 0; by < (p.ny + ty - 1) / ty; by++)
        for (int bx = 0; bx < (p.nx + 63) / 64; bx++) items.push_back(make_int4(i, bx, by, bz));
  }
  b->nitems = (int)items.size();
  return from_cuda_b(cudaMemcpy(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
}

size_t max_items(lbm_batch *b) {
  size_t m = 0;
  for (int ty : {4, 2, 8}) {
    size_t s = 0;
    for (lbm_ctx *c : b->ctxs) {
      const lbm_params &p = c->P;
      s += (size_t)((p.nx + 63) / 64) * ((p.ny + ty - 1) / ty) * ((p.nz + 8 / ty - 1) / (8 / ty));
    }
    m = std::max(m, s);
  }
  return m;
}

// unit offsets of the phase march with `rows` rows of y per thread
int upload_uoff(lbm_batch *b, int rows) {
  const int n = (int)b->ctxs.size();
  std::vector<long long> off(n + 1, 0);
  for (int i = 0; i < n; i++) {
    const lbm_params &p = b->ctxs[i]->P;
    off[i + 1] = off[i] + (long long)((p.nx + March3::OUT - 1) / March3::OUT) * ((p.ny + rows - 1) / rows) * p.nz;
  }
  return from_cuda_b(cudaMemcpy(b->d_uoff, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice));
}

int phase_blocks_for(lbm_batch *b, int rows) {
  long long units = 0;
  for (lbm_ctx *c : b->ctxs) {
    const lbm_params &p = c->P;
    units += (long long)((p.nx + March3::OUT - 1) / March3::OUT) * ((p.ny + rows - 1) / rows) * p.nz;
  }
  const long long want = (units + March3::MIN_RUN * March3::WARPS - 1) / (March3::MIN_RUN * March3::WARPS);
  return (int)std::max(1LL, std::min<long long>(want, phase_batch_blocks(rows)));
}

// Mean milliseconds of `reps` launches of f on the batch stream (after one untimed launch).
template <class F> int time_ms(lbm_batch *b, F &&f, int reps, double &ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
  for (int r = 0; r < reps && e == cudaSuccess; r++) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  ms = t / reps;
  return from_cuda_b(e);
}

// Mean milliseconds of a graph of one dry step of every context from parity 0: the near-contact
// pass, then (fused) the batched hydrodynamic and phase-field passes on the tuning table, or (per
// case) each context's own hydrodynamic and phase-field kernels on its branch, with the
// near-contact list updates off. It writes only the next-step buffers and the per-step scratch.
int time_dry_step(lbm_batch *b, bool fused, double &ms) {
  const int n = (int)b->ctxs.size();
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
  for (size_t s = 0; s < b->branches.size() && e == cudaSuccess; s++) e = cudaStreamWaitEvent(b->branches[s], b->fork, 0);
  for (int i = 0; i < n && e == cudaSuccess; i++) {
    lbm_ctx *c = b->ctxs[i];
    const cudaStream_t br = b->branches[i % b->branches.size()];
    const int cur = b->cur0[i], pc = b->pcur0[i];
    if (fused) {
      if (c->P.nci_on) e = nci_pass(c, pc, br);
    } else if (enqueue_step(c, cur, pc, false, br) != LBM_OK) {
      e = cudaErrorUnknown;
    }
  }
  for (size_t s = 0; s < b->branches.size() && e == cudaSuccess; s++) {
    e = cudaEventRecord(b->joins[s], b->branches[s]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->joins[s], 0);
  }
  if (fused && e == cudaSuccess) {
    const BatchCase *tune = b->d_cases + 2 * n;
    e = launch_hydro_batch(b->Q, b->store, b->hydro_ty, tune, b->d_items, b->nitems, b->hydro_blocks, b->stream);
    if (e == cudaSuccess) e = launch_phase_batch(b->phase_rows, tune, b->d_uoff, n, b->phase_blocks, b->stream);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess) e = ee;
  cudaGraphExec_t x = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
  int rc = from_cuda_b(e);
  if (rc == LBM_OK) rc = time_ms(b, [&] { return cudaGraphLaunch(x, b->stream); }, 3, ms);
  if (x) cudaGraphExecDestroy(x);
  if (g) cudaGraphDestroy(g);
  return rc;
}

// Times the candidates on the tuning copy of parity 0 and keeps the fastest of each pass, then
// the faster of the fused and the per-case execution.
int autotune(lbm_batch *b) {
  const int n = (int)b->ctxs.size();
  const BatchCase *tune = b->d_cases + 2 * n;
  int rc;
  const int tys[3] = {4, 2, 8};
  double best = 1e30;
  for (int k = 0; k < 3; k++) {
    const int ty = tys[k];
    if ((rc = upload_items(b, ty))) return rc;
    double ms = 0;
    rc = time_ms(b, [&] { return launch_hydro_batch(b->Q, b->store, ty, tune, b->d_items, b->nitems, b->hydro_blocks,
                                                    b->stream); }, 3, ms);
    if (rc) return rc;
    b->tune_ms[k] = ms;
    if (ms < best) { best = ms; b->hydro_ty = ty; }
  }
  best = 1e30;
  const int rowss[2] = {4, 2};
  for (int k = 0; k < 2; k++) {
    const int rows = rowss[k];
    if ((rc = upload_uoff(b, rows))) return rc;
    double ms = 0;
    const int blocks = phase_blocks_for(b, rows);
    rc = time_ms(b, [&] { return launch_phase_batch(rows, tune, b->d_uoff, n, blocks, b->stream); }, 3, ms);
    if (rc) return rc;
    b->tune_ms[3 + k] = ms;
    if (ms < best) { best = ms; b->phase_rows = rows; }
  }
  // the chosen configuration's tables
  if ((rc = upload_items(b, b->hydro_ty)) || (rc = upload_uoff(b, b->phase_rows))) return rc;
  b->phase_blocks = phase_blocks_for(b, b->phase_rows);
  // the execution mode: one dry step of the whole batch, fused and per case, each captured in a
  // graph on the branches. The fused mode is kept only when its dry step is at least 3 % faster:
  // in the real two-step graphs it joins every case twice per step, and on the 128-case sweep its
  // steps ran 6-7 % slower against the per-case graph than the dry steps (0.5 % apart) predicted.
  double ms_fused = 0, ms_case = 0;
  if ((rc = time_dry_step(b, true, ms_fused)) || (rc = time_dry_step(b, false, ms_case))) return rc;
  b->tune_ms[5] = ms_fused;
  b->tune_ms[6] = ms_case;
  b->fused = ms_fused < kFusedMargin * ms_case;
  return LBM_OK;
}

// Records the steps of graph g (two steps from parity g) into the capture stream.
int capture_steps(lbm_batch *b, int g) {
  const int n = (int)b->ctxs.size();
  cudaError_t e = cudaSuccess;
  int rc = LBM_OK;
  for (int st = 0; st < 2 && e == cudaSuccess && rc == LBM_OK; st++) {
    const int q = g ^ st;  // parity of this step relative to creation
    e = cudaEventRecord(b->fork, b->stream);
    for (size_t s = 0; s < b->branches.size() && e == cudaSuccess; s++) e = cudaStreamWaitEvent(b->branches[s], b->fork, 0);
    for (int i = 0; i < n && e == cudaSuccess && rc == LBM_OK; i++) {
      lbm_ctx *c = b->ctxs[i];
      const cudaStream_t br = b->branches[i % b->branches.size()];
      if (b->fused) {
        if (c->P.nci_on) e = nci_pass(c, b->pcur0[i] ^ q, br);
      } else {
        rc = enqueue_step(c, b->cur0[i] ^ q, b->pcur0[i] ^ q, true, br);
      }
    }
    for (size_t s = 0; s < b->branches.size() && e == cudaSuccess; s++) {
      e = cudaEventRecord(b->joins[s], b->branches[s]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->joins[s], 0);
    }
    if (b->fused && e == cudaSuccess) {
      const BatchCase *tab = b->d_cases + (size_t)q * n;
      e = launch_hydro_batch(b->Q, b->store, b->hydro_ty, tab, b->d_items, b->nitems, b->hydro_blocks, b->stream);
      if (e == cudaSuccess) e = launch_phase_batch(b->phase_rows, tab, b->d_uoff, n, b->phase_blocks, b->stream);
    }
  }
  return rc != LBM_OK ? rc : from_cuda_b(e);
}
}  // namespace

extern "C" void lbm_batch_destroy(lbm_batch *b) {
  if (!b) return;
  if (b->launch) cudaStreamSynchronize(b->launch);
  for (int g = 0; g < 2; g++) {
    if (b->exec[g]) cudaGraphExecDestroy(b->exec[g]);
    if (b->graph[g]) cudaGraphDestroy(b->graph[g]);
  }
  for (auto e : b->joins) cudaEventDestroy(e);
  for (auto s : b->branches) cudaStreamDestroy(s);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->stream) cudaStreamDestroy(b->stream);
  cudaFree(b->d_cases);
  cudaFree(b->d_items);
  cudaFree(b->d_uoff);
  delete b;
}

extern "C" int lbm_batch_create_ex(lbm_ctx *const *ctxs, int n, int nstreams, void *stream, int flags,
                                   lbm_batch **out) {
  const int known = LBM_BATCH_PER_CASE | LBM_BATCH_NO_TUNE | LBM_BATCH_HYDRO_TY2 | LBM_BATCH_HYDRO_TY8 |
                    LBM_BATCH_PHASE_ROWS2;
  if (!ctxs || n < 1 || nstreams < 1 || !out || (flags & ~known)) return LBM_ERR_ARG;
  if ((flags & LBM_BATCH_HYDRO_TY2) && (flags & LBM_BATCH_HYDRO_TY8)) return LBM_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
  for (int i = 0; i < n; i++) {
    lbm_ctx *c = ctxs[i];
    if (!c) return LBM_ERR_ARG;
    if (!c->initialised) return LBM_ERR_STATE;
    if (c->P.mass_check_every != 0 || c->prof || c->device != dev) return LBM_ERR_ARG;
    for (int j = 0; j < i; j++)
      if (ctxs[j] == c) return LBM_ERR_ARG;
  }
  lbm_batch *b = new lbm_batch();
  b->ctxs.assign(ctxs, ctxs + n);
  if (nstreams > n) nstreams = n;
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  b->launch = stream ? (cudaStream_t)stream : b->stream;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int s = 0; s < nstreams && e == cudaSuccess; s++) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branches.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->joins.push_back(ev);
  }
  // the contexts' pending work must be complete before their streams are swapped out
  for (int i = 0; i < n && e == cudaSuccess; i++) e = cudaStreamSynchronize(ctxs[i]->stream);
  if (e != cudaSuccess) {
    lbm_batch_destroy(b);
    return from_cuda_b(e);
  }
  for (int i = 0; i < n; i++) {
    b->cur0.push_back(ctxs[i]->cur);
    b->pcur0.push_back(ctxs[i]->pcur);
  }
  int rc = LBM_OK;
  b->fused = !(flags & LBM_BATCH_PER_CASE) && fusable(ctxs, n);
  if (b->fused) {
    b->Q = ctxs[0]->P.Q;
    b->store = ctxs[0]->P.store;
    b->hydro_blocks = hydro_batch_blocks(b->Q, b->store, 4);
    e = cudaMalloc(&b->d_cases, sizeof(BatchCase) * 3 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int4) * max_items(b));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_uoff, sizeof(long long) * (n + 1));
    rc = from_cuda_b(e);
    if (rc == LBM_OK && b->hydro_blocks <= 0) rc = LBM_ERR_CUDA;
    if (rc == LBM_OK) rc = upload_cases(b);
    if (rc == LBM_OK) {
      const int pin = LBM_BATCH_NO_TUNE | LBM_BATCH_HYDRO_TY2 | LBM_BATCH_HYDRO_TY8 | LBM_BATCH_PHASE_ROWS2;
      if (flags & pin) {
        b->hydro_ty = (flags & LBM_BATCH_HYDRO_TY2) ? 2 : ((flags & LBM_BATCH_HYDRO_TY8) ? 8 : 4);
        b->phase_rows = (flags & LBM_BATCH_PHASE_ROWS2) ? 2 : 4;
        rc = upload_items(b, b->hydro_ty);
        if (rc == LBM_OK) rc = upload_uoff(b, b->phase_rows);
        b->phase_blocks = phase_blocks_for(b, b->phase_rows);
      } else {
        rc = autotune(b);
      }
    }
    if (rc != LBM_OK) {
      lbm_batch_destroy(b);
      return rc;
    }
  }
  // capture two steps of every context, once from the current parity and once from the flipped one
  for (int g = 0; g < 2 && e == cudaSuccess; g++) {
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) rc = capture_steps(b, g);
    cudaGraph_t gr = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &gr);
    if (e == cudaSuccess) e = ee;
    b->graph[g] = gr;
    if (e == cudaSuccess && rc == LBM_OK) e = cudaGraphInstantiate(&b->exec[g], b->graph[g], 0);
    if (e != cudaSuccess || rc != LBM_OK) {
      lbm_batch_destroy(b);
      return rc != LBM_OK ? rc : from_cuda_b(e);
    }
  }
  *out = b;
  return LBM_OK;
}

extern "C" int lbm_batch_create(lbm_ctx *const *ctxs, int n, int nstreams, void *stream, lbm_batch **out) {
  return lbm_batch_create_ex(ctxs, n, nstreams, stream, 0, out);
}

extern "C" int lbm_batch_config(const lbm_batch *b, int *cfg, double *ms) {
  if (!b) return LBM_ERR_ARG;
  if (cfg) {
    cfg[0] = b->fused ? 1 : 0;
    cfg[1] = b->hydro_ty;
    cfg[2] = 8 / b->hydro_ty;
    cfg[3] = b->phase_rows;
    cfg[4] = (int)b->branches.size();
    cfg[5] = b->hydro_blocks;
    cfg[6] = b->phase_blocks;
    cfg[7] = b->nitems;
  }
  if (ms)
    for (int k = 0; k < 7; k++) ms[k] = b->tune_ms[k];
  return LBM_OK;
}

extern "C" int lbm_batch_step(lbm_batch *b, int nsteps) {
  if (!b || nsteps < 0) return LBM_ERR_ARG;
  // the graph whose buffers are the ones every context currently holds
  int g = -1;
  for (size_t i = 0; i < b->ctxs.size(); i++) {
    const lbm_ctx *c = b->ctxs[i];
    const int gi = (c->cur == b->cur0[i] && c->pcur == b->pcur0[i]) ? 0
                 : (c->cur == (b->cur0[i] ^ 1) && c->pcur == (b->pcur0[i] ^ 1)) ? 1 : -1;
    if (gi < 0 || (g >= 0 && gi != g)) return LBM_ERR_STATE;
    g = gi;
  }
  cudaError_t e = cudaSuccess;
  for (int k = 0; k + 1 < nsteps && e == cudaSuccess; k += 2) e = cudaGraphLaunch(b->exec[g], b->launch);
  if (e != cudaSuccess) return from_cuda_b(e);
  for (lbm_ctx *c : b->ctxs) c->steps += nsteps - (nsteps & 1);
  if (nsteps & 1) {
    // the odd last step: each context's plain step, issued on the launch stream after the graph
    for (lbm_ctx *c : b->ctxs) {
      const cudaStream_t saved = c->stream;
      c->stream = b->launch;
      const int rc = lbm_step(c, 1);
      c->stream = saved;
      if (rc) return rc;
    }
  }
  return LBM_OK;
}

extern "C" int lbm_batch_synchronize(lbm_batch *b) {
  if (!b) return LBM_ERR_ARG;
  return from_cuda_b(cudaStreamSynchronize(b->launch));
}
