// lbm_batch.cu -- many independent contexts advanced together through one CUDA graph.
//
// A batch captures two time steps of every context into one graph: the contexts are spread over
// concurrent stream branches forked from a capture stream and joined back into it, so one graph
// launch advances every case by two steps (two, because the population and phi buffers ping-pong
// and return to the same parity). Small cases then fill the GPU together instead of one after the
// other, and the per-kernel launch cost is paid once per graph.
//
// A graph bakes in the buffers of the parity it was captured from. An odd step count ends with one
// plain step per context, which flips every context's parity, so a second graph is captured from
// the flipped parity and each launch picks the graph whose parity the contexts hold.
#include <vector>

#include "ctx.h"

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
};

namespace {
int from_cuda_b(cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  if (e == cudaErrorMemoryAllocation) return LBM_ERR_OOM;
  return LBM_ERR_CUDA;
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
  delete b;
}

extern "C" int lbm_batch_create(lbm_ctx *const *ctxs, int n, int nstreams, void *stream, lbm_batch **out) {
  if (!ctxs || n < 1 || nstreams < 1 || !out) return LBM_ERR_ARG;
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
  // capture two steps of every context, once from the current parity and once from the flipped one
  for (int g = 0; g < 2 && e == cudaSuccess; g++) {
    int rc = LBM_OK;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    for (size_t s = 0; s < b->branches.size() && e == cudaSuccess; s++) e = cudaStreamWaitEvent(b->branches[s], b->fork, 0);
    for (int i = 0; i < n && e == cudaSuccess && rc == LBM_OK; i++) {
      lbm_ctx *c = ctxs[i];
      const cudaStream_t saved = c->stream;
      const long long steps = c->steps;
      c->stream = b->branches[i % b->branches.size()];
      c->cur = b->cur0[i] ^ g;
      c->pcur = b->pcur0[i] ^ g;
      rc = lbm_step(c, 2);
      c->stream = saved;
      c->cur = b->cur0[i];  // capture runs nothing: the contexts keep their state
      c->pcur = b->pcur0[i];
      c->steps = steps;
    }
    for (size_t s = 0; s < b->branches.size() && e == cudaSuccess; s++) {
      e = cudaEventRecord(b->joins[s], b->branches[s]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->joins[s], 0);
    }
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
  if (e != cudaSuccess) {
    lbm_batch_destroy(b);
    return from_cuda_b(e);
  }
  *out = b;
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
