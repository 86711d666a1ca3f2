// ctx.h -- the context behind the opaque lbm_ctx handle of include/lbm.h (internal to the library).
#pragma once

#include <vector>

#include "../../include/lbm.h"
#include "launch.h"

struct ProfPair {
  int kind;
  int kernels;  // kernel launches between the two events
  cudaEvent_t a, b;
};

struct lbm_ctx {
  lbm_params P;
  lbm::KParams K;
  lbm::NciTable T;
  long long N;
  size_t pop_bytes;
  cudaStream_t stream = nullptr;
  int device = 0;
  void *pop[2] = {nullptr, nullptr};
  int32_t *phi[2] = {nullptr, nullptr};
  float *u = nullptr;
  float4 *frep = nullptr;
  float4 *nrm = nullptr;  // interface normals at gated cells
  float *mom = nullptr;
  double *stage = nullptr;
  size_t stage_bytes = 0;
  int32_t *partner = nullptr;
  int *tiles[2] = {nullptr, nullptr};
  int *ntiles = nullptr;  // 2 counters, one per phi buffer
  int *lflag = nullptr;   // 2 x ntile marks: tile listed for phi[k] (3D)
  int ntile = 0;          // near-contact tiles of the grid
  lbm::NciAux aux;        // near-contact prefilter buffers (3D grids with sides multiple of 4)
  int nci_blocks = 0;
  // the split step: the near-contact pass and the hydrodynamic update of the listed tiles on the
  // high-priority stream `side`, concurrent with the hydrodynamic update of the other tiles
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int overlap_blocks = 0;  // resident near-contact scan blocks while split; 0: one stream
  int split_blocks = 0;    // blocks of the listed-tile hydrodynamic launch
  lbm::ReduceOut *red_part = nullptr, *red_out = nullptr;
  lbm::DiagOut *diag_part = nullptr, *diag_out = nullptr;  // film statistics, on first use
  unsigned long long *curv_hist = nullptr;  // curvature histogram (kMaxCurvBins), on first use
  double *curv_part = nullptr;              // 2 per reduction block + 2 for the result
  int cur = 0;        // population buffer holding the current state
  int pcur = 0;       // phi buffer holding phi^n
  bool initialised = false;
  long long steps = 0;
  long long phi_q30_ref = 0;
  // profiler
  bool prof = false;
  unsigned prof_mask = 0;  // kinds timed while prof is on
  std::vector<ProfPair> pairs;
  std::vector<cudaEvent_t> pool;
  double prof_ms[LBM_K_COUNT] = {0};
  int64_t prof_n[LBM_K_COUNT] = {0};
  int64_t prof_seen[LBM_K_COUNT] = {0};  // passes of each kind since the profiler was (re)started
  int prof_every = 1;                    // time one pass in every prof_every of each kind
};

// The near-contact list of phi buffer k.
inline lbm::TileList tile_list(const lbm_ctx *c, int k) {
  lbm::TileList t;
  t.tiles = c->tiles[k];
  t.count = c->ntiles + k;
  t.mark = c->lflag + (size_t)k * (size_t)c->ntile;
  return t;
}

// The prefilter buffers of the near-contact pass over listed tiles, or nullptr where it does not apply.
inline const lbm::NciAux *nci_aux(const lbm_ctx *c) { return c->aux.bricks ? &c->aux : nullptr; }
// Kernels of one near-contact pass over the listed tiles: normals, prefilter (where it applies), scan.
inline int nci_list_kernels(const lbm_ctx *c) { return nci_aux(c) ? 3 : 2; }

// Enqueues one step of c on stream s from buffers (cur, pcur) (lbm_api.cu); lists = false leaves the
// near-contact lists as they are. Returns an lbm_status.
int enqueue_step(lbm_ctx *c, int cur, int pcur, bool lists, cudaStream_t s);

// Looks up (once per device, current device) the static scratch of lbm_mass_noalloc, which loads
// its module; lbm_create calls it. Returns an lbm_status.
int lbm_noalloc_prepare_device();

