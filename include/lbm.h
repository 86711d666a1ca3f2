/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for one time step of the conservative Allen-Cahn
 * phase-field lattice Boltzmann model with adaptive near-contact repulsion of arXiv 2603.17481.
 *
 * One step advances, on a fully periodic box,
 *   (1) the near-contact interaction: interfacial gate, bounded-window partner search and the
 *       closed-form proximity indicator / repulsive force (Sec. 2.3, Eqs. 57-73);
 *   (2) the thread-safe recursive-regularized lattice Boltzmann hydrodynamics with Guo forcing and
 *       the force split F = F_sigma + F_p + F_nu + F_rep + F_ext (Sec. 2.1, Eqs. 3-23), as a pull
 *       scheme over structure-of-arrays populations;
 *   (3) the conservative Allen-Cahn phase field phi^{n+1} = phi^n - div(u phi) + D lap(phi) + S_comp
 *       with MUSCL-minmod advection and isotropic stencils (Sec. 2.1.1, Eqs. 24-35),
 * in that order: the hydrodynamics at step n uses phi^n and produces u^n, which advects phi^n.
 *
 * Conventions shared by every call:
 *   - cell index n = x + nx*(y + ny*z), x fastest; nz = 1 when dim = 2.
 *   - host arrays are FP64, owned by the caller, read or written only during the call.
 *   - vector fields are structure-of-arrays with 3 rows: v[a*N + n], a = 0..2 (the z row is
 *     ignored on input and written as 0 on output when dim = 2).
 *   - populations f[i*N + n] are the PRE-collision populations of the current step at cell n.
 *   - velocity order i = 0..Q-1: sorted by |c|^2 ascending, ties by (c_z, c_y, c_x) in
 *     lexicographic order with -1 < 0 < +1 (lbm_lattice() returns the table).
 *   - phi = 1 in the liquid, 0 in the gas; density rho(phi) = rho_g + (rho_l - rho_g) phi; the
 *     normalised pressure p* gives the pressure p = rho c_s^2 p* (Eq. 5), c_s^2 = 1/3.
 *   - every entry point returns LBM_OK (0) or a negative lbm_status; none aborts, exits or traps.
 *     After LBM_ERR_CUDA the context must be destroyed.
 *   - calls on one context are not thread-safe; different contexts are independent.
 *   - the library owns all device memory of a context (allocated in lbm_create / on first use).
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,      /* invalid argument or parameter set                                   */
  LBM_ERR_OOM = -2,      /* device memory allocation failed                                     */
  LBM_ERR_CUDA = -3,     /* CUDA runtime error (no device, launch or copy failure)              */
  LBM_ERR_UNSTABLE = -4, /* periodic check found NaN/Inf or a phi-mass drift above mass_tol     */
  LBM_ERR_STATE = -5     /* call out of order (e.g. lbm_step before lbm_init_fields)            */
} lbm_status;

typedef enum {
  LBM_STORE_F32 = 0,  /* populations stored as FP32                                             */
  LBM_STORE_F16 = 1,  /* populations stored as FP16, f_i / w_i (deviation from rest, p* = 0)    */
  LBM_STORE_BF16 = 2, /* populations stored as BF16, f_i / w_i                                  */
  LBM_STORE_MOMENTS = 3 /* 3D only: per cell the FP32 record of its post-collision state (the     */
                      /* thread-safe moment representation of Sec. 2.1): p*, u, F / rho and the  */
                      /* relaxed regularized A2 of Eq. 14, as 16 floats (64 B instead of 4 Q B); */
                      /* a cell pulls f_i by evaluating Eqs. 11, 15-17 and the Guo term at the    */
                      /* record of x - c_i. lbm_init_fields stores the record of f_eq(p*, u) at   */
                      /* every cell, so the first step pulls f_eq_i of x - c_i; lbm_set_state is  */
                      /* refused (LBM_ERR_STATE): arbitrary populations have no record form.      */
} lbm_store;

/* Kernel kinds reported by the profiler (lbm_profile_read). */
typedef enum {
  LBM_K_NCI = 0, LBM_K_HYDRO = 1, LBM_K_PHASE = 2, LBM_K_REDUCE = 3, LBM_K_CONVERT = 4,
  LBM_K_COUNT = 5
} lbm_kernel_kind;

typedef struct {
  int dim;            /* 2 or 3                                                                 */
  int nx, ny, nz;     /* periodic box; nz = 1 when dim = 2                                     */
  int Q;              /* hydrodynamic lattice: 9 (dim 2), 19 or 27 (dim 3)                      */
  int store;          /* lbm_store                                                              */
  double rho_l, rho_g;/* liquid / gas densities (> 0)                                           */
  double nu_l, nu_g;  /* kinematic viscosities (> 0); dynamic viscosity mixes linearly (Eq. 8)  */
  double sigma;       /* surface tension; chemical potential 4 beta phi(phi-1)(phi-1/2) - k lap */
                      /* phi with beta = 12 sigma / eps, k = 3 sigma eps / 2 (Eq. 19)           */
  double eps;         /* interface width epsilon (> 0): tanh profile width, kappa = 4 D / eps  */
                      /* (Eq. 26), proximity indicator scale (Eq. 70)                            */
  double D;           /* phase-field diffusivity (>= 0), tau_diff of Eq. 28                     */
  int nci_on;         /* near-contact interaction on (1) / off (0)                              */
  int w;              /* search-window radius, 1..3 (Eq. 60; paper: 3)                          */
  double A_rep;       /* repulsion amplitude (Eq. 72; paper: O(sigma))                          */
  double h0, p;       /* thickness weight 1/(1+(h/h0)^p) (Eq. 42; paper: h0 = 1, p = 4)        */
  double q_th;        /* interfacial gate (Eq. 59; paper 0.125)                                 */
  double eta;         /* iso-interface tolerance (Eq. 61; paper 0.1)                            */
  double cos_opp;     /* facing threshold (Eq. 62; paper -0.8)                                  */
  double eps_q, eps_n;/* floors of Eq. 67 and of the normal grad/(|grad| + eps_n), Eqs. 25, 57  */
  double g[3];        /* body acceleration; F_ext = (rho - rho_bar) g, rho_bar = mean initial rho */
  int mass_check_every; /* lbm_step runs the FP64 phi-mass / NaN check every this many steps; 0 = off */
  double mass_tol;    /* relative phi-mass drift that makes the check fail                      */
} lbm_params;

/* Fills *p with the paper's near-contact parameters (Sec. 2.3.2, Eq. 71) on a 64^3 D3Q19 box. */
void lbm_params_default(lbm_params *p);

/* Validates *p (LBM_ERR_ARG before any CUDA call), then allocates the device state of a context
 * on the current CUDA device. *out is set only on success. */
int lbm_create(const lbm_params *p, lbm_ctx **out);

/* Frees every device buffer of ctx; ctx may be NULL. */
void lbm_destroy(lbm_ctx *ctx);

/* Kernels and copies of ctx go to this cudaStream_t (NULL = the legacy default stream). Calls
 * still return only after their work is complete, except lbm_step (see below). */
int lbm_set_stream(lbm_ctx *ctx, void *stream);

/* Host arrays of lbm_init_fields and lbm_read_fields: an array that lies in page-locked host
 * memory (cudaHostAlloc, cudaHostRegister; e.g. a pinned torch tensor, or a view into one) is read
 * or written in place by the conversion kernels over the host link; any other host array goes
 * through a device staging buffer (5 N doubles, allocated on first use and kept) with one copy.
 * An output in memory the device may only read (cudaHostRegisterReadOnly) is not stored to by a
 * kernel: it takes the staging route. Either way the call returns only after its last access to
 * the caller's arrays. */

/* Initial state: phi (N), u (3N) and p* (N, or NULL for p* = 0) on the host. Populations become
 * the third-order equilibrium f_eq(p*, u) (Eq. 11, evaluated in FP32); rho_bar is the mean of
 * rho(phi). */
int lbm_init_fields(lbm_ctx *ctx, const double *phi, const double *u, const double *pstar);

/* Full state: pre-collision populations f (Q*N) and phi (N). rho_bar becomes the mean rho(phi). */
int lbm_set_state(lbm_ctx *ctx, const double *f, const double *phi);
/* Reads the full state back (f: Q*N, phi: N; either may be NULL). */
int lbm_get_state(lbm_ctx *ctx, double *f, double *phi);

/* Advances n >= 0 steps. Enqueues the work on the context stream and returns; it synchronises
 * only when the periodic mass check runs (mass_check_every > 0), which may return
 * LBM_ERR_UNSTABLE.
 * A step is the near-contact pass (Sec. 2.3) on phi^n, the hydrodynamic update (Sec. 2.1) and the
 * phase-field update (Sec. 2.1.1), in that order on the context stream. */
int lbm_step(lbm_ctx *ctx, int n);

/* The split step of lbm_step, where it applies (3D, nci_on, nx even, Q N <= 2^32): the
 * near-contact pass and then the hydrodynamic update of the cells of the near-contact tiles listed
 * for phi^n (32 x 8 x 4 tiles holding a cell with q >= q_th) run on a second, high-priority stream
 * of the context, while the context stream updates the other cells, which are not gated and so do
 * not read F_rep (Eq. 73); the streams join before the phase-field update. Each cell is updated by
 * one of the two launches with the same arithmetic, so every state is bit-identical to the
 * one-stream step's. blocks > 0 runs it with that many resident near-contact scan blocks (capped
 * at one per SM); blocks = 0 (the default) runs every step on the context stream alone. Takes
 * effect at the next lbm_step or batch capture. blocks < 0 or NULL ctx: LBM_ERR_ARG; blocks > 0
 * on a context where the split step does not apply: LBM_ERR_STATE. */
int lbm_set_overlap(lbm_ctx *ctx, int blocks);
/* *blocks = the scan blocks of the split step, 0 when every step runs on one stream. */
int lbm_get_overlap(const lbm_ctx *ctx, int *blocks);

/* phi^n (N), the velocity u (3N) and p* (N) of the current state: moments of the pre-collision
 * populations with the forces evaluated on phi^n (Eqs. 6-7, with F_nu from u without F_nu).
 * Any output pointer may be NULL. */
int lbm_read_fields(lbm_ctx *ctx, double *phi, double *u, double *pstar);

/* FP64 integrals of the current state: sum(phi) (exact sum of the stored fixed-point phi) and
 * sum(rho u) (3 values, u as in lbm_read_fields). Either pointer may be NULL. */
int lbm_mass(lbm_ctx *ctx, double *phi_mass, double *mom);

/* The same integrals as lbm_mass without allocating any device memory, for callers that cannot
 * allocate at that moment: a process whose device memory is reserved by another allocator (a
 * framework's caching allocator owning nearly all of HBM), or a latency-critical loop that cannot
 * take cudaMalloc's implicit device synchronisation. The paper has no counterpart; it is a service
 * of this library. The reduction scratch is a fixed static device array (4097 slots of 40 bytes,
 * about 160 KB) that every GPU loading the library holds until the process exits.
 * Limits and errors: at most 16,777,216 cells (one slot per 4096 cells), else LBM_ERR_ARG; the
 * context's device must be current, else LBM_ERR_ARG; the moment buffer must already exist, i.e.
 * lbm_mass or lbm_read_fields ran once on this context, else LBM_ERR_STATE (it is not allocated
 * here). The scratch lives in the library's module, which the CUDA runtime loads lazily: lbm_create
 * looks its address up (cudaGetSymbolAddress) once per device, which loads the module and takes
 * the 160 KB there, while allocating is allowed, so that no later call needs to. Should that
 * look-up fail there, the first lbm_mass_noalloc call on the device repeats it (and then may take
 * the memory itself); make that first call during set-up, before any stream capture. All calls on a device share the scratch:
 * calls whose work overlaps on the GPU (e.g. two contexts on different streams) race, so serialise
 * them. Each call overwrites every slot it reads; nothing needs clearing between calls.
 * Synchronises the context stream. Either output pointer may be NULL. */
int lbm_mass_noalloc(lbm_ctx *ctx, double *phi_mass, double *mom);

/* Near-contact diagnostics on the current phi: partner offsets (3 int32 per cell, INT32_MIN where
 * chi = 0) and the repulsive force density F_rep (3N). Either pointer may be NULL. */
int lbm_read_nci(lbm_ctx *ctx, int32_t *partner, double *frep);

/* Near-contact film statistics of the current phi (Sec. 3.3, Eq. 74): the near-contact pass is run
 * on the current phi, then, over the film Omega_film = {chi = 1} with n the normal of Eq. 57 and
 * F_cap = mu_phi grad(phi) (Eq. 19), FP64 sums in a fixed order give
 *   out[0] V_film (cells), out[1] sum |F_rep . n|, out[2] sum |F_cap . n|, out[3] max |F_rep|,
 *   out[4] sum |F_rep|, out[5] R_n = out[1] / out[2] (0 without film), out[6] out[4] / out[0].
 * out: 7 doubles (host), written on success; all zero when the near-contact model is off.
 * Allocates 24 KB of device scratch on the first call. Synchronises the context's stream. */
int lbm_nci_diagnostics(lbm_ctx *ctx, double *out);

/* Interfacial mean curvature of the current phi (Sec. 3.4, Eq. 78): kappa = div n with the outward
 * unit normal n = grad(phi) / (|grad(phi)| + eps_n) (Eq. 57; phi = 0 inside a bubble), the
 * divergence by the isotropic stencil of Eq. 22, at the cells of the band q >= q_th (Eq. 59).
 * hist: nbins int64 counts of kappa over equal bins of [kmin, kmax) (values outside are not
 * binned; nbins = 0 skips it and hist may be NULL); out[0] = band cells, out[1] = mean kappa.
 * 0 <= nbins <= 4096 and kmax > kmin, else LBM_ERR_ARG. The normals of every cell are written to
 * the near-contact normal buffer, which the next step recomputes where it reads it. Allocates
 * 42 KB of device scratch on the first call; synchronises the context's stream. */
int lbm_curvature(lbm_ctx *ctx, double kmin, double kmax, int nbins, int64_t *hist, double *out);

/* Carrier-phase kinetic-energy spectrum of the current state (Sec. 3.4): the liquid (phi >= 1/2)
 * velocity fluctuation u' = chi (u - <u>_liquid), with u the velocity of lbm_read_fields, transformed
 * per component (cuFFT, real to complex); E[K] = sum over the wave vectors k_a = 2 pi m_a / n_a
 * with floor(|k| / (2 pi / max(n_a)) + 1/2) = K of |u_hat(k)|^2 / 2, u_hat = FFT / N, so the sum of
 * all shells is <|u'|^2> / 2. E: nshells doubles (host), 1 <= nshells <= 1024 (else LBM_ERR_ARG);
 * energy beyond the last shell is not returned. Allocates about 8N bytes of device memory plus the
 * transform's workspace for the call; LBM_ERR_CUDA if that or the transform fails. Synchronises. */
int lbm_energy_spectrum(lbm_ctx *ctx, int nshells, double *E);

/* Batches: independent contexts advanced together (a parameter sweep of uneven cases; no
 * counterpart in the paper, which runs one case at a time). One CUDA graph holds two steps of
 * every context, the contexts spread over nstreams concurrent branches, so that small cases fill
 * the GPU together and each kernel launch is paid once per graph rather than once per call.
 * ctxs: n distinct contexts, initialised, on the current device, with mass_check_every = 0 and
 * the profiler off (else LBM_ERR_ARG; uninitialised: LBM_ERR_STATE). They stay owned by the caller
 * and must outlive the batch; while the batch exists only lbm_batch_step may advance them (reads
 * and lbm_mass on their own streams remain allowed once lbm_batch_step's work is complete).
 * stream: the cudaStream_t the graph is launched on (NULL: a stream of the batch's own).
 * *out receives the batch; on error nothing is allocated. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_ctx *const *ctxs, int n, int nstreams, void *stream, lbm_batch **out);
/* lbm_batch_create with flags. Without flags, when every context is 3D with one lattice (19 or 27)
 * and one store type, nx even and Q N <= 2^32, the batch runs FUSED: per step, the near-contact
 * pass of each context on the concurrent branches, then one launch of the hydrodynamic pass and
 * one launch of the phase-field pass over all contexts together (persistent grids walking a work
 * list of every case's tiles), with the same per-cell arithmetic as lbm_step, so the results are
 * identical. An autotuner then times, on the contexts' own state and without changing it, the
 * hydrodynamic tile shape (64 x ty x 8/ty cells, ty = 4, 2, 8) and the rows of y per thread of the
 * phase-field march (4 or 2), keeps the fastest, and finally times one step of that fused
 * execution against one step of the per-case graph, keeping the fused execution only when it is at
 * least 3 % faster (lbm_batch_config reports both times).
 * Otherwise, or with LBM_BATCH_PER_CASE, the graph holds every context's own steps on the branches.
 * LBM_BATCH_NO_TUNE keeps ty = 4 and 4 rows; LBM_BATCH_HYDRO_TY2 / _TY8 and LBM_BATCH_PHASE_ROWS2
 * pin those choices instead (no tuning). Creation allocates the work lists (8 B per tile) and a
 * case table; unknown or contradictory flags: LBM_ERR_ARG. */
#define LBM_BATCH_PER_CASE 1
#define LBM_BATCH_NO_TUNE 2
#define LBM_BATCH_HYDRO_TY2 4
#define LBM_BATCH_HYDRO_TY8 8
#define LBM_BATCH_PHASE_ROWS2 16
int lbm_batch_create_ex(lbm_ctx *const *ctxs, int n, int nstreams, void *stream, int flags, lbm_batch **out);
/* The batch's configuration: cfg (8 ints, may be NULL) = fused (1/0), hydrodynamic tile ty, tz,
 * phase-field rows per thread, branches, hydrodynamic blocks, phase-field blocks, hydrodynamic
 * work items; ms (7 doubles, may be NULL) = the tuner's time per pass of the hydrodynamic
 * candidates ty = 4, 2, 8 and of the phase-field candidates rows = 4, 2, then of one step of the
 * fused and of the per-case execution (0 when not tuned). */
int lbm_batch_config(const lbm_batch *b, int *cfg, double *ms);
/* Advances every context by nsteps: one graph launch per two steps, and for an odd nsteps a last
 * plain step of each context, all on the batch's launch stream. Asynchronous like lbm_step:
 * synchronise the launch stream (or call lbm_batch_synchronize) before reading results. Two graphs
 * are captured at creation, one per ping-pong parity of the buffers (an odd nsteps flips it); a
 * launch uses the one that every context holds. LBM_ERR_STATE if the contexts hold neither together
 * (one was re-initialised or stepped outside the batch): nothing is launched. */
int lbm_batch_step(lbm_batch *b, int nsteps);
/* Waits for the batch's launch stream. */
int lbm_batch_synchronize(lbm_batch *b);
/* Waits for the batch's work, then frees the graph and the batch's streams (not the contexts). */
void lbm_batch_destroy(lbm_batch *b);

/* Waits for all work of ctx. */
int lbm_synchronize(lbm_ctx *ctx);

/* Per-kernel timing with CUDA events on the context stream (enable = 1 starts a fresh tally of every
 * kind, enable = 0 stops). Synchronises the stream first. Each timed pass records two events on the
 * stream, which adds a little time between kernels (and ends the launch overlap between the step
 * kernels around it). Null ctx: LBM_ERR_ARG; a CUDA failure of the synchronisation: LBM_ERR_CUDA. */
int lbm_profile(lbm_ctx *ctx, int enable);
/* As lbm_profile, timing only the kinds whose bit (1u << kind, kind an lbm_kernel_kind) is set in
 * mask; mask = 0 stops. Bits of kinds beyond LBM_K_COUNT are ignored. Same errors as lbm_profile. */
int lbm_profile_kinds(lbm_ctx *ctx, unsigned mask);
/* Times only the first and then every `every`-th pass of each profiled kind (counted from the last
 * lbm_profile / lbm_profile_kinds call), so that a long run can be sampled with fewer events between
 * its kernels; 1 (the default) times every pass. The setting stays until changed. every < 1 or NULL
 * ctx: LBM_ERR_ARG. */
int lbm_profile_sample(lbm_ctx *ctx, int every);
/* Accumulated device milliseconds and kernel launch counts per lbm_kernel_kind (arrays of
 * LBM_K_COUNT; either may be NULL). A pass of several kernels counts each of them: the near-contact
 * pass over the listed tiles is 3 kernels where the brick prefilter applies (3D, every side a
 * multiple of 4) and 2 elsewhere; a reduction is 2; the split step's hydrodynamic pass is 2, timed
 * from its first launch to the join of both (the concurrent near-contact pass runs inside that time).
 * Synchronises the stream. */
int lbm_profile_read(lbm_ctx *ctx, double *ms, int64_t *launches);

/* Velocity table of a hydrodynamic lattice in the order above: c is 3*Q ints, w is Q doubles. */
int lbm_lattice(int dim, int Q, int *c, double *w);

const char *lbm_strerror(int status);
const char *lbm_kernel_name(int kind);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
