/*
 * lbm_oracle.h -- plain FP64 CPU oracle of one time step of the phase-field lattice Boltzmann model
 * with near-contact repulsion of arXiv 2603.17481.
 *
 * TEST INFRASTRUCTURE. This header and lbm_oracle.c are the correctness reference of the CUDA
 * library, not part of it: only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load them. They share no code, header, table or helper with the CUDA library.
 *
 * Array conventions (all arrays are caller-owned, FP64 unless stated):
 *   cell index  n = x + nx*(y + ny*z), x fastest; nz = 1 in 2D.
 *   populations f[i*N + n], i in [0,Q), pre-collision populations of step t located at cell n.
 *   vectors     v[a*N + n], a in [0,3) (the z component is present and zero in 2D).
 *   velocity order: by |c|^2 ascending, ties by (c_z, c_y, c_x) lexicographic with -1 < 0 < +1.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim, nx, ny, nz;
  int Q;                  /* hydrodynamic lattice: 9 (2D), 19 or 27 (3D)                      */
  double rho_l, rho_g;    /* liquid (phi = 1) and gas (phi = 0) densities                     */
  double nu_l, nu_g;      /* kinematic viscosities                                            */
  double sigma;           /* surface tension                                                  */
  double eps;             /* interface width epsilon (= delta = W)                            */
  double D;               /* interface diffusivity (tau_diff of Eq. 28)                       */
  int nci_on;             /* near-contact interaction on/off                                  */
  int w;                  /* search-window radius (Eq. 60)                                    */
  double A_rep, h0, p;    /* amplitude, thickness-weight scale and exponent (Eqs. 42, 71)     */
  double q_th, eta, cos_opp, eps_q, eps_n;  /* Eqs. 57-62, 67                                  */
  double g[3];            /* body acceleration for the buoyancy force                         */
  double rho_bar;         /* mean density of the initial field (buoyancy reference)           */
  int decide_f32;         /* 1: near-contact gate decisions taken in binary32                  */
} orc_params;

/* Lattice tables. Returns 0, or -1 for an unsupported (dim, Q). c is Q*3 ints, w is Q doubles. */
int orc_lattice(int dim, int Q, int *c, double *w);

/* Third-order Hermite equilibrium, Eq. 11 (Q outputs). */
void orc_feq(int dim, int Q, double pstar, const double *u, double *feq);
/* Guo source term, Eq. 17, with Fr = F/rho (Q outputs). */
void orc_guo(int dim, int Q, const double *u, const double *Fr, double *S);
/* Regularized non-equilibrium reconstruction, Eq. 14 with A3 from Eq. 16 (Q outputs). A2 is 3x3. */
void orc_regularized(int dim, int Q, const double *u, const double *A2, double *out);

/* One cell of the hydrodynamic update (Eqs. 3-21): pre-collision populations f (Q), phase field and
 * its isotropic gradient / Laplacian at the cell, near-contact force Frep (3). Outputs post-collision
 * populations (Q), the velocity u (3) and p*. */
void orc_hydro_cell(const orc_params *P, const double *f, double phi, const double *gphi,
                    double lphi, const double *Frep, double *fpost, double *u, double *pstar);

/* Isotropic gradient (Eq. 22) and Laplacian (Eq. 23) on the D2Q9 (2D) / D3Q27 (3D) stencil. */
void orc_grad_iso(const orc_params *P, const double *psi, double *grad);
void orc_lap_iso(const orc_params *P, const double *psi, double *lap);

double orc_minmod(double a, double b);          /* Eq. 32 */
double orc_h_of_q(double q, double eps);        /* Eq. 70 */
double orc_w_h(double h, double h0, double p);  /* Eq. 42 */

/* Near-contact interaction (Sec. 2.3): partner offsets (3 ints per cell, INT_MIN where chi = 0),
 * repulsive force density Frep (3N) and, if margin != NULL, the decision margin of every cell. */
void orc_nci(const orc_params *P, const double *phi, int *partner, double *frep, double *margin);

/* Phase-field update, Eq. 28 with Eqs. 29-35, given the velocity u (3N). */
void orc_phi_update(const orc_params *P, const double *phi, const double *u, double *phi_new);

/* Equilibrium initial populations f = feq(p*0, u0); pstar may be NULL (p*0 = 0). */
void orc_init(const orc_params *P, const double *phi, const double *u, const double *pstar, double *f);

/* Mean density of phi under the linear mixture rule (for rho_bar). */
double orc_mean_density(const orc_params *P, const double *phi);

/* p* and u of the current state (forces evaluated on the current phi), as used by a step. */
void orc_moments(const orc_params *P, const double *f, const double *phi, double *pstar, double *u);

/* Advance nsteps full time steps in place. u_last (3N, may be NULL) receives the velocity of the
 * last step (the one that advected phi). Returns 0, or -1 on allocation failure. */
int orc_step(const orc_params *P, double *f, double *phi, int nsteps, double *u_last);

/* Self-tuning diagnostics of the near-contact interaction (Sec. 3.3, Eq. 74) on phi, over the film
 * region Omega_film = {chi = 1} (cells with a partner, Sec. 2.3.2), with n the normal of Eq. 57,
 * F_rep of Eq. 73 and the capillary force F_cap = mu_phi grad(phi) of Eq. 19 (mu_phi of reading R3):
 *   out[0] = V_film (number of film cells; dV = 1),  out[1] = sum |F_rep . n|,
 *   out[2] = sum |F_cap . n|,  out[3] = max |F_rep|,  out[4] = sum |F_rep|.
 * R_n = out[1] / out[2] and <|F_rep|>_film = out[4] / out[0]. Returns 0, or -1 on allocation failure. */
int orc_nci_diagnostics(const orc_params *P, const double *phi, double *out);

/* Interfacial mean curvature (Sec. 3.4, Eq. 78): kappa = div n with the outward unit normal
 * n = grad(phi) / (|grad(phi)| + eps_n) of Eq. 57 (phi = 0 inside a bubble, 1 in the liquid), the
 * divergence taken with the isotropic stencil of Eq. 22, at the cells of the interfacial band
 * q >= q_th (Eq. 59). Histogram of kappa over nbins equal bins of [kmin, kmax) into hist (values
 * outside are not binned); out[0] = number of band cells, out[1] = sum of kappa over the band.
 * Returns 0, or -1 on allocation failure or nbins < 1. */
int orc_curvature(const orc_params *P, const double *phi, double kmin, double kmax, int nbins, long long *hist,
                  double *out);

#ifdef __cplusplus
}
#endif
#endif
