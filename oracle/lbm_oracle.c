/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the per-time-step lattice update of arXiv 2603.17481
 * ("Adaptive near-contact repulsion in conservative Allen-Cahn phase-field lattice Boltzmann
 * multiphase model"):
 *   - recursive-regularized lattice Boltzmann hydrodynamics with Guo forcing, Sec. 2.1, Eqs. 3-23;
 *   - conservative Allen-Cahn phase field, MUSCL-minmod advection + isotropic Laplacian and
 *     compressive divergence, Sec. 2.1.1, Eqs. 24-35;
 *   - near-contact interaction (gate, bounded-window pairing, closed-form proximity indicator,
 *     repulsive force), Sec. 2.3, Eqs. 57-73.
 *
 * TEST INFRASTRUCTURE. This file is the correctness reference of the CUDA library, not part of the
 * product: only the test-suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header, table or helper with the CUDA library. Every intermediate is a plain
 * full-size FP64 array and every step is the paper's formula in the paper's order; nothing is
 * fused, blocked or reordered. The OpenMP pragmas only split independent per-cell loops.
 *
 * Readings taken where the paper is silent, ambiguous or garbled:
 *   R1  step order: hydrodynamics on phi^n gives u^n, then phi^{n+1} = Phi(phi^n, u^n).
 *   R2  rho(phi) = rho_g + (rho_l - rho_g) phi (Sec. 2.1 announces a mixture rule but never prints it).
 *   R3  mu_phi = 4 beta phi (phi - 1)(phi - 1/2) - k lap(phi), beta = 12 sigma/eps, k = 3 sigma eps/2
 *       (Eq. 19 refers to a chemical potential that is never printed).
 *   R4  partner ties after the facing score go to the smallest canonical window index.
 *   R5  n_sym is oriented toward the partner, r_hat . n_sym >= 0 (Sec. 2.3.3 text).
 *   R6  F_nu (Eq. 21) uses f_eq evaluated with the velocity u0 that excludes F_nu itself.
 *   R7  the symmetrisation S() of Eqs. 13 and 16 sums the 3 distinct index permutations.
 *   R8  buoyancy F_ext = (rho - rho_bar) g with rho_bar the initial mean density (periodic box).
 *   R9  Eq. 3 is applied to the regularized form of f - f_eq + S/2 (Sec. 2.1 text):
 *       f_post = f_eq + (1 - omega) Reg(f - f_eq + S/2) + S/2.
 *   R10 the Laplacian of Eq. 28 is the isotropic Eq. 23 and tau_diff = D.
 *   R11 S_comp of Eq. 35 is -(C_sharp / c_s^2) sum_i w_i c_i . a(x + c_i) with a = phi(1-phi) n and
 *       C_sharp = kappa = 4 D / eps (Eq. 26); the D2Q9 (2D) / D3Q27 (3D) stencil weights.
 *   R12 the near-contact normals use the same isotropic gradient (Eq. 57), the gate clamps phi to
 *       [0,1] (Sec. 2.3.1); the stored phi is never clamped.
 *   R13 with decide_f32 set, the gate/similarity/facing comparisons and the facing-score tie-break
 *       are evaluated in binary32, the precision of the GPU kernels (the paper fixes none).
 *   R14 the initial normalised pressure is p* = 0 unless given: p = rho c_s^2 p* (Eq. 5) is then
 *       uniform, whereas p* = 1 with a density contrast puts a pressure jump of
 *       (1 - rho_g/rho_l) c_s^2 across every interface.
 */
#include "lbm_oracle.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define CS2 (1.0 / 3.0)

typedef struct {
  int Q;
  int c[27][3];
  double w[27];
} lattice_t;

/* Velocity sets with weights by |c|^2 class (D2Q9, D3Q19, D3Q27 of the textbook lattices);
 * ordering: |c|^2 ascending, then (c_z, c_y, c_x) lexicographic. */
static int build_lattice(int dim, int Q, lattice_t *L) {
  double wc[4] = {0, 0, 0, 0};
  int maxn;
  if (dim == 2 && Q == 9) {
    wc[0] = 4.0 / 9.0; wc[1] = 1.0 / 9.0; wc[2] = 1.0 / 36.0; maxn = 2;
  } else if (dim == 3 && Q == 19) {
    wc[0] = 1.0 / 3.0; wc[1] = 1.0 / 18.0; wc[2] = 1.0 / 36.0; maxn = 2;
  } else if (dim == 3 && Q == 27) {
    wc[0] = 8.0 / 27.0; wc[1] = 2.0 / 27.0; wc[2] = 1.0 / 54.0; wc[3] = 1.0 / 216.0; maxn = 3;
  } else {
    return -1;
  }
  int k = 0;
  int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
  for (int n2 = 0; n2 <= maxn; n2++)
    for (int cz = zlo; cz <= zhi; cz++)
      for (int cy = -1; cy <= 1; cy++)
        for (int cx = -1; cx <= 1; cx++)
          if (cx * cx + cy * cy + cz * cz == n2) {
            L->c[k][0] = cx; L->c[k][1] = cy; L->c[k][2] = cz;
            L->w[k] = wc[n2];
            k++;
          }
  L->Q = k;
  return k == Q ? 0 : -1;
}

/* Stencil lattice of the discrete derivatives: D2Q9 in 2D, D3Q27 in 3D (Sec. 2.1, Sec. 2.3.1). */
static void stencil_lattice(int dim, lattice_t *L) { build_lattice(dim, dim == 2 ? 9 : 27, L); }

int orc_lattice(int dim, int Q, int *c, double *w) {
  lattice_t L;
  if (build_lattice(dim, Q, &L)) return -1;
  for (int i = 0; i < Q; i++) {
    for (int a = 0; a < 3; a++) c[3 * i + a] = L.c[i][a];
    w[i] = L.w[i];
  }
  return 0;
}

static inline int wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}
static inline long cell(const orc_params *P, int x, int y, int z) {
  return (long)x + (long)P->nx * ((long)y + (long)P->ny * z);
}
static inline long ncells(const orc_params *P) { return (long)P->nx * P->ny * P->nz; }
static inline double delta(int a, int b) { return a == b ? 1.0 : 0.0; }

/* Hermite tensors, Eqs. 12-13 (R7: three distinct permutations). */
static inline double H2(const int *c, int a, int b) { return c[a] * c[b] - CS2 * delta(a, b); }
static inline double H3(const int *c, int a, int b, int d) {
  return c[a] * c[b] * c[d] - CS2 * (c[a] * delta(b, d) + c[b] * delta(a, d) + c[d] * delta(a, b));
}

/* Eq. 11. */
static void feq_cell(const lattice_t *L, int dim, double pstar, const double *u, double *out) {
  const double cs4 = CS2 * CS2, cs6 = cs4 * CS2;
  for (int i = 0; i < L->Q; i++) {
    const int *c = L->c[i];
    double cu = 0, h2 = 0, h3 = 0;
    for (int a = 0; a < dim; a++) cu += c[a] * u[a];
    for (int a = 0; a < dim; a++)
      for (int b = 0; b < dim; b++) h2 += H2(c, a, b) * u[a] * u[b];
    for (int a = 0; a < dim; a++)
      for (int b = 0; b < dim; b++)
        for (int d = 0; d < dim; d++) h3 += H3(c, a, b, d) * u[a] * u[b] * u[d];
    out[i] = L->w[i] * (pstar + cu / CS2 + h2 / (2 * cs4) + h3 / (6 * cs6));
  }
}

/* Eq. 17 with Fr = F / rho. */
static void guo_cell(const lattice_t *L, int dim, const double *u, const double *Fr, double *S) {
  const double cs4 = CS2 * CS2;
  for (int i = 0; i < L->Q; i++) {
    const int *c = L->c[i];
    double cu = 0, s = 0;
    for (int a = 0; a < dim; a++) cu += c[a] * u[a];
    for (int a = 0; a < dim; a++) s += ((c[a] - u[a]) / CS2 + cu * c[a] / cs4) * Fr[a];
    S[i] = L->w[i] * s;
  }
}

/* Eq. 14 with the recursive third-order tensor of Eq. 16. A2 is a 3x3 row-major tensor. */
static void reg_cell(const lattice_t *L, int dim, const double *u, const double *A2, double *out) {
  const double cs4 = CS2 * CS2, cs6 = cs4 * CS2;
  double A3[3][3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      for (int d = 0; d < 3; d++)
        A3[a][b][d] = u[a] * A2[3 * b + d] + u[b] * A2[3 * a + d] + u[d] * A2[3 * a + b];
  for (int i = 0; i < L->Q; i++) {
    const int *c = L->c[i];
    double t2 = 0, t3 = 0;
    for (int a = 0; a < dim; a++)
      for (int b = 0; b < dim; b++) t2 += H2(c, a, b) * A2[3 * a + b];
    for (int a = 0; a < dim; a++)
      for (int b = 0; b < dim; b++)
        for (int d = 0; d < dim; d++) t3 += H3(c, a, b, d) * A3[a][b][d];
    out[i] = L->w[i] * (t2 / (2 * cs4) + t3 / (6 * cs6));
  }
}

void orc_feq(int dim, int Q, double pstar, const double *u, double *feq) {
  lattice_t L;
  if (build_lattice(dim, Q, &L)) return;
  feq_cell(&L, dim, pstar, u, feq);
}
void orc_guo(int dim, int Q, const double *u, const double *Fr, double *S) {
  lattice_t L;
  if (build_lattice(dim, Q, &L)) return;
  guo_cell(&L, dim, u, Fr, S);
}
void orc_regularized(int dim, int Q, const double *u, const double *A2, double *out) {
  lattice_t L;
  if (build_lattice(dim, Q, &L)) return;
  reg_cell(&L, dim, u, A2, out);
}

/* One hydrodynamic cell update: Eqs. 6-10 (moments and mixture properties), 17-21 (forces),
 * 11, 14, 16 (equilibrium and regularization) and Eq. 3 in the regularized form of R9. */
static void hydro_cell(const orc_params *P, const lattice_t *L, const double *f, double phi,
                       const double *gphi, double lphi, const double *Frep, double *fpost,
                       double *u, double *pstar_out) {
  const int dim = P->dim, Q = L->Q;
  double fe[27], S[27], R[27];

  /* mixture properties: R2, Eqs. 8-10 */
  double rho = P->rho_g + (P->rho_l - P->rho_g) * phi;
  double grho[3] = {0, 0, 0};
  for (int a = 0; a < dim; a++) grho[a] = (P->rho_l - P->rho_g) * gphi[a];
  double mu = P->rho_g * P->nu_g + (P->rho_l * P->nu_l - P->rho_g * P->nu_g) * phi;
  double nu = mu / rho;
  double omega = 1.0 / (0.5 + nu / CS2);

  /* capillary force, Eq. 19 with the chemical potential of R3 */
  double beta = 12.0 * P->sigma / P->eps, kap = 1.5 * P->sigma * P->eps;
  double muphi = 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - kap * lphi;
  double Fs[3] = {0, 0, 0};
  for (int a = 0; a < dim; a++) Fs[a] = muphi * gphi[a];

  /* p*, Eq. 6 */
  double pstar = 0;
  for (int i = 0; i < Q; i++) pstar += f[i];

  /* pressure correction, Eq. 20; buoyancy, R8 */
  double Fp[3] = {0, 0, 0}, Fext[3] = {0, 0, 0};
  for (int a = 0; a < dim; a++) {
    Fp[a] = -pstar * CS2 * grho[a];
    Fext[a] = (rho - P->rho_bar) * P->g[a];
  }

  /* velocity without F_nu (R6), Eq. 7 with the first moment of S equal to F / rho */
  double u0[3] = {0, 0, 0};
  for (int a = 0; a < dim; a++) {
    double j = 0;
    for (int i = 0; i < Q; i++) j += f[i] * L->c[i][a];
    u0[a] = j + (Fs[a] + Fp[a] + Frep[a] + Fext[a]) / (2.0 * rho);
  }

  /* viscous correction, Eq. 21 */
  feq_cell(L, dim, pstar, u0, fe);
  double Pi[3][3] = {{0}};
  for (int a = 0; a < dim; a++)
    for (int b = 0; b < dim; b++) {
      double s = 0;
      for (int i = 0; i < Q; i++) s += (f[i] - fe[i]) * L->c[i][a] * L->c[i][b];
      Pi[a][b] = s;
    }
  double Fnu[3] = {0, 0, 0};
  for (int a = 0; a < dim; a++) {
    double s = 0;
    for (int b = 0; b < dim; b++) s += Pi[a][b] * grho[b];
    Fnu[a] = -(nu * omega / CS2) * s;
  }

  /* total force, Eq. 18; final velocity, Eq. 7 */
  double F[3] = {0, 0, 0}, Fr[3] = {0, 0, 0};
  for (int a = 0; a < 3; a++) u[a] = 0;
  for (int a = 0; a < dim; a++) {
    F[a] = Fs[a] + Fp[a] + Fnu[a] + Frep[a] + Fext[a];
    u[a] = u0[a] + Fnu[a] / (2.0 * rho);
    Fr[a] = F[a] / rho;
  }

  /* equilibrium, source, regularized non-equilibrium: Eqs. 11, 17, 14, 16 */
  feq_cell(L, dim, pstar, u, fe);
  guo_cell(L, dim, u, Fr, S);
  double A2[9] = {0};
  for (int a = 0; a < dim; a++)
    for (int b = 0; b < dim; b++) {
      double s = 0;
      for (int i = 0; i < Q; i++) s += H2(L->c[i], a, b) * (f[i] - fe[i] + 0.5 * S[i]);
      A2[3 * a + b] = s;
    }
  reg_cell(L, dim, u, A2, R);

  /* collision, Eq. 3 in the form of R9 */
  for (int i = 0; i < Q; i++) fpost[i] = fe[i] + (1.0 - omega) * R[i] + 0.5 * S[i];
  if (pstar_out) *pstar_out = pstar;
}

void orc_hydro_cell(const orc_params *P, const double *f, double phi, const double *gphi,
                    double lphi, const double *Frep, double *fpost, double *u, double *pstar) {
  lattice_t L;
  if (build_lattice(P->dim, P->Q, &L)) return;
  hydro_cell(P, &L, f, phi, gphi, lphi, Frep, fpost, u, pstar);
}

/* Eq. 22 */
void orc_grad_iso(const orc_params *P, const double *psi, double *grad) {
  lattice_t S;
  stencil_lattice(P->dim, &S);
  const long N = ncells(P);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    int x = (int)(n % P->nx), y = (int)((n / P->nx) % P->ny), z = (int)(n / ((long)P->nx * P->ny));
    double g[3] = {0, 0, 0};
    for (int i = 0; i < S.Q; i++) {
      double v = psi[cell(P, wrap(x + S.c[i][0], P->nx), wrap(y + S.c[i][1], P->ny),
                          wrap(z + S.c[i][2], P->nz))];
      for (int a = 0; a < 3; a++) g[a] += S.w[i] * v * S.c[i][a];
    }
    for (int a = 0; a < 3; a++) grad[a * N + n] = g[a] / CS2;
  }
}

/* Eq. 23 */
void orc_lap_iso(const orc_params *P, const double *psi, double *lap) {
  lattice_t S;
  stencil_lattice(P->dim, &S);
  const long N = ncells(P);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    int x = (int)(n % P->nx), y = (int)((n / P->nx) % P->ny), z = (int)(n / ((long)P->nx * P->ny));
    double s = 0;
    for (int i = 1; i < S.Q; i++)
      s += S.w[i] * psi[cell(P, wrap(x + S.c[i][0], P->nx), wrap(y + S.c[i][1], P->ny),
                             wrap(z + S.c[i][2], P->nz))];
    lap[n] = (2.0 / CS2) * (s - (1.0 - S.w[0]) * psi[n]);
  }
}

/* Eq. 32 */
double orc_minmod(double a, double b) {
  if (a * b <= 0) return 0.0;
  double m = fabs(a) < fabs(b) ? fabs(a) : fabs(b);
  return a > 0 ? m : -m;
}

/* Eq. 70 (literal arcosh form) */
double orc_h_of_q(double q, double eps) { return eps * acosh(1.0 / (2.0 * sqrt(q))); }

/* Eq. 42 */
double orc_w_h(double h, double h0, double p) { return 1.0 / (1.0 + pow(h / h0, p)); }

/* interfacial indicator of Eq. 58 on phi clamped to [0, 1] (Sec. 2.3.1) */
static inline double q_of_phi(double phi) {
  double pc = phi < 0 ? 0 : (phi > 1 ? 1 : phi);
  return pc * (1.0 - pc);
}
static inline float q_of_phi_f32(double phi) {
  float pc = (float)phi;
  pc = pc < 0.0f ? 0.0f : (pc > 1.0f ? 1.0f : pc);
  return pc * (1.0f - pc);
}

/* Near-contact detection and pairing (Sec. 2.3.2, Eqs. 59-65) and force construction
 * (Sec. 2.3.3, Eqs. 66-73). */
void orc_nci(const orc_params *P, const double *phi, int *partner, double *frep, double *margin) {
  const long N = ncells(P);
  const int dim = P->dim, w = P->w, W = 2 * w + 1;
  double *grad = (double *)malloc(sizeof(double) * 3 * N);
  double *nrm = (double *)malloc(sizeof(double) * 3 * N);
  double *q = (double *)malloc(sizeof(double) * N);
  if (!grad || !nrm || !q) {
    free(grad); free(nrm); free(q);
    return;
  }
  /* normals, Eq. 57, and interfacial indicator, Eq. 58 */
  orc_grad_iso(P, phi, grad);
  for (long n = 0; n < N; n++) {
    double g2 = 0;
    for (int a = 0; a < 3; a++) g2 += grad[a * N + n] * grad[a * N + n];
    double gn = sqrt(g2);
    for (int a = 0; a < 3; a++) nrm[a * N + n] = grad[a * N + n] / (gn + P->eps_n);
    q[n] = q_of_phi(phi[n]);
  }
  const float qth_f = (float)P->q_th, eta_f = (float)P->eta, cos_f = (float)P->cos_opp,
              epsq_f = (float)P->eps_q;

#pragma omp parallel for schedule(dynamic, 64)
  for (long n = 0; n < N; n++) {
    int x = (int)(n % P->nx), y = (int)((n / P->nx) % P->ny), z = (int)(n / ((long)P->nx * P->ny));
    for (int a = 0; a < 3; a++) {
      partner[3 * n + a] = INT_MIN;
      frep[a * N + n] = 0.0;
    }
    double qx = q[n];
    double marg = fabs(qx - P->q_th);
    /* interfacial gate, Eq. 59 */
    int gated = P->decide_f32 ? (q_of_phi_f32(phi[n]) >= qth_f) : (qx >= P->q_th);
    if (!gated) {
      if (margin) margin[n] = marg;
      continue;
    }
    double nxv[3] = {nrm[n], nrm[N + n], nrm[2 * N + n]};

    /* bounded window, Eq. 60; candidate criteria, Eqs. 61-62; selection, Eq. 65 with R4 */
    int have = 0, best_d2 = 0, best_k = 0, best_r[3] = {0, 0, 0};
    double best_ff = 0;
    long best_m = -1;
    int zr = dim == 3 ? w : 0;
    /* first pass: choose the partner */
    for (int rz = -zr; rz <= zr; rz++)
      for (int ry = -w; ry <= w; ry++)
        for (int rx = -w; rx <= w; rx++) {
          if (rx == 0 && ry == 0 && rz == 0) continue;
          long m = cell(P, wrap(x + rx, P->nx), wrap(y + ry, P->ny), wrap(z + rz, P->nz));
          double qy = q[m];
          double dot = nxv[0] * nrm[m] + nxv[1] * nrm[N + m] + nxv[2] * nrm[2 * N + m];
          int ok;
          double ff;
          if (P->decide_f32) {
            float qxf = q_of_phi_f32(phi[n]), qyf = q_of_phi_f32(phi[m]);
            float dotf = (float)nxv[0] * (float)nrm[m] + (float)nxv[1] * (float)nrm[N + m] +
                         (float)nxv[2] * (float)nrm[2 * N + m];
            float mq = qxf > epsq_f ? qxf : epsq_f;
            ok = (qyf >= qth_f) && (fabsf(qyf - qxf) <= eta_f * mq) && (dotf <= cos_f);
            ff = -dotf > 0.0f ? -dotf : 0.0f;
          } else {
            double mq = qx > P->eps_q ? qx : P->eps_q;
            ok = (qy >= P->q_th) && (fabs(qy - qx) <= P->eta * mq) && (dot <= P->cos_opp);
            ff = -dot > 0 ? -dot : 0.0;
          }
          if (!ok) continue;
          int d2 = rx * rx + ry * ry + rz * rz;
          int k = ((rz + zr) * W + (ry + w)) * W + (rx + w);
          int better = !have || d2 < best_d2 || (d2 == best_d2 && ff > best_ff) ||
                       (d2 == best_d2 && ff == best_ff && k < best_k);
          if (better) {
            have = 1; best_d2 = d2; best_ff = ff; best_k = k; best_m = m;
            best_r[0] = rx; best_r[1] = ry; best_r[2] = rz;
          }
        }

    /* decision margins (test diagnostics only): how far each decision that could change the
     * chosen partner lies from its threshold */
    for (int rz = -zr; rz <= zr; rz++)
      for (int ry = -w; ry <= w; ry++)
        for (int rx = -w; rx <= w; rx++) {
          if (rx == 0 && ry == 0 && rz == 0) continue;
          int d2 = rx * rx + ry * ry + rz * rz;
          if (have && d2 > best_d2) continue;
          long m = cell(P, wrap(x + rx, P->nx), wrap(y + ry, P->ny), wrap(z + rz, P->nz));
          double qy = q[m];
          double dot = nxv[0] * nrm[m] + nxv[1] * nrm[N + m] + nxv[2] * nrm[2 * N + m];
          double mq = qx > P->eps_q ? qx : P->eps_q;
          double m1 = qy - P->q_th, m2 = P->eta * mq - fabs(qy - qx), m3 = P->cos_opp - dot;
          int p1 = m1 >= 0, p2 = m2 >= 0, p3 = m3 >= 0;
          double cm;
          if (p1 && p2 && p3) {
            cm = fmin(m1, fmin(m2, m3));
          } else {
            cm = 0;
            if (!p1) cm = fmax(cm, -m1);
            if (!p2) cm = fmax(cm, -m2);
            if (!p3) cm = fmax(cm, -m3);
          }
          if (have && d2 == best_d2 && m != best_m && p1 && p2 && p3) {
            double ffo = -dot > 0 ? -dot : 0.0;
            double ffb = 0;
            double dotb = nxv[0] * nrm[best_m] + nxv[1] * nrm[N + best_m] + nxv[2] * nrm[2 * N + best_m];
            ffb = -dotb > 0 ? -dotb : 0.0;
            cm = fmin(cm, fabs(ffb - ffo));
          }
          marg = fmin(marg, cm);
        }

    if (have) {
      long m = best_m;
      partner[3 * n] = best_r[0]; partner[3 * n + 1] = best_r[1]; partner[3 * n + 2] = best_r[2];
      double nyv[3] = {nrm[m], nrm[N + m], nrm[2 * N + m]};
      /* Eqs. 66-67 */
      double qpair = 0.5 * (qx + q[m]);
      double qcl = fmin(fmax(qpair, P->eps_q), 0.25 - P->eps_q);
      /* Eq. 68 */
      double dot = nxv[0] * nyv[0] + nxv[1] * nyv[1] + nxv[2] * nyv[2];
      double ff = -dot > 0 ? -dot : 0.0;
      /* Eq. 69 with the line-of-centres fallback and the orientation of R5 */
      double rn = sqrt((double)best_d2);
      double rhat[3] = {best_r[0] / rn, best_r[1] / rn, best_r[2] / rn};
      double nt[3] = {nxv[0] - nyv[0], nxv[1] - nyv[1], nxv[2] - nyv[2]};
      double ntn = sqrt(nt[0] * nt[0] + nt[1] * nt[1] + nt[2] * nt[2]);
      double ns[3];
      if (ntn < 1e-8) {
        for (int a = 0; a < 3; a++) ns[a] = rhat[a];
      } else {
        for (int a = 0; a < 3; a++) ns[a] = nt[a] / (ntn + P->eps_n);
      }
      double rdot = rhat[0] * ns[0] + rhat[1] * ns[1] + rhat[2] * ns[2];
      if (rdot < 0)
        for (int a = 0; a < 3; a++) ns[a] = -ns[a];
      marg = fmin(marg, fabs(rdot));
      /* Eqs. 70-73 */
      double h = orc_h_of_q(qcl, P->eps);
      double wh = orc_w_h(h, P->h0, P->p);
      double rho = P->rho_g + (P->rho_l - P->rho_g) * phi[n];
      for (int a = 0; a < dim; a++) frep[a * N + n] = rho * P->A_rep * qcl * wh * ff * ns[a];
    }
    if (margin) margin[n] = marg;
  }
  free(grad); free(nrm); free(q);
}

/* Eq. 28: MUSCL-minmod advection (Eqs. 29-34), isotropic Laplacian (R10) and compressive
 * divergence (Eq. 35, R11). */
void orc_phi_update(const orc_params *P, const double *phi, const double *u, double *phi_new) {
  lattice_t S;
  stencil_lattice(P->dim, &S);
  const long N = ncells(P);
  const int dim = P->dim;
  const double kappa = 4.0 * P->D / P->eps; /* Eq. 26 */
  double *grad = (double *)malloc(sizeof(double) * 3 * N);
  double *lap = (double *)malloc(sizeof(double) * N);
  double *av = (double *)malloc(sizeof(double) * 3 * N);
  if (!grad || !lap || !av) {
    free(grad); free(lap); free(av);
    return;
  }
  orc_grad_iso(P, phi, grad);
  orc_lap_iso(P, phi, lap);
  /* compressive vector a = phi (1 - phi) n, n from Eq. 25 on the isotropic gradient */
  for (long n = 0; n < N; n++) {
    double g2 = 0;
    for (int a = 0; a < 3; a++) g2 += grad[a * N + n] * grad[a * N + n];
    double gn = sqrt(g2);
    for (int a = 0; a < 3; a++) av[a * N + n] = phi[n] * (1.0 - phi[n]) * grad[a * N + n] / (gn + P->eps_n);
  }
  const int nsz[3] = {P->nx, P->ny, P->nz};
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    int xyz[3] = {(int)(n % P->nx), (int)((n / P->nx) % P->ny), (int)(n / ((long)P->nx * P->ny))};
    /* Eq. 29: flux difference per axis */
    double div = 0;
    for (int a = 0; a < dim; a++) {
      /* phi and u along axis a at offsets -2..+2 */
      double ph[5], ua[5];
      for (int k = -2; k <= 2; k++) {
        int p[3] = {xyz[0], xyz[1], xyz[2]};
        p[a] = wrap(p[a] + k, nsz[a]);
        long m = cell(P, p[0], p[1], p[2]);
        ph[k + 2] = phi[m];
        ua[k + 2] = u[a * N + m];
      }
      /* face i+1/2 uses cells i, i+1 (indices 2, 3); face i-1/2 uses cells i-1, i (1, 2) */
      double flux[2];
      for (int side = 0; side < 2; side++) {
        int l = 1 + side; /* left cell of the face */
        double uf = 0.5 * (ua[l] + ua[l + 1]);                                /* face velocity */
        double sl = orc_minmod(ph[l] - ph[l - 1], ph[l + 1] - ph[l]);         /* Eq. 31 */
        double sr = orc_minmod(ph[l + 1] - ph[l], ph[l + 2] - ph[l + 1]);
        double pL = ph[l] + 0.5 * sl, pR = ph[l + 1] - 0.5 * sr;               /* Eq. 33 */
        double pup = uf >= 0 ? pL : pR;                                        /* Eq. 34 */
        flux[side] = uf * pup;                                                 /* Eq. 30 */
      }
      div += flux[1] - flux[0];
    }
    /* Eq. 35 with R11 */
    double sdiv = 0;
    for (int i = 0; i < S.Q; i++) {
      long m = cell(P, wrap(xyz[0] + S.c[i][0], P->nx), wrap(xyz[1] + S.c[i][1], P->ny),
                    wrap(xyz[2] + S.c[i][2], P->nz));
      for (int a = 0; a < 3; a++) sdiv += S.w[i] * S.c[i][a] * av[a * N + m];
    }
    double scomp = -(kappa / CS2) * sdiv;
    phi_new[n] = phi[n] - div + P->D * lap[n] + scomp;
  }
  free(grad); free(lap); free(av);
}

void orc_init(const orc_params *P, const double *phi, const double *u, const double *pstar, double *f) {
  lattice_t L;
  if (build_lattice(P->dim, P->Q, &L)) return;
  const long N = ncells(P);
  (void)phi;
  for (long n = 0; n < N; n++) {
    double uu[3] = {u[n], u[N + n], u[2 * N + n]}, fe[27];
    feq_cell(&L, P->dim, pstar ? pstar[n] : 0.0, uu, fe);
    for (int i = 0; i < L.Q; i++) f[i * N + n] = fe[i];
  }
}

double orc_mean_density(const orc_params *P, const double *phi) {
  const long N = ncells(P);
  double s = 0;
  for (long n = 0; n < N; n++) s += P->rho_g + (P->rho_l - P->rho_g) * phi[n];
  return s / (double)N;
}

/* shared body of orc_moments and orc_step: phi-derived fields, near-contact force, and the
 * per-cell hydrodynamic update of every cell. fpost may be NULL (moments only). */
static int hydro_pass(const orc_params *P, const lattice_t *L, const double *f, const double *phi,
                      double *fpost, double *u, double *pstar) {
  const long N = ncells(P);
  const int Q = L->Q;
  double *grad = (double *)malloc(sizeof(double) * 3 * N);
  double *lap = (double *)malloc(sizeof(double) * N);
  double *frep = (double *)calloc(3 * N, sizeof(double));
  int *part = (int *)malloc(sizeof(int) * 3 * N);
  if (!grad || !lap || !frep || !part) {
    free(grad); free(lap); free(frep); free(part);
    return -1;
  }
  orc_grad_iso(P, phi, grad);
  orc_lap_iso(P, phi, lap);
  if (P->nci_on) orc_nci(P, phi, part, frep, NULL);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double fi[27], fo[27], uu[3], ps;
    for (int i = 0; i < Q; i++) fi[i] = f[i * N + n];
    double g[3] = {grad[n], grad[N + n], grad[2 * N + n]};
    double fr[3] = {frep[n], frep[N + n], frep[2 * N + n]};
    hydro_cell(P, L, fi, phi[n], g, lap[n], fr, fo, uu, &ps);
    if (fpost)
      for (int i = 0; i < Q; i++) fpost[i * N + n] = fo[i];
    for (int a = 0; a < 3; a++) u[a * N + n] = uu[a];
    if (pstar) pstar[n] = ps;
  }
  free(grad); free(lap); free(frep); free(part);
  return 0;
}

void orc_moments(const orc_params *P, const double *f, const double *phi, double *pstar, double *u) {
  lattice_t L;
  if (build_lattice(P->dim, P->Q, &L)) return;
  hydro_pass(P, &L, f, phi, NULL, u, pstar);
}

int orc_step(const orc_params *P, double *f, double *phi, int nsteps, double *u_last) {
  lattice_t L;
  if (build_lattice(P->dim, P->Q, &L)) return -1;
  const long N = ncells(P);
  const int Q = L.Q;
  double *fpost = (double *)malloc(sizeof(double) * Q * N);
  double *u = (double *)calloc(3 * N, sizeof(double));
  double *phin = (double *)malloc(sizeof(double) * N);
  if (!fpost || !u || !phin) {
    free(fpost); free(u); free(phin);
    return -1;
  }
  for (int s = 0; s < nsteps; s++) {
    /* hydrodynamics on phi^n (R1) */
    if (hydro_pass(P, &L, f, phi, fpost, u, NULL)) {
      free(fpost); free(u); free(phin);
      return -1;
    }
    /* streaming: f_i(x + c_i, t + 1) = f_post_i(x, t), Eq. 3 */
    for (int i = 0; i < Q; i++)
#pragma omp parallel for schedule(static)
      for (long n = 0; n < N; n++) {
        int x = (int)(n % P->nx), y = (int)((n / P->nx) % P->ny), z = (int)(n / ((long)P->nx * P->ny));
        long m = cell(P, wrap(x + L.c[i][0], P->nx), wrap(y + L.c[i][1], P->ny), wrap(z + L.c[i][2], P->nz));
        f[i * N + m] = fpost[i * N + n];
      }
    /* phase field with the velocity of this step (R1) */
    orc_phi_update(P, phi, u, phin);
    memcpy(phi, phin, sizeof(double) * N);
  }
  if (u_last) memcpy(u_last, u, sizeof(double) * 3 * N);
  free(fpost); free(u); free(phin);
  return 0;
}

/* Eq. 74 and the film statistics of Sec. 3.3: one pass over the cells that have a partner. */
int orc_nci_diagnostics(const orc_params *P, const double *phi, double *out) {
  const long N = ncells(P);
  int *partner = (int *)malloc(sizeof(int) * 3 * N);
  double *frep = (double *)malloc(sizeof(double) * 3 * N);
  double *grad = (double *)malloc(sizeof(double) * 3 * N);
  double *lap = (double *)malloc(sizeof(double) * N);
  if (!partner || !frep || !grad || !lap) {
    free(partner); free(frep); free(grad); free(lap);
    return -1;
  }
  orc_nci(P, phi, partner, frep, NULL);
  orc_grad_iso(P, phi, grad);
  orc_lap_iso(P, phi, lap);
  const double beta = 12.0 * P->sigma / P->eps, kap = 1.5 * P->sigma * P->eps;
  double vfilm = 0, srn = 0, scn = 0, fmax = 0, sabs = 0;
  for (long n = 0; n < N; n++) {
    if (partner[3 * n] == INT_MIN) continue;
    double g2 = 0;
    for (int a = 0; a < 3; a++) g2 += grad[a * N + n] * grad[a * N + n];
    const double gn = sqrt(g2);
    const double muphi = 4.0 * beta * phi[n] * (phi[n] - 1.0) * (phi[n] - 0.5) - kap * lap[n];
    double rn = 0, cn = 0, fr2 = 0;
    for (int a = 0; a < 3; a++) {
      const double na = grad[a * N + n] / (gn + P->eps_n);
      rn += frep[a * N + n] * na;
      cn += muphi * grad[a * N + n] * na;
      fr2 += frep[a * N + n] * frep[a * N + n];
    }
    vfilm += 1.0;
    srn += fabs(rn);
    scn += fabs(cn);
    sabs += sqrt(fr2);
    if (sqrt(fr2) > fmax) fmax = sqrt(fr2);
  }
  out[0] = vfilm; out[1] = srn; out[2] = scn; out[3] = fmax; out[4] = sabs;
  free(partner); free(frep); free(grad); free(lap);
  return 0;
}

/* Eq. 78: kappa = div n over the interfacial band, n from Eq. 57, divergence by Eq. 22. */
int orc_curvature(const orc_params *P, const double *phi, double kmin, double kmax, int nbins, long long *hist,
                  double *out) {
  if (nbins < 1) return -1;
  const long N = ncells(P);
  double *grad = (double *)malloc(sizeof(double) * 3 * N);
  double *nrm = (double *)malloc(sizeof(double) * 3 * N);
  double *div = (double *)malloc(sizeof(double) * 3 * N);
  if (!grad || !nrm || !div) {
    free(grad); free(nrm); free(div);
    return -1;
  }
  orc_grad_iso(P, phi, grad);
  for (long n = 0; n < N; n++) {
    double g2 = 0;
    for (int a = 0; a < 3; a++) g2 += grad[a * N + n] * grad[a * N + n];
    for (int a = 0; a < 3; a++) nrm[a * N + n] = grad[a * N + n] / (sqrt(g2) + P->eps_n);
  }
  /* div n = sum_a d_a n_a: the isotropic gradient of each component, then its own axis */
  double *ga = (double *)malloc(sizeof(double) * 3 * N);
  if (!ga) {
    free(grad); free(nrm); free(div);
    return -1;
  }
  for (int a = 0; a < 3; a++) {
    orc_grad_iso(P, nrm + a * N, ga);
    for (long n = 0; n < N; n++) div[a * N + n] = ga[a * N + n];
  }
  for (int k = 0; k < nbins; k++) hist[k] = 0;
  double cnt = 0, sum = 0;
  for (long n = 0; n < N; n++) {
    /* the band gate, in binary32 under reading R13 like the near-contact gate */
    const int band = P->decide_f32 ? (q_of_phi_f32(phi[n]) >= (float)P->q_th) : (q_of_phi(phi[n]) >= P->q_th);
    if (!band) continue;
    const double kap = div[n] + div[N + n] + div[2 * N + n];
    cnt += 1.0;
    sum += kap;
    if (kap >= kmin && kap < kmax) {
      int b = (int)((kap - kmin) / (kmax - kmin) * nbins);
      if (b >= nbins) b = nbins - 1;
      hist[b]++;
    }
  }
  out[0] = cnt;
  out[1] = sum;
  free(grad); free(nrm); free(div); free(ga);
  return 0;
}
