/*
 * lbpf_oracle.h -- plain FP64 CPU oracle for the lattice-Boltzmann phase-field
 * scheme of Cartalade, Younsi & Plapp (arXiv 1602.07483).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * restatement of the paper's algorithm that the CUDA path is checked against.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no source, header, table or helper with
 * the CUDA library (the lattice tables below are typed separately from the
 * paper's Tables 1 and 2).
 *
 * Layout: every field is a flat array indexed  ((z*ny + y)*nx + x), x fastest.
 * Populations are stored POST-STREAMING, i.e. g_i(x, t) as it enters the
 * collision of Eq. (collision stage, Sec. 3.4), population-major: [Q][site].
 */
#ifndef LBPF_ORACLE_H
#define LBPF_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double W0, tau0;      /* interface width and relaxation time, Eq. (PhaseField_KarmaRappel) */
  double D, kappa;      /* solute and thermal diffusivities, Eqs. (Concentration), (Temp) */
  double lambda;        /* coupling constant, Eq. (PhaseField_KarmaRappel) */
  double Mc_inf;        /* scaled liquidus slope times c_inf, Eq. (PhaseField_KarmaRappel) */
  double k;             /* partition coefficient, Eq. (Concentration) */
  int32_t aniso;        /* 0: Eq. (Anisotropic-Function_As); 1: Eq. (As_K41-K61) */
  double eps1, eps2;    /* aniso 0: eps1 = eps_s.  aniso 1: eps1 = eps_s, eps2 = delta */
  double dx, dt;        /* space and time steps, Sec. 3.1 */
  int32_t antitrapping; /* 1: j_at of Eq. (AntiTrapping_Current) on; 0: off */
  double grad2_min;     /* |grad phi|^2 below which the normal is undefined */
} ora_params;

typedef struct ora_sim ora_sim;

/* Lattice tables (Tables 1-4 of Sec. 3.4).  q in {7, 15, 19} (3D) or {5, 9} (2D,
 * stored with e_z = 0: an nz = 1 grid then runs the 2D scheme).
 * e: q*3 ints, w/A/B: q doubles, opp: q ints.  Returns 0, or -1 for a bad q. */
int ora_lattice(int q, int32_t* e, double* w, double* A, double* B, double* e2, int32_t* opp);

/* Anisotropy function a_s and its derivatives d a_s / d(d_alpha phi)
 * at the gradient grad[3] (physical units).  Returns a_s; das may be NULL. */
double ora_aniso(int aniso, double eps1, double eps2, const double grad[3], double das[3]);

/* Equilibria, for moment checks.  N[3] physical units; J[3] physical units. */
void ora_geq(int q, double phi, const double N[3], double dt_dx_W2_tau0, double* g0);
void ora_heq(int q, double U, double q_over_zeta, const double J[3], double dt_dx, double* h0);

ora_sim* ora_create(int nx, int ny, int nz, int q_phi, int q_u, int q_theta, const ora_params* p);
void ora_destroy(ora_sim* s);

/* Seeds: n spheres, centres (3n, lattice units, may be fractional) and radii (lattice
 * units).  phi = max over seeds of tanh((R - r) dx / (sqrt2 W0)); U = U0; theta = theta0.
 * Populations: g = w phi, h = (A + B q/zeta) U, f = w theta.  Returns 0. */
int ora_init_seed(ora_sim* s, int n, const double* centres, const double* radii, double U0, double theta0);

/* Replace the state by caller-given post-streaming populations (layout [Q][site]);
 * f may be NULL when q_theta == 0.  Moments are recomputed as population sums.
 * theta0 is used as the frozen temperature when q_theta == 0. */
void ora_set_state(ora_sim* s, const double* g, const double* h, const double* f, double theta0);
void ora_get_pops(const ora_sim* s, int field /*0 g, 1 h, 2 f*/, double* out);
void ora_get_fields(const ora_sim* s, double* phi, double* U, double* theta);

/* Advance n steps (Sec. 3.4 "Algorithm implementation"). */
void ora_step(ora_sim* s, int64_t n);

/* Per-site terms of the last U update, for invariant checks: S + Q_U/zeta
 * (the source multiplying w_i dt in Eq. (LBE_Eq_Transport)). */
void ora_get_usource(const ora_sim* s, double* out);

/* Diagnostics.  Sums: [sum phi, sum U, sum theta, sum zeta(phi)(1+(1-k)U)]. */
void ora_sums(const ora_sim* s, double out[4]);
/* Tip along +axis (0, 1, 2 = x, y, z) from node (cx, cy, cz): first crossing
 * phi >= 0 > phi_next, linear interpolation.  Returns the tip coordinate along the axis
 * (lattice units) or -1 when there is no crossing.  rho (may be NULL): tip radius in
 * lattice units from the parabola fit in each plane spanned by the axis and another axis
 * with more than one node, averaged (-1 when undefined). */
double ora_tip(const ora_sim* s, int axis, int cx, int cy, int cz, double* rho);

int64_t ora_steps_done(const ora_sim* s);

/* ---------------------------------------------------------------------
 * Explicit finite-difference solver of the same PDEs (cross-check only).
 * Conservative second-order stencils, forward Euler, zero-flux walls.
 * --------------------------------------------------------------------- */
typedef struct fd_sim fd_sim;
fd_sim* fd_create(int nx, int ny, int nz, int theta_evolves, const ora_params* p);
void fd_destroy(fd_sim* s);
int fd_init_seed(fd_sim* s, int n, const double* centres, const double* radii, double U0, double theta0);
void fd_step(fd_sim* s, int64_t n);
void fd_get_fields(const fd_sim* s, double* phi, double* U, double* theta);

#ifdef __cplusplus
}
#endif
#endif
