/*
 * lbpf_oracle.c -- plain FP64 CPU oracle of the lattice-Boltzmann scheme of
 * Cartalade, Younsi & Plapp, "Lattice Boltzmann simulations of 3D crystal
 * growth: numerical schemes for a phase-field model with anti-trapping
 * current" (arXiv 1602.07483).
 *
 * TEST INFRASTRUCTURE ONLY (see lbpf_oracle.h).  Written for reading, not for
 * speed: whole-field arrays, one pass per quantity, the paper's order of
 * operations, no blocking and no fusion.  Compile with -O2 -ffp-contract=off.
 *
 * Readings of the paper where it is silent or garbled (each is listed with
 * its reason in the design notes of the repository):
 *  R1 time levels: the phi collision uses phi^n, U^n, theta^n; the U and theta
 *     collisions use phi^{n+1} for every phi-dependent factor and
 *     dphi/dt = (phi^{n+1} - phi^n)/dt (explicit Euler, Sec. 3.4); the
 *     [1+(1-k)U] factors use U^n.
 *  R2 seed profile: phi = tanh((R - r) dx / (sqrt2 W0)) with R, r in lattice units.
 *  R3 undefined normal: when |grad phi|^2 < grad2_min, a_s = 1, N = 0, n = 0.
 *  R4 boundary nodes (any coordinate 0 or N-1): a_s^2 := 1 in the 1/a_s^2
 *     prefactor and in the non-local term of the collision; eta_phi and N keep
 *     the computed a_s.
 *  R5 gradients: 2-point centred differences with mirror ghosts
 *     phi(-1) = phi(0), phi(N) = phi(N-1).
 *  R6 div(D q F): compact face form with face q = mean of the nodal values.
 *  R7 derivative rule of Eq. (Derivees_As): beta, gamma are the two other axes.
 *  R8 derivatives of Eq. (As_K41-K61): derived analytically (not in the paper).
 *  R9 bounce-back: halfway (link-wise): g_i(x, t+dt) = g*_{i'}(x, t) whenever
 *     x - e_i lies outside the domain.
 *  R10 initial populations: g = w phi, h = (A + B q/zeta) U, f = w theta.
 *  R11 the source weights w_i of Eq. (LBE_Eq_Transport) are the U lattice's w.
 */
#include "lbpf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Lattices: Table 1 (vectors e_i) and Table 2 (w_i, A_i, B_i, e^2), Sec. 3.4 */
/* ------------------------------------------------------------------------ */

static const int32_t E7[7][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

/* D3Q15 = D3Q7 plus the eight cube diagonals e_7..e_14 */
static const int32_t E15[15][3] = {
    {0, 0, 0},   {1, 0, 0},  {0, 1, 0},   {-1, 0, 0},  {0, -1, 0},
    {0, 0, 1},   {0, 0, -1}, {1, 1, 1},   {-1, 1, 1},  {-1, -1, 1},
    {1, -1, 1},  {1, 1, -1}, {-1, 1, -1}, {-1, -1, -1}, {1, -1, -1}};

/* D3Q19 = D3Q7 plus the twelve edge diagonals e_7..e_18 */
static const int32_t E19[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0},  {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, 1, 0},   {-1, 1, 0},  {1, -1, 0},
    {-1, -1, 0}, {1, 0, 1}, {-1, 0, 1},  {1, 0, -1},  {-1, 0, -1},
    {0, 1, 1},  {0, -1, 1}, {0, 1, -1},  {0, -1, -1}};

/* 2D lattices of Tables 3-4 (Sec. 3.4), stored with e_z = 0 so that an nz = 1 grid
 * runs the paper's 2D scheme */
static const int32_t E5[5][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}};
static const int32_t E9[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};

typedef struct {
  int q;
  int32_t e[19][3];
  double w[19], A[19], B[19];
  double e2;
  int32_t opp[19];
} lattice;

static int make_lattice(int q, lattice* L) {
  memset(L, 0, sizeof(*L));
  L->q = q;
  const int32_t(*E)[3];
  double w0, w1, wd, B0, B1, Bd;
  if (q == 7) {
    E = E7; L->e2 = 1.0 / 4.0;
    w0 = 1.0 / 4.0; w1 = 1.0 / 8.0; wd = 0.0;
    B0 = -3.0 / 4.0; B1 = 1.0 / 8.0; Bd = 0.0;
  } else if (q == 15) {
    E = E15; L->e2 = 1.0 / 3.0;
    w0 = 2.0 / 9.0; w1 = 1.0 / 9.0; wd = 1.0 / 72.0;
    B0 = -7.0 / 9.0; B1 = 1.0 / 9.0; Bd = 1.0 / 72.0;
  } else if (q == 19) {
    E = E19; L->e2 = 1.0 / 3.0;
    w0 = 1.0 / 3.0; w1 = 1.0 / 18.0; wd = 1.0 / 36.0;
    B0 = -2.0 / 3.0; B1 = 1.0 / 18.0; Bd = 1.0 / 36.0;
  } else if (q == 5) {
    E = E5; L->e2 = 1.0 / 3.0;
    w0 = 1.0 / 3.0; w1 = 1.0 / 6.0; wd = 0.0;
    B0 = -2.0 / 3.0; B1 = 1.0 / 6.0; Bd = 0.0;
  } else if (q == 9) {
    E = E9; L->e2 = 1.0 / 3.0;
    w0 = 4.0 / 9.0; w1 = 1.0 / 9.0; wd = 1.0 / 36.0;
    B0 = -5.0 / 9.0; B1 = 1.0 / 9.0; Bd = 1.0 / 36.0;
  } else {
    return -1;
  }
  /* number of axis directions: 6 in 3D, 4 in 2D */
  const int naxis = (q == 5 || q == 9) ? 4 : 6;
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < 3; ++a) L->e[i][a] = E[i][a];
    L->w[i] = (i == 0) ? w0 : (i <= naxis ? w1 : wd);
    L->A[i] = (i == 0) ? 1.0 : 0.0;
    L->B[i] = (i == 0) ? B0 : (i <= naxis ? B1 : Bd);
  }
  /* opposite direction: the j with e_j = -e_i */
  for (int i = 0; i < q; ++i) {
    L->opp[i] = -1;
    for (int j = 0; j < q; ++j)
      if (E[j][0] == -E[i][0] && E[j][1] == -E[i][1] && E[j][2] == -E[i][2]) L->opp[i] = j;
  }
  return 0;
}

int ora_lattice(int q, int32_t* e, double* w, double* A, double* B, double* e2, int32_t* opp) {
  lattice L;
  if (make_lattice(q, &L)) return -1;
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
    w[i] = L.w[i]; A[i] = L.A[i]; B[i] = L.B[i]; opp[i] = L.opp[i];
  }
  *e2 = L.e2;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Anisotropy (Eq. Anisotropic-Function_As, Eq. Derivees_As, Eq. As_K41-K61) */
/* ------------------------------------------------------------------------ */

double ora_aniso(int aniso, double eps1, double eps2, const double g[3], double das[3]) {
  const double G2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  const double S4 = g[0] * g[0] * g[0] * g[0] + g[1] * g[1] * g[1] * g[1] + g[2] * g[2] * g[2] * g[2];
  const double G4 = G2 * G2, G6 = G4 * G2;
  if (aniso == 0) {
    /* a_s = 1 - 3 eps + 4 eps sum n_a^4, with n = -grad phi/|grad phi| */
    const double eps = eps1;
    const double as = 1.0 - 3.0 * eps + 4.0 * eps * S4 / G4;
    if (das) {
      /* Eq. (Derivees_As): for alpha, beta, gamma = (x,y,z), (y,x,z), (z,x,y) */
      for (int a = 0; a < 3; ++a) {
        const int b = (a == 0) ? 1 : 0;
        const int c = (a == 2) ? 1 : 2;
        const double pa = g[a], pb = g[b], pc = g[c];
        das[a] = -16.0 * eps / G6 * pa *
                 (pb * pb * pb * pb - pa * pa * pb * pb - pa * pa * pc * pc + pc * pc * pc * pc);
      }
    }
    return as;
  } else {
    /* a_s = 1 + eps(sum n^4 - 3/5) + delta(3 sum n^4 + 66 nx^2 ny^2 nz^2 - 17/7) */
    const double P3 = g[0] * g[0] * g[1] * g[1] * g[2] * g[2];
    const double as = 1.0 + eps1 * (S4 / G4 - 3.0 / 5.0) +
                      eps2 * (3.0 * S4 / G4 + 66.0 * P3 / G6 - 17.0 / 7.0);
    if (das) {
      const double G8 = G4 * G4;
      for (int a = 0; a < 3; ++a) {
        const int b = (a == 0) ? 1 : 0;
        const int c = (a == 2) ? 1 : 2;
        /* d(S4/G^4)/d phi_a = 4 phi_a (phi_a^2 G^2 - S4) / G^6 */
        const double dS = 4.0 * g[a] * (g[a] * g[a] * G2 - S4) / G6;
        /* d(P3/G^6)/d phi_a = 2 phi_a phi_b^2 phi_c^2 (G^2 - 3 phi_a^2) / G^8 */
        const double dP = 2.0 * g[a] * g[b] * g[b] * g[c] * g[c] * (G2 - 3.0 * g[a] * g[a]) / G8;
        das[a] = (eps1 + 3.0 * eps2) * dS + 66.0 * eps2 * dP;
      }
    }
    return as;
  }
}

/* ------------------------------------------------------------------------ */
/* Equilibria: Eq. (Feq_Phase) and Eq. (Feq_Transport)                       */
/* ------------------------------------------------------------------------ */

static void geq(const lattice* L, double phi, const double N[3], double c, double* g0) {
  /* g_i^(0) = w_i (phi - e^-2 e_i.N dt/dx W0^2/tau0), c = dt/dx W0^2/tau0 */
  for (int i = 0; i < L->q; ++i) {
    const double eN = L->e[i][0] * N[0] + L->e[i][1] * N[1] + L->e[i][2] * N[2];
    g0[i] = L->w[i] * (phi - eN * c / L->e2);
  }
}

static void heq(const lattice* L, double U, double qz, const double J[3], double dt_dx, double* h0) {
  /* h_i^(0) = A_i U + B_i (q/zeta U + e^-2 e_i.J dt/dx) */
  for (int i = 0; i < L->q; ++i) {
    const double eJ = L->e[i][0] * J[0] + L->e[i][1] * J[1] + L->e[i][2] * J[2];
    h0[i] = L->A[i] * U + L->B[i] * (qz * U + eJ * dt_dx / L->e2);
  }
}

void ora_geq(int q, double phi, const double N[3], double c, double* g0) {
  lattice L;
  if (make_lattice(q, &L) == 0) geq(&L, phi, N, c, g0);
}

void ora_heq(int q, double U, double qz, const double J[3], double dt_dx, double* h0) {
  lattice L;
  if (make_lattice(q, &L) == 0) heq(&L, U, qz, J, dt_dx, h0);
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */

struct ora_sim {
  int nx, ny, nz;
  int64_t n;          /* sites */
  lattice Lp, Lu, Lt; /* phi, U, theta lattices */
  int has_theta;
  ora_params p;
  double theta0;
  double *g, *h, *f;  /* post-streaming populations [Q][site] */
  double *gs;         /* post-collision scratch, largest Q */
  double *phi, *U, *theta;
  double *phi_new, *usrc;
  double *tmp[8];     /* per-site work arrays */
  int64_t steps;
};

static inline int64_t IDX(const ora_sim* s, int x, int y, int z) {
  return ((int64_t)z * s->ny + y) * s->nx + x;
}

/* mirror ghost index (R5): -1 -> 0, N -> N-1 */
static inline int mir(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

ora_sim* ora_create(int nx, int ny, int nz, int q_phi, int q_u, int q_theta, const ora_params* p) {
  if (nx < 1 || ny < 1 || nz < 1) return NULL;
  ora_sim* s = (ora_sim*)calloc(1, sizeof(ora_sim));
  s->nx = nx; s->ny = ny; s->nz = nz;
  s->n = (int64_t)nx * ny * nz;
  s->p = *p;
  if (make_lattice(q_phi, &s->Lp) || make_lattice(q_u, &s->Lu)) { free(s); return NULL; }
  s->has_theta = q_theta != 0;
  if (s->has_theta && make_lattice(q_theta, &s->Lt)) { free(s); return NULL; }
  const int64_t n = s->n;
  s->g = (double*)calloc((size_t)(q_phi * n), sizeof(double));
  s->h = (double*)calloc((size_t)(q_u * n), sizeof(double));
  s->f = s->has_theta ? (double*)calloc((size_t)(q_theta * n), sizeof(double)) : NULL;
  s->gs = (double*)calloc((size_t)(19 * n), sizeof(double));
  s->phi = (double*)calloc((size_t)n, sizeof(double));
  s->U = (double*)calloc((size_t)n, sizeof(double));
  s->theta = (double*)calloc((size_t)n, sizeof(double));
  s->phi_new = (double*)calloc((size_t)n, sizeof(double));
  s->usrc = (double*)calloc((size_t)n, sizeof(double));
  for (int k = 0; k < 8; ++k) s->tmp[k] = (double*)calloc((size_t)n, sizeof(double));
  return s;
}

void ora_destroy(ora_sim* s) {
  if (!s) return;
  free(s->g); free(s->h); free(s->f); free(s->gs);
  free(s->phi); free(s->U); free(s->theta); free(s->phi_new); free(s->usrc);
  for (int k = 0; k < 8; ++k) free(s->tmp[k]);
  free(s);
}

int64_t ora_steps_done(const ora_sim* s) { return s->steps; }

/* zeroth moments of the post-streaming populations */
static void moment(const lattice* L, const double* pop, int64_t n, double* out) {
  for (int64_t x = 0; x < n; ++x) {
    double m = 0.0;
    for (int i = 0; i < L->q; ++i) m += pop[(int64_t)i * n + x];
    out[x] = m;
  }
}

int ora_init_seed(ora_sim* s, int nseed, const double* c, const double* R, double U0, double theta0) {
  const ora_params* p = &s->p;
  const double k = p->k;
  s->theta0 = theta0;
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        /* R2: phi = tanh((R - r) dx / (sqrt2 W0)); overlapping seeds take the max */
        double ph = -1.0;
        for (int m = 0; m < nseed; ++m) {
          const double dxs = x - c[3 * m], dys = y - c[3 * m + 1], dzs = z - c[3 * m + 2];
          const double r = sqrt(dxs * dxs + dys * dys + dzs * dzs);
          const double v = tanh((R[m] - r) * p->dx / (sqrt(2.0) * p->W0));
          if (m == 0 || v > ph) ph = v;
        }
        const int64_t id = IDX(s, x, y, z);
        /* R10: equilibrium-like initial populations */
        for (int i = 0; i < s->Lp.q; ++i) s->g[(int64_t)i * s->n + id] = s->Lp.w[i] * ph;
        const double q = 0.5 * (1.0 - ph);
        const double zeta = 0.5 * ((1.0 + k) - (1.0 - k) * ph);
        for (int i = 0; i < s->Lu.q; ++i)
          s->h[(int64_t)i * s->n + id] = (s->Lu.A[i] + s->Lu.B[i] * q / zeta) * U0;
        if (s->has_theta)
          for (int i = 0; i < s->Lt.q; ++i) s->f[(int64_t)i * s->n + id] = s->Lt.w[i] * theta0;
      }
  moment(&s->Lp, s->g, s->n, s->phi);
  moment(&s->Lu, s->h, s->n, s->U);
  if (s->has_theta) moment(&s->Lt, s->f, s->n, s->theta);
  else for (int64_t x = 0; x < s->n; ++x) s->theta[x] = theta0;
  s->steps = 0;
  return 0;
}

void ora_set_state(ora_sim* s, const double* g, const double* h, const double* f, double theta0) {
  memcpy(s->g, g, sizeof(double) * (size_t)(s->Lp.q * s->n));
  memcpy(s->h, h, sizeof(double) * (size_t)(s->Lu.q * s->n));
  if (s->has_theta && f) memcpy(s->f, f, sizeof(double) * (size_t)(s->Lt.q * s->n));
  s->theta0 = theta0;
  moment(&s->Lp, s->g, s->n, s->phi);
  moment(&s->Lu, s->h, s->n, s->U);
  if (s->has_theta) moment(&s->Lt, s->f, s->n, s->theta);
  else for (int64_t x = 0; x < s->n; ++x) s->theta[x] = theta0;
}

void ora_get_pops(const ora_sim* s, int field, double* out) {
  if (field == 0) memcpy(out, s->g, sizeof(double) * (size_t)(s->Lp.q * s->n));
  else if (field == 1) memcpy(out, s->h, sizeof(double) * (size_t)(s->Lu.q * s->n));
  else if (field == 2 && s->has_theta) memcpy(out, s->f, sizeof(double) * (size_t)(s->Lt.q * s->n));
}

void ora_get_fields(const ora_sim* s, double* phi, double* U, double* theta) {
  if (phi) memcpy(phi, s->phi, sizeof(double) * (size_t)s->n);
  if (U) memcpy(U, s->U, sizeof(double) * (size_t)s->n);
  if (theta) memcpy(theta, s->theta, sizeof(double) * (size_t)s->n);
}

void ora_get_usource(const ora_sim* s, double* out) {
  memcpy(out, s->usrc, sizeof(double) * (size_t)s->n);
}

/* centred gradient of a nodal field with mirror ghosts (R5), physical units */
static void grad_at(const ora_sim* s, const double* a, int x, int y, int z, double g[3]) {
  const double inv2dx = 1.0 / (2.0 * s->p.dx);
  g[0] = (a[IDX(s, mir(x + 1, s->nx), y, z)] - a[IDX(s, mir(x - 1, s->nx), y, z)]) * inv2dx;
  g[1] = (a[IDX(s, x, mir(y + 1, s->ny), z)] - a[IDX(s, x, mir(y - 1, s->ny), z)]) * inv2dx;
  g[2] = (a[IDX(s, x, y, mir(z + 1, s->nz))] - a[IDX(s, x, y, mir(z - 1, s->nz))]) * inv2dx;
}

/* boundary node (R4): on a wall that the phase-field lattice has links through
 * (the 2D lattices have none through the z walls) */
static inline int is_boundary(const ora_sim* s, int x, int y, int z) {
  int zlinks = 0;
  for (int i = 0; i < s->Lp.q; ++i) zlinks |= s->Lp.e[i][2] != 0;
  return x == 0 || y == 0 || x == s->nx - 1 || y == s->ny - 1 || (zlinks && (z == 0 || z == s->nz - 1));
}

static inline int inside(const ora_sim* s, int x, int y, int z) {
  return x >= 0 && y >= 0 && z >= 0 && x < s->nx && y < s->ny && z < s->nz;
}

/* Streaming, Eq. (Deplacement_STD), with halfway bounce-back (R9):
 * pop_i(x, t+dt) = post_i(x - e_i) if x - e_i is inside, else post_{i'}(x). */
static void stream(const ora_sim* s, const lattice* L, const double* post, double* pop) {
  const int64_t n = s->n;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        const int64_t id = IDX(s, x, y, z);
        for (int i = 0; i < L->q; ++i) {
          const int xs = x - L->e[i][0], ys = y - L->e[i][1], zs = z - L->e[i][2];
          if (inside(s, xs, ys, zs))
            pop[(int64_t)i * n + id] = post[(int64_t)i * n + IDX(s, xs, ys, zs)];
          else
            pop[(int64_t)i * n + id] = post[(int64_t)L->opp[i] * n + id];
        }
      }
}

/* ---- phase field: Eqs. (LBE_Eq_Phase)-(LBE_RelaxationTime), collision stage
 *      of Sec. 3.4, using phi^n, U^n, theta^n (R1) ---- */
static void step_phi(ora_sim* s) {
  const ora_params* p = &s->p;
  const lattice* L = &s->Lp;
  const int64_t n = s->n;
  const double W2t = p->W0 * p->W0 / p->tau0;
  const double c_neq = p->dt / p->dx * W2t;      /* dt/dx W0^2/tau0 in g^(0) */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        const int64_t id = IDX(s, x, y, z);
        const double ph = s->phi[id];
        double gr[3], das[3], N[3] = {0.0, 0.0, 0.0};
        grad_at(s, s->phi, x, y, z, gr);
        const double G2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
        double as = 1.0;
        if (G2 >= p->grad2_min) {          /* R3 */
          as = ora_aniso(p->aniso, p->eps1, p->eps2, gr, das);
          /* Eq. (TermesAnisotropes): N = |grad phi|^2 a_s d a_s / d(grad phi) */
          for (int a = 0; a < 3; ++a) N[a] = G2 * as * das[a];
        }
        const double as2 = as * as;
        /* Eq. (LBE_RelaxationTime) */
        const double eta = as2 * W2t * p->dt / (p->dx * p->dx) / L->e2 + 0.5;
        /* Eq. (LBE_SourceTerm) */
        const double omp2 = 1.0 - ph * ph;
        const double Q = (ph - p->lambda * (p->Mc_inf * s->U[id] + s->theta[id]) * omp2) * omp2;
        double g0[19];
        geq(L, ph, N, c_neq, g0);
        const int bnd = is_boundary(s, x, y, z);
        const double a2 = bnd ? 1.0 : as2; /* R4 */
        for (int i = 0; i < L->q; ++i) {
          const double gi = s->g[(int64_t)i * n + id];
          /* non-local term g_i(x + e_i, t); x + e_i is inside for non-boundary nodes */
          double gnl = 0.0;
          if (!bnd)
            gnl = s->g[(int64_t)i * n + IDX(s, x + L->e[i][0], y + L->e[i][1], z + L->e[i][2])];
          s->gs[(int64_t)i * n + id] =
              (gi - (1.0 - a2) * gnl - (gi - g0[i]) / eta + L->w[i] * Q * p->dt / p->tau0) / a2;
        }
      }
  stream(s, L, s->gs, s->g);
  moment(L, s->g, n, s->phi_new);
}

/* ---- supersaturation: Eqs. (Supersaturation_Bis)-(RelaxationTime_Concentration),
 *      with phi := phi^{n+1}, dphi/dt Euler, U^n (R1) ---- */
static void step_U(ora_sim* s) {
  const ora_params* p = &s->p;
  const lattice* L = &s->Lu;
  const int64_t n = s->n;
  const double k = p->k;
  double* q = s->tmp[0];
  double* iz = s->tmp[1];   /* 1/zeta */
  double* qz = s->tmp[2];   /* q/zeta */
  const double* ph1 = s->phi_new;
  for (int64_t id = 0; id < n; ++id) {
    q[id] = 0.5 * (1.0 - ph1[id]);                              /* q(phi) */
    const double zeta = 0.5 * ((1.0 + k) - (1.0 - k) * ph1[id]); /* zeta(phi) */
    iz[id] = 1.0 / zeta;
    qz[id] = q[id] / zeta;
  }
  /* Eq. (RelaxationTime_Concentration) */
  const double etaU = p->D * p->dt / (p->dx * p->dx) / L->e2 + 0.5;
  const double dt_dx = p->dt / p->dx;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        const int64_t id = IDX(s, x, y, z);
        const double U = s->U[id];
        const double dphidt = (ph1[id] - s->phi[id]) / p->dt;
        double gph[3], gqz[3], F[3];
        grad_at(s, ph1, x, y, z, gph);
        grad_at(s, qz, x, y, z, gqz);
        grad_at(s, iz, x, y, z, F);                 /* F = grad(1/zeta) */
        /* R6: div(D q F) in compact face form */
        double divDqF = 0.0;
        {
          const int xp = mir(x + 1, s->nx), xm = mir(x - 1, s->nx);
          const int yp = mir(y + 1, s->ny), ym = mir(y - 1, s->ny);
          const int zp = mir(z + 1, s->nz), zm = mir(z - 1, s->nz);
          const int64_t nb[3][2] = {{IDX(s, xp, y, z), IDX(s, xm, y, z)},
                                    {IDX(s, x, yp, z), IDX(s, x, ym, z)},
                                    {IDX(s, x, y, zp), IDX(s, x, y, zm)}};
          for (int a = 0; a < 3; ++a) {
            const double qp = 0.5 * (q[id] + q[nb[a][0]]);
            const double qm = 0.5 * (q[id] + q[nb[a][1]]);
            divDqF += qp * (iz[nb[a][0]] - iz[id]) - qm * (iz[id] - iz[nb[a][1]]);
          }
          divDqF *= p->D / (p->dx * p->dx);
        }
        /* Eq. (AntiTrapping_Current): j_at = -(1/(2 sqrt2)) W0 [1+(1-k)U] dphi/dt grad phi/|grad phi| */
        double jat[3] = {0.0, 0.0, 0.0};
        const double G2 = gph[0] * gph[0] + gph[1] * gph[1] + gph[2] * gph[2];
        if (p->antitrapping && G2 >= p->grad2_min) {
          const double G = sqrt(G2);
          const double amp = -p->W0 / (2.0 * sqrt(2.0)) * (1.0 + (1.0 - k) * U) * dphidt;
          for (int a = 0; a < 3; ++a) jat[a] = amp * gph[a] / G;
        }
        /* Eq. (Def_Jtot), Eq. (Def_S), Eq. (Def_Qu) */
        double J[3];
        for (int a = 0; a < 3; ++a) J[a] = p->D * (gqz[a] + q[id] * F[a]) * U + jat[a] * iz[id];
        const double S = U * divDqF + (jat[0] * F[0] + jat[1] * F[1] + jat[2] * F[2]);
        const double QU = (1.0 + (1.0 - k) * U) * 0.5 * dphidt;
        const double src = S + QU * iz[id];
        s->usrc[id] = src;
        double h0[19];
        heq(L, U, qz[id], J, dt_dx, h0);
        /* Eq. (LBE_Eq_Transport), collision part */
        for (int i = 0; i < L->q; ++i) {
          const double hi = s->h[(int64_t)i * n + id];
          s->gs[(int64_t)i * n + id] = hi - (hi - h0[i]) / etaU + L->w[i] * src * p->dt;
        }
      }
  stream(s, L, s->gs, s->h);
}

/* ---- temperature: Eqs. (LBE_Eq_Temp)-(ThermalDiffusivity), Q_theta = dphi/dt / 2 ---- */
static void step_theta(ora_sim* s) {
  const ora_params* p = &s->p;
  const lattice* L = &s->Lt;
  const int64_t n = s->n;
  const double etaT = p->kappa * p->dt / (p->dx * p->dx) / L->e2 + 0.5;
  for (int64_t id = 0; id < n; ++id) {
    const double th = s->theta[id];
    const double Qth = 0.5 * (s->phi_new[id] - s->phi[id]) / p->dt;
    for (int i = 0; i < L->q; ++i) {
      const double fi = s->f[(int64_t)i * n + id];
      s->gs[(int64_t)i * n + id] = fi - (fi - L->w[i] * th) / etaT + L->w[i] * Qth * p->dt;
    }
  }
  stream(s, L, s->gs, s->f);
}

void ora_step(ora_sim* s, int64_t nsteps) {
  for (int64_t t = 0; t < nsteps; ++t) {
    step_phi(s);                                   /* phi first (Sec. 3.4) */
    step_U(s);                                     /* then U with phi^{n+1} */
    if (s->has_theta) step_theta(s);               /* then theta */
    /* new moments */
    memcpy(s->phi, s->phi_new, sizeof(double) * (size_t)s->n);
    moment(&s->Lu, s->h, s->n, s->U);
    if (s->has_theta) moment(&s->Lt, s->f, s->n, s->theta);
    s->steps++;
  }
}

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */

void ora_sums(const ora_sim* s, double out[4]) {
  const double k = s->p.k;
  double a = 0, b = 0, c = 0, d = 0;
  for (int64_t id = 0; id < s->n; ++id) {
    a += s->phi[id];
    b += s->U[id];
    c += s->theta[id];
    const double zeta = 0.5 * ((1.0 + k) - (1.0 - k) * s->phi[id]);
    d += zeta * (1.0 + (1.0 - k) * s->U[id]);
  }
  out[0] = a; out[1] = b; out[2] = c; out[3] = d;
}

/* first crossing phi_i >= 0 > phi_{i+1} scanning +axis from node p0 along its line */
static double crossing(const ora_sim* s, int axis, const int p0[3]) {
  const int n[3] = {s->nx, s->ny, s->nz};
  for (int a = 0; a < 3; ++a)
    if (p0[a] < 0 || p0[a] >= n[a]) return -1.0;
  int p[3] = {p0[0], p0[1], p0[2]};
  int q[3] = {p0[0], p0[1], p0[2]};
  for (int t = p0[axis]; t + 1 < n[axis]; ++t) {
    p[axis] = t;
    q[axis] = t + 1;
    const double a = s->phi[IDX(s, p[0], p[1], p[2])], b = s->phi[IDX(s, q[0], q[1], q[2])];
    if (a >= 0.0 && b < 0.0) return t + a / (a - b);
  }
  return -1.0;
}

/* Tip along +axis from node c (Sec. 4.1 tip reading): x_tip is the first crossing on the
 * line through c; rho is the least-squares parabola x(j) = x_tip - j^2/(2 rho) through the
 * crossings of the lines offset by j = +-1..+-4 along each other axis b, one fit per plane
 * (axis, b), averaged over the planes that exist (extent along b > 1: both in 3D, the
 * grid plane on an nz = 1 grid). */
double ora_tip(const ora_sim* s, int axis, int cx, int cy, int cz, double* rho) {
  const int c[3] = {cx, cy, cz};
  const int n[3] = {s->nx, s->ny, s->nz};
  const double xt = crossing(s, axis, c);
  if (rho) {
    double sum = 0.0;
    int planes = 0, ok_all = 1;
    for (int b = 0; b < 3; ++b) {
      if (b == axis || n[b] == 1) continue;
      double num = 0.0, den = 0.0; /* least squares in u = 1/(2 rho): u = num / den */
      int ok = xt >= 0.0;
      for (int j = -4; j <= 4; ++j) {
        if (j == 0) continue;
        int p[3] = {cx, cy, cz};
        p[b] += j;
        const double xj = crossing(s, axis, p);
        if (xj < 0.0) ok = 0;
        num += (double)(j * j) * (xt - xj);
        den += (double)(j * j) * (double)(j * j);
      }
      if (ok && num > 0.0) sum += den / (2.0 * num);
      else ok_all = 0;
      ++planes;
    }
    *rho = (planes > 0 && ok_all) ? sum / planes : -1.0;
  }
  return xt;
}
