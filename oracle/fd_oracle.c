/*
 * fd_oracle.c -- explicit finite-difference solver of the phase-field PDEs of
 * Sec. 2 (Eqs. PhaseField_KarmaRappel, Concentration_Echebarria, Temp_Ramirez),
 * used only as an independent cross-check of the lattice-Boltzmann oracle, the
 * way the paper validates its LB schemes against finite-difference codes
 * (Sec. 4.1, Sec. 4.2).  TEST INFRASTRUCTURE ONLY.
 *
 * Discretisation (this file's own choice; the paper prints no FD scheme):
 *  - node-centred grid, zero-flux walls at x = -1/2 and x = N - 1/2;
 *  - nodal gradients by centred differences with mirror ghosts (for n, a_s, N, j_at);
 *  - every divergence in conservative face form: face coefficient = mean of the two
 *    nodal values, face flux through a wall = 0;
 *  - forward Euler; dphi/dt from the phase-field equation is used in the U and
 *    theta equations of the same step.
 */
#include "lbpf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct fd_sim {
  int nx, ny, nz;
  int64_t n;
  int theta_evolves;
  ora_params p;
  double *phi, *U, *theta;
  double *as2, *N[3], *jat[3], *dphi, *q, *tmp;
};

static inline int64_t FI(const fd_sim* s, int x, int y, int z) {
  return ((int64_t)z * s->ny + y) * s->nx + x;
}
static inline int fmir(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

fd_sim* fd_create(int nx, int ny, int nz, int theta_evolves, const ora_params* p) {
  fd_sim* s = (fd_sim*)calloc(1, sizeof(fd_sim));
  s->nx = nx; s->ny = ny; s->nz = nz;
  s->n = (int64_t)nx * ny * nz;
  s->theta_evolves = theta_evolves;
  s->p = *p;
  const size_t n = (size_t)s->n;
  s->phi = calloc(n, sizeof(double)); s->U = calloc(n, sizeof(double));
  s->theta = calloc(n, sizeof(double)); s->as2 = calloc(n, sizeof(double));
  for (int a = 0; a < 3; ++a) { s->N[a] = calloc(n, sizeof(double)); s->jat[a] = calloc(n, sizeof(double)); }
  s->dphi = calloc(n, sizeof(double)); s->q = calloc(n, sizeof(double)); s->tmp = calloc(n, sizeof(double));
  return s;
}

void fd_destroy(fd_sim* s) {
  if (!s) return;
  free(s->phi); free(s->U); free(s->theta); free(s->as2);
  for (int a = 0; a < 3; ++a) { free(s->N[a]); free(s->jat[a]); }
  free(s->dphi); free(s->q); free(s->tmp);
  free(s);
}

int fd_init_seed(fd_sim* s, int nseed, const double* c, const double* R, double U0, double theta0) {
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        double ph = -1.0;
        for (int m = 0; m < nseed; ++m) {
          const double a = x - c[3 * m], b = y - c[3 * m + 1], d = z - c[3 * m + 2];
          const double v = tanh((R[m] - sqrt(a * a + b * b + d * d)) * s->p.dx / (sqrt(2.0) * s->p.W0));
          if (m == 0 || v > ph) ph = v;
        }
        const int64_t id = FI(s, x, y, z);
        s->phi[id] = ph; s->U[id] = U0; s->theta[id] = theta0;
      }
  return 0;
}

void fd_get_fields(const fd_sim* s, double* phi, double* U, double* theta) {
  if (phi) memcpy(phi, s->phi, sizeof(double) * (size_t)s->n);
  if (U) memcpy(U, s->U, sizeof(double) * (size_t)s->n);
  if (theta) memcpy(theta, s->theta, sizeof(double) * (size_t)s->n);
}

/* conservative divergence of  c_face * (a(x+e) - a(x))/dx  (zero flux at walls) */
static double div_cgrad(const fd_sim* s, const double* c, const double* a, int x, int y, int z) {
  const int dims[3] = {s->nx, s->ny, s->nz};
  const int pos[3] = {x, y, z};
  const int64_t id = FI(s, x, y, z);
  double acc = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    for (int sg = -1; sg <= 1; sg += 2) {
      int nb[3] = {x, y, z};
      nb[ax] = pos[ax] + sg;
      if (nb[ax] < 0 || nb[ax] >= dims[ax]) continue; /* wall face: zero flux */
      const int64_t jd = FI(s, nb[0], nb[1], nb[2]);
      const double cf = c ? 0.5 * (c[id] + c[jd]) : 1.0;
      acc += cf * (a[jd] - a[id]);
    }
  }
  return acc / (s->p.dx * s->p.dx);
}

/* conservative divergence of a nodal vector field v (face value = mean; wall face = 0) */
static double div_vec(const fd_sim* s, double* const v[3], int x, int y, int z) {
  const int dims[3] = {s->nx, s->ny, s->nz};
  const int pos[3] = {x, y, z};
  const int64_t id = FI(s, x, y, z);
  double acc = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    for (int sg = -1; sg <= 1; sg += 2) {
      int nb[3] = {x, y, z};
      nb[ax] = pos[ax] + sg;
      if (nb[ax] < 0 || nb[ax] >= dims[ax]) continue;
      const int64_t jd = FI(s, nb[0], nb[1], nb[2]);
      acc += sg * 0.5 * (v[ax][id] + v[ax][jd]);
    }
  }
  return acc / s->p.dx;
}

static void fd_grad(const fd_sim* s, const double* a, int x, int y, int z, double g[3]) {
  const double h = 1.0 / (2.0 * s->p.dx);
  g[0] = (a[FI(s, fmir(x + 1, s->nx), y, z)] - a[FI(s, fmir(x - 1, s->nx), y, z)]) * h;
  g[1] = (a[FI(s, x, fmir(y + 1, s->ny), z)] - a[FI(s, x, fmir(y - 1, s->ny), z)]) * h;
  g[2] = (a[FI(s, x, y, fmir(z + 1, s->nz))] - a[FI(s, x, y, fmir(z - 1, s->nz))]) * h;
}

void fd_step(fd_sim* s, int64_t nsteps) {
  const ora_params* p = &s->p;
  const double k = p->k, W2 = p->W0 * p->W0;
  for (int64_t t = 0; t < nsteps; ++t) {
    /* nodal a_s^2 and N (Eq. TermesAnisotropes) */
    for (int z = 0; z < s->nz; ++z)
      for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
          const int64_t id = FI(s, x, y, z);
          double g[3], das[3];
          fd_grad(s, s->phi, x, y, z, g);
          const double G2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
          double as = 1.0;
          s->N[0][id] = s->N[1][id] = s->N[2][id] = 0.0;
          if (G2 >= p->grad2_min) {
            as = ora_aniso(p->aniso, p->eps1, p->eps2, g, das);
            for (int a = 0; a < 3; ++a) s->N[a][id] = G2 * as * das[a];
          }
          s->as2[id] = as * as;
        }
    /* Eq. (PhaseField_KarmaRappel) with tau(n) = tau0 a_s^2 */
    for (int z = 0; z < s->nz; ++z)
      for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
          const int64_t id = FI(s, x, y, z);
          const double ph = s->phi[id];
          const double rhs = W2 * div_cgrad(s, s->as2, s->phi, x, y, z) + W2 * div_vec(s, s->N, x, y, z) +
                             ph - ph * ph * ph -
                             p->lambda * (p->Mc_inf * s->U[id] + s->theta[id]) * (1 - ph * ph) * (1 - ph * ph);
          s->dphi[id] = rhs / (p->tau0 * s->as2[id]);
        }
    /* anti-trapping current, Eq. (AntiTrapping_Current), and q(phi) */
    for (int z = 0; z < s->nz; ++z)
      for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
          const int64_t id = FI(s, x, y, z);
          double g[3];
          fd_grad(s, s->phi, x, y, z, g);
          const double G2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
          s->q[id] = 0.5 * (1.0 - s->phi[id]);
          for (int a = 0; a < 3; ++a) s->jat[a][id] = 0.0;
          if (p->antitrapping && G2 >= p->grad2_min) {
            const double amp = -p->W0 / (2.0 * sqrt(2.0)) * (1.0 + (1.0 - k) * s->U[id]) * s->dphi[id] / sqrt(G2);
            for (int a = 0; a < 3; ++a) s->jat[a][id] = amp * g[a];
          }
        }
    /* Eq. (Concentration_Echebarria): zeta dU/dt = div(D q grad U - j_at) + [1+(1-k)U] dphi/dt / 2 */
    for (int z = 0; z < s->nz; ++z)
      for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
          const int64_t id = FI(s, x, y, z);
          const double zeta = 0.5 * ((1.0 + k) - (1.0 - k) * s->phi[id]);
          const double rhs = p->D * div_cgrad(s, s->q, s->U, x, y, z) - div_vec(s, s->jat, x, y, z) +
                             (1.0 + (1.0 - k) * s->U[id]) * 0.5 * s->dphi[id];
          s->tmp[id] = s->U[id] + p->dt * rhs / zeta;
        }
    /* Eq. (Temp_Ramirez) */
    if (s->theta_evolves) {
      /* theta update uses the old theta everywhere: compute into jat[0] scratch */
      for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
          for (int x = 0; x < s->nx; ++x) {
            const int64_t id = FI(s, x, y, z);
            s->jat[0][id] = s->theta[id] + p->dt * (p->kappa * div_cgrad(s, NULL, s->theta, x, y, z) +
                                                    0.5 * s->dphi[id]);
          }
      memcpy(s->theta, s->jat[0], sizeof(double) * (size_t)s->n);
    }
    memcpy(s->U, s->tmp, sizeof(double) * (size_t)s->n);
    for (int64_t id = 0; id < s->n; ++id) s->phi[id] += p->dt * s->dphi[id];
  }
}
