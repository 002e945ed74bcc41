/*
 * Plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see pf_oracle.h).
 *
 * Serial loops, no blocking, no fusion: every operator is written cell by
 * cell, face by face, the way the equations read.  Citations are to the
 * paper's sections and equations:
 *   Eq. F_bulk            Landau bulk energy (Section Theory)
 *   Eqs. F_grad, dF_grad  domain-wall gradient energy and its force
 *   Eqs. F_elec           E = -dF_elec/dP
 *   Eq. TDGL              dP/dt = -dF/dP (+ noise, not used here)
 *   Eqs. rho, Poisson     rho = div P,  eps Lap phi = rho  (Section
 *                         Electrostatics Calculation), boundary kinds listed
 *                         in the same section
 *   Section Time Integration: explicit forward Euler and the
 *                         predictor-corrector ("velocity Verlet") scheme
 *   Section Numerical Performance: the Krylov solve is warm-started from the
 *                         previous step's potential
 *
 * Built twice from this one source: serially (liboracle.so, the reference
 * the tests use) and with OpenMP (liboracle_omp.so, a timing baseline on all
 * host cores).  The "omp parallel for" lines only split the z loops of the
 * operators and the vector updates over threads; they change no arithmetic.
 * The one difference is the dot product of the OpenMP build, which sums
 * fixed chunks of cells and then the chunk sums in chunk order: the same
 * result for any thread count, and the serial sum up to rounding order.
 */
#include "pf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static long ncells(const or_grid* G) { return (long)G->nx * G->ny * G->nz; }

static long cell_index(const or_grid* G, int x, int y, int z) {
  return ((long)z * G->ny + y) * G->nx + x;
}

/* Periodic wrap of an index that is at most one step outside [0, n). */
static int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

static double eps_of(const or_grid* G, long c) { return G->eps ? G->eps[c] : 1.0; }

/* Face of cell (x,y,z) in direction d (0=x,1=y,2=z) on side s (-1 or +1).
 * Returns 1 for an interior face (neighbour index in *nb) and 0 for a z
 * boundary face (its mask type in *btype, voltage in *bvolt). */
static int face_of(const or_grid* G, int x, int y, int z, int d, int s,
                   long* nb, int* btype, double* bvolt) {
  int q[3] = {x, y, z};
  int n[3] = {G->nx, G->ny, G->nz};
  int t = q[d] + s;
  if (d < 2 || G->periodic_z) {
    q[d] = wrap(t, n[d]);
    *nb = cell_index(G, q[0], q[1], q[2]);
    return 1;
  }
  if (t >= 0 && t < n[2]) {
    q[2] = t;
    *nb = cell_index(G, q[0], q[1], q[2]);
    return 1;
  }
  long m = (long)y * G->nx + x;
  if (s < 0) {
    *btype = G->type_lo[m];
    *bvolt = G->volt_lo[m];
  } else {
    *btype = G->type_hi[m];
    *bvolt = G->volt_hi[m];
  }
  return 0;
}

/* Eq. F_bulk: f = a1 sum P_i^2 + a11 sum P_i^4 + a12 (Px^2 Py^2 + Py^2 Pz^2 + Pz^2 Px^2). */
double or_landau_energy(const double* P, long n, double a1, double a11, double a12) {
  double F = 0.0;
  for (long c = 0; c < n; ++c) {
    double x2 = P[c] * P[c], y2 = P[n + c] * P[n + c], z2 = P[2 * n + c] * P[2 * n + c];
    F += a1 * (x2 + y2 + z2) + a11 * (x2 * x2 + y2 * y2 + z2 * z2) +
         a12 * (x2 * y2 + y2 * z2 + z2 * x2);
  }
  return F;
}

/* df/dP_i = 2 a1 P_i + 4 a11 P_i^3 + 2 a12 P_i (P_j^2 + P_k^2), from Eq. F_bulk. */
static void landau_at(const double p[3], double a1, double a11, double a12, double h[3]) {
  for (int i = 0; i < 3; ++i) {
    int j = (i + 1) % 3, k = (i + 2) % 3;
    h[i] = 2.0 * a1 * p[i] + 4.0 * a11 * p[i] * p[i] * p[i] + 2.0 * a12 * p[i] * (p[j] * p[j] + p[k] * p[k]);
  }
}

void or_landau_force(const double* P, long n, double a1, double a11, double a12, double* out) {
#pragma omp parallel for schedule(static)
  for (long c = 0; c < n; ++c) {
    double p[3] = {P[c], P[n + c], P[2 * n + c]}, h[3];
    landau_at(p, a1, a11, a12, h);
    for (int i = 0; i < 3; ++i) out[i * n + c] = h[i];
  }
}

/* Air layers (Section Results, open-circuit device: the top layers of the
 * grid are air, with permittivity 1 against 100 in the film): a cell is
 * ferroelectric below z = nz - n_air.  Air cells carry no polarization, and
 * the film's surface under the air is a free surface for P (zero normal
 * flux in the gradient term, like a z face of the grid). */
static int is_film(const or_grid* G, int z) { return z < G->nz - G->n_air; }

/* Face of cell (x,y,z) in direction d, side s, that carries gradient (wall)
 * energy: an interior face between two film cells. */
static int wall_face(const or_grid* G, int x, int y, int z, int d, int s, long* nb) {
  int bt;
  double bv;
  if (!is_film(G, z) || !face_of(G, x, y, z, d, s, nb, &bt, &bv)) return 0;
  if (d == 2 && !G->periodic_z && !is_film(G, z + s)) return 0;
  return 1;
}

/* P = 0 in the air cells. */
static void zero_air(const or_grid* G, double* P) {
  if (G->n_air <= 0) return;
  long n = ncells(G), nxy = (long)G->nx * G->ny;
  for (int i = 0; i < 3; ++i)
    for (long c = (long)(G->nz - G->n_air) * nxy; c < n; ++c) P[(long)i * n + c] = 0.0;
}

/* Eq. dF_grad/dP: Lap f as the sum over the cell's interior faces of
 * (f_nb - f_c)/dx^2.  A non-periodic z face is dropped (zero normal flux),
 * and so is a film/air face; air cells get 0. */
static double laplacian_at(const or_grid* G, const double* f, int x, int y, int z) {
  long c = cell_index(G, x, y, z);
  double acc = 0.0;
  for (int d = 0; d < 3; ++d)
    for (int s = -1; s <= 1; s += 2) {
      long nb;
      if (wall_face(G, x, y, z, d, s, &nb)) acc += f[nb] - f[c];
    }
  return acc / (G->dx * G->dx);
}

void or_laplacian(const or_grid* G, const double* f, double* out) {
#pragma omp parallel for schedule(static)
  for (int z = 0; z < G->nz; ++z)
    for (int y = 0; y < G->ny; ++y)
      for (int x = 0; x < G->nx; ++x) out[cell_index(G, x, y, z)] = laplacian_at(G, f, x, y, z);
}

/* Face permittivity between cells c and nb: the harmonic mean of the two
 * cell values (reading R4); 1 when no permittivity field is given. */
static double eps_face(const or_grid* G, long c, long nb) {
  if (!G->eps) return 1.0;
  double a = G->eps[c], b = G->eps[nb];
  return 2.0 * a * b / (a + b);
}

/* Eqs. rho, Poisson: div(eps grad phi) = div P.  In SPD form A phi = b with
 * b = -div P + (Dirichlet terms).  div P is the sum of outward normal face
 * values of P divided by dx; face values per reading R3. */
void or_rhs(const or_grid* G, const double* P, double* b) {
  long n = ncells(G);
  double ih = 1.0 / G->dx, ih2 = ih * ih;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < G->nz; ++z)
    for (int y = 0; y < G->ny; ++y)
      for (int x = 0; x < G->nx; ++x) {
        long c = cell_index(G, x, y, z);
        double div = 0.0, dir = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double* Pd = P + (long)d * n;
          for (int s = -1; s <= 1; s += 2) {
            long nb;
            int bt;
            double bv, Pf;
            if (face_of(G, x, y, z, d, s, &nb, &bt, &bv)) {
              Pf = 0.5 * (Pd[c] + Pd[nb]);
            } else if (bt == 1) {
              Pf = Pd[c];                              /* electrode: surface charge screened */
              dir += 2.0 * eps_of(G, c) * bv;          /* ghost 2V - phi_c moved to the rhs */
            } else {
              Pf = 0.0;                                /* open surface */
            }
            div += s * Pf;
          }
        }
        b[c] = -div * ih + dir * ih2;
      }
}

/* A phi = sum over faces of eps_f (phi_c - phi_nb)/dx^2, with the Dirichlet
 * ghost 2V - phi_c taken at V = 0 (flux 2 eps_c phi_c) and Neumann faces
 * contributing nothing (Section Electrostatics Calculation, R4). */
void or_apply(const or_grid* G, const double* phi, double* out) {
  double ih2 = 1.0 / (G->dx * G->dx);
#pragma omp parallel for schedule(static)
  for (int z = 0; z < G->nz; ++z)
    for (int y = 0; y < G->ny; ++y)
      for (int x = 0; x < G->nx; ++x) {
        long c = cell_index(G, x, y, z);
        double acc = 0.0;
        for (int d = 0; d < 3; ++d)
          for (int s = -1; s <= 1; s += 2) {
            long nb;
            int bt;
            double bv;
            if (face_of(G, x, y, z, d, s, &nb, &bt, &bv))
              acc += eps_face(G, c, nb) * (phi[c] - phi[nb]);
            else if (bt == 1)
              acc += 2.0 * eps_of(G, c) * phi[c];
          }
        out[c] = acc * ih2;
      }
}

void or_diag(const or_grid* G, double* dg) {
  double ih2 = 1.0 / (G->dx * G->dx);
#pragma omp parallel for schedule(static)
  for (int z = 0; z < G->nz; ++z)
    for (int y = 0; y < G->ny; ++y)
      for (int x = 0; x < G->nx; ++x) {
        long c = cell_index(G, x, y, z);
        double acc = 0.0;
        for (int d = 0; d < 3; ++d)
          for (int s = -1; s <= 1; s += 2) {
            long nb;
            int bt;
            double bv;
            if (face_of(G, x, y, z, d, s, &nb, &bt, &bv))
              acc += eps_face(G, c, nb);
            else if (bt == 1)
              acc += 2.0 * eps_of(G, c);
          }
        dg[c] = acc * ih2;
      }
}

/* Eqs. F_elec: E = -grad phi, per component the difference of the two face
 * values of phi divided by dx; face values per reading R3. */
/* E at cell (x,y,z) from face values (R3). */
static void field_at(const or_grid* G, const double* phi, int x, int y, int z, double E[3]) {
  double ih = 1.0 / G->dx;
  long c = cell_index(G, x, y, z);
  for (int d = 0; d < 3; ++d) {
    double f[2];
    for (int s = -1; s <= 1; s += 2) {
      long nb;
      int bt;
      double bv;
      if (face_of(G, x, y, z, d, s, &nb, &bt, &bv))
        f[(s + 1) / 2] = 0.5 * (phi[c] + phi[nb]);
      else
        f[(s + 1) / 2] = (bt == 1) ? bv : phi[c];
    }
    E[d] = -(f[1] - f[0]) * ih;
  }
}

void or_field(const or_grid* G, const double* phi, double* E) {
  long n = ncells(G);
#pragma omp parallel for schedule(static)
  for (int z = 0; z < G->nz; ++z)
    for (int y = 0; y < G->ny; ++y)
      for (int x = 0; x < G->nx; ++x) {
        double e[3];
        field_at(G, phi, x, y, z, e);
        for (int d = 0; d < 3; ++d) E[(long)d * n + cell_index(G, x, y, z)] = e[d];
      }
}

int or_has_dirichlet(const or_grid* G) {
  if (G->periodic_z) return 0;
  long m = (long)G->nx * G->ny;
  for (long i = 0; i < m; ++i)
    if (G->type_lo[i] == 1 || G->type_hi[i] == 1) return 1;
  return 0;
}

#ifdef _OPENMP
#include <omp.h>
#define OR_CHUNK 4096L
static double dot(const double* a, const double* b, long n) {
  long nc = (n + OR_CHUNK - 1) / OR_CHUNK;
  double* part = (double*)malloc(sizeof(double) * (size_t)nc);
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nc; ++k) {
    long e = (k + 1) * OR_CHUNK < n ? (k + 1) * OR_CHUNK : n;
    double s = 0.0;
    for (long i = k * OR_CHUNK; i < e; ++i) s += a[i] * b[i];
    part[k] = s;
  }
  double s = 0.0;
  for (long k = 0; k < nc; ++k) s += part[k];
  free(part);
  return s;
}
int or_threads(void) { return omp_get_max_threads(); }
#else
static double dot(const double* a, const double* b, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}
int or_threads(void) { return 1; }
#endif

static double mean(const double* a, long n) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i];
  return s / (double)n;
}

/* Reading R6: Jacobi-preconditioned conjugate gradients (the paper uses a
 * PETSc Krylov solver, Section Numerical Performance, warm-started from the
 * previous potential).  Textbook Hestenes-Stiefel PCG; stop when the
 * recursive residual satisfies ||r||/||b|| < rtol. */
int or_solve(const or_grid* G, const double* b_in, double* phi, double rtol, int maxit,
             int* iters, double* relres) {
  long n = ncells(G);
  int singular = !or_has_dirichlet(G);
  double* b = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * n);
  double* dg = (double*)malloc(sizeof(double) * n);
  memcpy(b, b_in, sizeof(double) * n);
  if (singular) {
    double m = mean(b, n);
    for (long i = 0; i < n; ++i) b[i] -= m;
  }
  or_diag(G, dg);
  int status = OR_OK, k = 0;
  double bnorm = sqrt(dot(b, b, n)), rel = 0.0;
  if (bnorm == 0.0) {
    memset(phi, 0, sizeof(double) * n);
    goto done;
  }
  or_apply(G, phi, q);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
  rel = sqrt(dot(r, r, n)) / bnorm;
  if (rel < rtol) goto finish;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) z[i] = r[i] / dg[i];
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) p[i] = z[i];
  double rz = dot(r, z, n);
  status = OR_NOCONV;
  for (k = 1; k <= maxit; ++k) {
    or_apply(G, p, q);
    double pq = dot(p, q, n);
    if (!(pq > 0.0)) break;                 /* breakdown: keep the current iterate */
    double alpha = rz / pq;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) phi[i] += alpha * p[i];
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) r[i] -= alpha * q[i];
    rel = sqrt(dot(r, r, n)) / bnorm;
    if (rel < rtol) {
      status = OR_OK;
      break;
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) z[i] = r[i] / dg[i];
    double rz_new = dot(r, z, n);
    double beta = rz_new / rz;
    rz = rz_new;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  if (k > maxit) k = maxit;
finish:
  if (singular) {
    double m = mean(phi, n);
    for (long i = 0; i < n; ++i) phi[i] -= m;
  }
done:
  if (iters) *iters = k;
  if (relres) *relres = rel;
  free(b); free(r); free(z); free(p); free(q); free(dg);
  return status;
}

int or_solve_potential(const or_grid* G, const double* P, double* phi, double rtol, int maxit,
                       int* iters, double* relres) {
  long n = ncells(G);
  double* b = (double*)malloc(sizeof(double) * n);
  or_rhs(G, P, b);
  int st = or_solve(G, b, phi, rtol, maxit, iters, relres);
  free(b);
  return st;
}

/* Eq. TDGL with the deterministic driving force
 *   -dF/dP_i = -(df/dP_i) + g Lap P_i + E_i      (Eqs. F_bulk, dF_grad, F_elec)
 * advanced by forward Euler (Section Time Integration):
 *   P_{n+1} = P_n + dt L (-df/dP + g Lap P + E),   E from the potential of P_n. */
int or_step(const or_grid* G, const or_params* prm, double* P, double* phi, int nsteps,
            or_info* info) {
  long n = ncells(G);
  double* b = (double*)malloc(sizeof(double) * n);
  double* h = (double*)malloc(sizeof(double) * 3 * n);
  double* lap = (double*)malloc(sizeof(double) * 3 * n);
  double* E = (double*)malloc(sizeof(double) * 3 * n);
  or_info inf;
  memset(&inf, 0, sizeof(inf));
  int status = OR_OK;
  for (int s = 0; s < nsteps; ++s) {
    int it = 0;
    double rel = 0.0;
    or_rhs(G, P, b);
    int st = or_solve(G, b, phi, prm->rtol, prm->maxit, &it, &rel);
    if (st != OR_OK) {
      status = st;
      inf.nonconverged++;
    }
    inf.last_iters = it;
    inf.total_iters += it;
    inf.last_relres = rel;
    or_field(G, phi, E);
    or_landau_force(P, n, prm->a1, prm->a11, prm->a12, h);
    for (int c = 0; c < 3; ++c) or_laplacian(G, P + (long)c * n, lap + (long)c * n);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < 3 * n; ++i)
      P[i] = P[i] + prm->dt * prm->L * (-h[i] + prm->g * lap[i] + E[i]);
    zero_air(G, P);
    inf.steps_done = s + 1;
  }
  if (info) *info = inf;
  free(b); free(h); free(lap); free(E);
  return status;
}

/* TDGL rate dP/dt = L (-df/dP + g Lap P + E(phi)) at the state P with the
 * potential phi (Eq. TDGL with Eqs. F_bulk, dF_grad/dP and F_elec). */
void or_rate(const or_grid* G, const or_params* prm, const double* P, const double* phi, double* R) {
  long n = ncells(G);
  double* h = (double*)malloc(sizeof(double) * 3 * n);
  double* lap = (double*)malloc(sizeof(double) * 3 * n);
  double* E = (double*)malloc(sizeof(double) * 3 * n);
  or_field(G, phi, E);
  or_landau_force(P, n, prm->a1, prm->a11, prm->a12, h);
  for (int c = 0; c < 3; ++c) or_laplacian(G, P + (long)c * n, lap + (long)c * n);
  for (long i = 0; i < 3 * n; ++i) R[i] = prm->L * (-h[i] + prm->g * lap[i] + E[i]);
  zero_air(G, R);
  free(h); free(lap); free(E);
}

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC 2011): ten rounds on a 4 x 32-bit counter with a
 * 2 x 32-bit key.  A round multiplies counter words 0 and 2 by the two
 * round multipliers into 64-bit products and recombines the high and low
 * halves with words 1 and 3 and the key; between rounds the key is bumped
 * by the two Weyl constants. */
static void philox4x32_10(const unsigned ctr_in[4], const unsigned key_in[2], unsigned out[4]) {
  unsigned c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  unsigned k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    unsigned long long p0 = (unsigned long long)0xD2511F53u * c[0];
    unsigned long long p2 = (unsigned long long)0xCD9E8D57u * c[2];
    unsigned hi0 = (unsigned)(p0 >> 32), lo0 = (unsigned)p0;
    unsigned hi2 = (unsigned)(p2 >> 32), lo2 = (unsigned)p2;
    unsigned n0 = hi2 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo2;
    c[2] = n2;
    c[3] = lo0;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void or_philox(unsigned long long seed, unsigned long long step, unsigned long long cell, unsigned out[4]) {
  const unsigned ctr[4] = {(unsigned)cell, (unsigned)(cell >> 32), (unsigned)step, (unsigned)(step >> 32)};
  const unsigned key[2] = {(unsigned)seed, (unsigned)(seed >> 32)};
  philox4x32_10(ctr, key, out);
}

/* Four standard normal variates for (seed, step, cell): the Box-Muller
 * transform (Box & Muller 1958) of the two pairs of Philox words, with the
 * first word of a pair mapped to (0, 1] and the second to [0, 1). */
void or_gauss4(unsigned long long seed, unsigned long long step, unsigned long long cell, double g[4]) {
  unsigned x[4];
  or_philox(seed, step, cell, x);
  const double two32 = 4294967296.0, twopi = 6.283185307179586;
  for (int j = 0; j < 2; ++j) {
    double u1 = ((double)x[2 * j] + 1.0) / two32;
    double u2 = (double)x[2 * j + 1] / two32;
    double r = sqrt(-2.0 * log(u1));
    g[2 * j] = r * cos(twopi * u2);
    g[2 * j + 1] = r * sin(twopi * u2);
  }
}

/* The thermal random force of Eq. TDGL over one step: zeta_i(r, t) dt has
 * zero mean and Gaussian variance; sigma sqrt(dt) g with g standard normal,
 * one draw per cell, component and step (components: the first three of
 * or_gauss4 at the cell's linear index). */
static void add_noise(const or_grid* G, double* P, double amp, unsigned long long seed, unsigned long long step) {
  long n = ncells(G);
  for (long c = 0; c < n; ++c) {
    double g[4];
    or_gauss4(seed, step, (unsigned long long)c, g);
    for (int i = 0; i < 3; ++i) P[(long)i * n + c] += amp * g[i];
  }
}

/* The TDGL rate at m listed cells (linear indices), out[3 * k + i] for
 * component i of cell k: the same per-cell terms as or_rate, evaluated only
 * there, so that a state of any size can be checked at samples. */
void or_rate_at(const or_grid* G, const or_params* prm, const double* P, const double* phi, const long* cells,
                int m, double* out) {
  long n = ncells(G), nxy = (long)G->nx * G->ny;
  for (int k = 0; k < m; ++k) {
    long c = cells[k];
    int z = (int)(c / nxy), y = (int)((c % nxy) / G->nx), x = (int)(c % G->nx);
    if (!is_film(G, z)) {
      out[3 * k] = out[3 * k + 1] = out[3 * k + 2] = 0.0;
      continue;
    }
    double p[3] = {P[c], P[n + c], P[2 * n + c]}, h[3], E[3];
    landau_at(p, prm->a1, prm->a11, prm->a12, h);
    field_at(G, phi, x, y, z, E);
    for (int i = 0; i < 3; ++i)
      out[3 * k + i] = prm->L * (-h[i] + prm->g * laplacian_at(G, P + (long)i * n, x, y, z) + E[i]);
  }
}

/* One potential solve for the state P, warm-started from phi, booked in inf. */
static int solve_booked(const or_grid* G, const or_params* prm, const double* P, double* phi, double* b,
                        or_info* inf) {
  int it = 0;
  double rel = 0.0;
  or_rhs(G, P, b);
  int st = or_solve(G, b, phi, prm->rtol, prm->maxit, &it, &rel);
  if (st != OR_OK) inf->nonconverged++;
  inf->last_iters = it;
  inf->total_iters += it;
  inf->last_relres = rel;
  return st;
}

/* Time integration with the options of Sections Time Integration and
 * Numerical Performance.
 *   integrator OR_EULER: P_{n+1} = P_n + dt R(P_n, phi(P_n)).
 *   integrator OR_HEUN, the paper's predictor-corrector: the predictor
 *     P^p = P^c_n + dt R(P^c_n) takes the rate at the corrected state, the
 *     rate used for the step is the mean of that rate and the rate at the
 *     predicted state, and the corrected state is P^c_{n+1} = P^c_n + dt times
 *     that mean.  Each rate has the potential of its own state.
 *   every: the long-range (electrostatic) potential is solved only on steps
 *     whose global index n0 + s is a multiple of every; the other steps, both
 *     Heun stages included, keep the last potential solved.
 *   sigma: the thermal random force of Eq. TDGL (zero mean, Gaussian): every
 *     step adds sigma sqrt(dt) g to each component of each cell, g standard
 *     normal from or_gauss4(seed, n0 + s, cell) (Euler-Maruyama; the
 *     predictor-corrector adds the same increment to both stages).
 * On return phi is the last potential solved (warm start of the next one). */
int or_step_ex(const or_grid* G, const or_params* prm, int integrator, int every, long n0, double* P,
               double* phi, int nsteps, double sigma, unsigned long long seed, or_info* info) {
  long n = ncells(G);
  double* b = (double*)malloc(sizeof(double) * n);
  double* R = (double*)malloc(sizeof(double) * 3 * n);
  double* Rp = (double*)malloc(sizeof(double) * 3 * n);
  double* Pp = (double*)malloc(sizeof(double) * 3 * n);
  or_info inf;
  memset(&inf, 0, sizeof(inf));
  int status = OR_OK;
  if (every < 1) every = 1;
  for (int s = 0; s < nsteps; ++s) {
    const int refresh = ((n0 + s) % every) == 0;
    if (refresh && solve_booked(G, prm, P, phi, b, &inf) != OR_OK) status = OR_NOCONV;
    or_rate(G, prm, P, phi, R);
    const double amp = sigma * sqrt(prm->dt);
    const unsigned long long step = (unsigned long long)(n0 + s);
    if (integrator == OR_HEUN) {
      /* the same random increment in the predictor and the corrector */
      for (long i = 0; i < 3 * n; ++i) Pp[i] = P[i] + prm->dt * R[i];
      if (sigma != 0.0) add_noise(G, Pp, amp, seed, step);
      zero_air(G, Pp);
      if (refresh && solve_booked(G, prm, Pp, phi, b, &inf) != OR_OK) status = OR_NOCONV;
      or_rate(G, prm, Pp, phi, Rp);
      for (long i = 0; i < 3 * n; ++i) P[i] = P[i] + prm->dt * (0.5 * (R[i] + Rp[i]));
    } else {
      for (long i = 0; i < 3 * n; ++i) P[i] = P[i] + prm->dt * R[i];
    }
    if (sigma != 0.0) add_noise(G, P, amp, seed, step);
    zero_air(G, P);
    inf.steps_done = s + 1;
  }
  if (info) *info = inf;
  free(b); free(R); free(Rp); free(Pp);
  return status;
}

/* Discrete free energy whose gradient is the force used in or_step:
 *   F = sum_c f(P_c) + (g/2) sum_{interior faces} |P_c - P_nb|^2 / dx^2
 *       - 1/2 sum_c P_c . (E_c + E_ext,c)
 * E is the field of P (with electrodes); E_ext the field of the electrodes
 * alone (P = 0).  -dF/dP_c then equals the driving force of Eq. TDGL. */
double or_energy(const or_grid* G, const or_params* prm, const double* P, double rtol) {
  long n = ncells(G);
  double F = or_landau_energy(P, n, prm->a1, prm->a11, prm->a12);
  double ih2 = 1.0 / (G->dx * G->dx), fg = 0.0;
  for (int z = 0; z < G->nz; ++z)
    for (int y = 0; y < G->ny; ++y)
      for (int x = 0; x < G->nx; ++x) {
        long c = cell_index(G, x, y, z);
        for (int d = 0; d < 3; ++d) {
          long nb;
          if (!wall_face(G, x, y, z, d, +1, &nb)) continue;
          for (int i = 0; i < 3; ++i) {
            double dp = P[(long)i * n + nb] - P[(long)i * n + c];
            fg += dp * dp;
          }
        }
      }
  F += 0.5 * prm->g * fg * ih2;

  double* phi = (double*)calloc(n, sizeof(double));
  double* E = (double*)malloc(sizeof(double) * 3 * n);
  double* zero = (double*)calloc(3 * n, sizeof(double));
  or_solve_potential(G, P, phi, rtol, 100000, NULL, NULL);
  or_field(G, phi, E);
  double fe = 0.0;
  for (long i = 0; i < 3 * n; ++i) fe += P[i] * E[i];
  memset(phi, 0, sizeof(double) * n);
  or_solve_potential(G, zero, phi, rtol, 100000, NULL, NULL);
  or_field(G, phi, E);
  for (long i = 0; i < 3 * n; ++i) fe += P[i] * E[i];
  F -= 0.5 * fe;
  free(phi); free(E); free(zero);
  return F;
}

/* Discrete adjoint of one forward-Euler step of or_step.
 *
 * One step maps P_n to P_{n+1} = P_n + dt L (-f'(P_n) + g Lap P_n + E(phi_n))
 * with A phi_n = -div P_n + B(V) (Eqs. TDGL, rho, Poisson; Section Time
 * Integration).  Write E(phi) = E0(phi) + E_V, where E0 is the face rule R3
 * with every electrode voltage at zero and E_V the field of the voltages
 * alone.  By R3, E0 is the transpose of the divergence, and A and Lap are
 * symmetric, so for a cotangent lambda = dJ/dP_{n+1}:
 *   dJ/dP_n = lambda + dt L (-H(P_n) lambda + g Lap lambda + E0(psi)),
 *   A psi = -div lambda,
 * with H the 3x3 Hessian of the Landau density of each cell.  The step's
 * parameter sensitivities lambda . dP_{n+1}/dtheta are added to grad
 * (a1, a11, a12, g) and, per face cell, to gv_lo / gv_hi (the voltage of
 * that face cell; nothing is added at a Neumann cell).  psi holds the warm
 * start of the adjoint solve and is updated in place. */
int or_adjoint_step(const or_grid* G, const or_params* prm, const double* P, const double* lam,
                    double* lam_out, double* psi, double* grad, double* gv_lo, double* gv_hi,
                    int* iters) {
  long n = ncells(G), nxy = (long)G->nx * G->ny;
  double ih = 1.0 / G->dx, ih2 = ih * ih, dtL = prm->dt * prm->L;
  double* zero_v = (double*)calloc(2 * nxy, sizeof(double));
  or_grid G0 = *G;                              /* same grid, electrodes at 0 V */
  G0.volt_lo = zero_v;
  G0.volt_hi = zero_v + nxy;
  double* b = (double*)malloc(sizeof(double) * n);
  double* E = (double*)malloc(sizeof(double) * 3 * n);
  double* lapl = (double*)malloc(sizeof(double) * 3 * n);
  double* lapP = (double*)malloc(sizeof(double) * 3 * n);

  or_rhs(&G0, lam, b);                          /* -div lambda */
  int st = or_solve(&G0, b, psi, prm->rtol, prm->maxit, iters, NULL);
  or_field(&G0, psi, E);                        /* E0(psi) */
  for (int c = 0; c < 3; ++c) {
    or_laplacian(G, lam + (long)c * n, lapl + (long)c * n);
    or_laplacian(G, P + (long)c * n, lapP + (long)c * n);
  }
  for (long c = 0; c < n; ++c) {
    double p[3] = {P[c], P[n + c], P[2 * n + c]};
    double l[3] = {lam[c], lam[n + c], lam[2 * n + c]};
    for (int i = 0; i < 3; ++i) {
      int j = (i + 1) % 3, k = (i + 2) % 3;
      double Hl = (2.0 * prm->a1 + 12.0 * prm->a11 * p[i] * p[i] +
                   2.0 * prm->a12 * (p[j] * p[j] + p[k] * p[k])) * l[i] +
                  4.0 * prm->a12 * p[i] * (p[j] * l[j] + p[k] * l[k]);
      long ic = (long)i * n + c;
      lam_out[ic] = l[i] + dtL * (-Hl + prm->g * lapl[ic] + E[ic]);
      /* d/dtheta of dt L (-f'_i(P) + g Lap P_i) */
      grad[0] += l[i] * dtL * -(2.0 * p[i]);
      grad[1] += l[i] * dtL * -(4.0 * p[i] * p[i] * p[i]);
      grad[2] += l[i] * dtL * -(2.0 * p[i] * (p[j] * p[j] + p[k] * p[k]));
      grad[3] += l[i] * dtL * lapP[ic];
    }
  }
  /* A face voltage V enters b of its cell as 2 eps_c V / dx^2 and the face
   * value of phi in E_z of that cell (R3, R4). */
  if (!G->periodic_z) {
    for (int y = 0; y < G->ny; ++y)
      for (int x = 0; x < G->nx; ++x) {
        long m = (long)y * G->nx + x;
        long c0 = cell_index(G, x, y, 0), c1 = cell_index(G, x, y, G->nz - 1);
        if (G->type_lo[m] == 1)
          gv_lo[m] += dtL * (-psi[c0] * 2.0 * eps_of(G, c0) * ih2 + lam[2 * n + c0] * ih);
        if (G->type_hi[m] == 1)
          gv_hi[m] += dtL * (-psi[c1] * 2.0 * eps_of(G, c1) * ih2 - lam[2 * n + c1] * ih);
      }
  }
  free(zero_v); free(b); free(E); free(lapl); free(lapP);
  return st;
}

/* Run diagnostics of a state (P, phi), each summed over all cells:
 *   out[0..2]  mean of P_x, P_y, P_z (the polarization of P-V loops);
 *   out[3]     fraction of cells with P_x > threshold (switched domains);
 *   out[4]     sum f(P)                                  (Eq. F_bulk);
 *   out[5]     (g/2) sum over interior faces |P_nb - P_c|^2 / dx^2
 *                                                        (Eq. F_grad, R1);
 *   out[6]     -1/2 sum P . E(phi), E from phi with the face voltages (R3)
 *                                                        (Eq. F_elec).
 * With the electrodes at 0 V and phi the potential of P, out[4] + out[5] +
 * out[6] is the free energy or_energy returns. */
void or_diagnostics(const or_grid* G, const or_params* prm, const double* P, const double* phi,
                    double threshold, double* out) {
  long n = ncells(G);
  for (int k = 0; k < 7; ++k) out[k] = 0.0;
  for (long c = 0; c < n; ++c) {
    out[0] += P[c];
    out[1] += P[n + c];
    out[2] += P[2 * n + c];
    if (P[c] > threshold) out[3] += 1.0;
  }
  for (int k = 0; k < 4; ++k) out[k] /= (double)n;
  out[4] = or_landau_energy(P, n, prm->a1, prm->a11, prm->a12);
  double fg = 0.0;
  for (int z = 0; z < G->nz; ++z)
    for (int y = 0; y < G->ny; ++y)
      for (int x = 0; x < G->nx; ++x) {
        long c = cell_index(G, x, y, z);
        for (int d = 0; d < 3; ++d) {
          long nb;
          if (!wall_face(G, x, y, z, d, +1, &nb)) continue;
          for (int i = 0; i < 3; ++i) {
            double dp = P[(long)i * n + nb] - P[(long)i * n + c];
            fg += dp * dp;
          }
        }
      }
  out[5] = 0.5 * prm->g * fg / (G->dx * G->dx);
  double* E = (double*)malloc(sizeof(double) * 3 * n);
  or_field(G, phi, E);
  double pe = 0.0;
  for (long i = 0; i < 3 * n; ++i) pe += P[i] * E[i];
  out[6] = -0.5 * pe;
  free(E);
}
