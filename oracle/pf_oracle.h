/*
 * Plain FP64 CPU oracle of the time-domain ferroelectric phase-field step
 * (Ashraf & Salahuddin, "A Massively Parallel Time Domain Phase Field Model
 * for Multi-domain Ferroelectric Device Simulation").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or helper with the CUDA library and never
 * calls into it.
 *
 * Discretisation (the paper fixes only the continuum equations, see the
 * "readings" below):
 *   - cell-centred unknowns on an nx*ny*nz grid of spacing dx, index
 *     (z*ny + y)*nx + x (x varies fastest, then y, then z: the natural
 *     ordering of Section "Assembly");
 *   - x and y are periodic; z is periodic when periodic_z != 0, otherwise the
 *     two z faces carry a per-(x,y) electrical boundary mask:
 *     type 1 = Dirichlet (electrode at the given voltage), 0 = Neumann
 *     (open surface, zero normal field)  -- Section "Electrostatics
 *     Calculation";
 *   - polarization P is stored component-major: P[c*N + idx], c = x,y,z.
 *
 * Readings of the paper used here (each restated where it is applied):
 *   R1 gradient energy = (g/2) sum |grad P_i|^2, so -dF/dP_i = +g Lap P_i
 *      (the printed Eq. for F_grad is garbled; Eq. dF_grad/dP fixes G11 Lap);
 *      P has zero normal flux at non-periodic z faces.
 *   R2 Poisson: div(eps grad phi) = div P taken literally (Eqs. rho, Poisson).
 *   R3 face values: interior faces take the mean of the two cells; at a
 *      Dirichlet face phi_f = V and P_f = P_cell; at a Neumann face
 *      phi_f = phi_cell and P_f = 0.  E = -grad phi from face values.
 *   R4 Dirichlet ghost 2V - phi_c; interior face eps = harmonic mean; a
 *      Dirichlet face uses the cell's eps.
 *   R5 step order: solve phi from P_n (warm start from the previous phi),
 *      then the explicit forward-Euler update (Section "Time Integration").
 *   R6 Krylov solve = Jacobi-preconditioned CG on the SPD form
 *      A phi = b, A = -div eps grad, b = -div P + Dirichlet terms, stopped
 *      on the recursive residual ||r||/||b|| < rtol; ||b|| = 0 gives phi = 0.
 *      With no Dirichlet face anywhere A is singular: b is projected to zero
 *      mean and the returned phi has zero mean.
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;
  double dx;
  int periodic_z;                 /* 1: z periodic, masks ignored */
  const signed char* type_lo;     /* nx*ny, face z = -1/2; 1 Dirichlet, 0 Neumann */
  const double* volt_lo;          /* nx*ny volts (used where type = 1) */
  const signed char* type_hi;     /* nx*ny, face z = nz - 1/2 */
  const double* volt_hi;
  const double* eps;              /* N cell permittivities, or NULL for eps = 1 */
  int n_air;                      /* top layers z >= nz - n_air are air: P = 0 there, and the
                                     film/air faces carry no gradient (wall) energy */
} or_grid;

typedef struct {
  double a1, a11, a12;            /* Landau coefficients, Eq. F_bulk */
  double g;                       /* gradient coefficient G11, Eq. dF_grad/dP */
  double L;                       /* mobility (1 in the paper's TDGL) */
  double dt;                      /* forward-Euler step */
  double rtol;                    /* CG relative residual target */
  int maxit;                      /* CG iteration cap per solve */
} or_params;

typedef struct {
  int steps_done;
  int last_iters;                 /* CG iterations of the last solve */
  long total_iters;               /* summed over the steps */
  double last_relres;             /* recursive ||r||/||b|| of the last solve */
  int nonconverged;               /* solves that hit maxit */
} or_info;

enum { OR_OK = 0, OR_NOCONV = 3 };

/* Landau free energy summed over cells and its derivative (Eq. F_bulk). */
double or_landau_energy(const double* P, long n, double a1, double a11, double a12);
void   or_landau_force(const double* P, long n, double a1, double a11, double a12, double* out);

/* 7-point Laplacian of one scalar field with zero flux at non-periodic z faces. */
void or_laplacian(const or_grid* G, const double* f, double* out);

/* b = -div P + Dirichlet terms (the right-hand side of A phi = b). */
void or_rhs(const or_grid* G, const double* P, double* b);

/* A phi = -div(eps grad phi) with homogeneous boundary data (no V terms). */
void or_apply(const or_grid* G, const double* phi, double* out);

/* Diagonal of A. */
void or_diag(const or_grid* G, double* d);

/* E = -grad phi from face values (R3); out is 3N, component-major. */
void or_field(const or_grid* G, const double* phi, double* E);

/* 1 if the grid has a Dirichlet face somewhere (A nonsingular). */
int or_has_dirichlet(const or_grid* G);

/* Jacobi-PCG solve of A phi = b from the initial guess in phi (R6). */
int or_solve(const or_grid* G, const double* b, double* phi, double rtol, int maxit,
             int* iters, double* relres);

/* Potential of the current P: phi <- solve(A phi = rhs(P)). */
int or_solve_potential(const or_grid* G, const double* P, double* phi, double rtol, int maxit,
                       int* iters, double* relres);

/* nsteps forward-Euler TDGL steps (Eq. TDGL, R5); P and phi updated in place.
 * On return phi is the potential used by the last update. */
int or_step(const or_grid* G, const or_params* prm, double* P, double* phi, int nsteps,
            or_info* info);

/* Integrators of Section Time Integration (or_step_ex). */
enum { OR_EULER = 0, OR_HEUN = 1 };

/* TDGL rate L(-df/dP + g Lap P + E(phi)) at the state P (3N) and potential phi. */
void or_rate(const or_grid* G, const or_params* prm, const double* P, const double* phi, double* R);

/* The rate of or_rate at m listed cells (linear indices): out[3k + i] is
 * component i at cells[k].  For checks of large states at sampled cells. */
void or_rate_at(const or_grid* G, const or_params* prm, const double* P, const double* phi, const long* cells,
                int m, double* out);

/* nsteps steps of forward Euler (OR_EULER) or of the paper's predictor-corrector
 * (OR_HEUN: P^p = P^c + dt R(P^c); P^c <- P^c + dt (R(P^c) + R(P^p))/2, each
 * rate with the potential of its own state).  The potential is solved only on
 * steps whose global index n0 + s is a multiple of every (>= 1); other steps
 * keep the last potential (Section Numerical Performance: long-range terms
 * every 5 steps).  phi: warm start in, last solved potential out.  sigma > 0
 * adds the thermal random force of Eq. TDGL: sigma sqrt(dt) times standard
 * normal draws or_gauss4(seed, n0 + s, cell) per step (the same draw in both
 * predictor-corrector stages). */
int or_step_ex(const or_grid* G, const or_params* prm, int integrator, int every, long n0, double* P,
               double* phi, int nsteps, double sigma, unsigned long long seed, or_info* info);

/* Philox4x32-10 output for counter (cell, step) and key seed, and four
 * standard normal variates from it by Box-Muller (the thermal noise of
 * or_step_ex: components 0..2 of cell c at step n are or_gauss4(seed, n, c)). */
void or_philox(unsigned long long seed, unsigned long long step, unsigned long long cell, unsigned out[4]);
void or_gauss4(unsigned long long seed, unsigned long long step, unsigned long long cell, double g[4]);

/* Total free energy: sum f(P) + (g/2) sum_faces |dP|^2/dx^2 - 1/2 sum P.(E + E_ext),
 * with phi solved to rtol; E_ext is the field of the electrodes with P = 0. */
double or_energy(const or_grid* G, const or_params* prm, const double* P, double rtol);

/* Discrete adjoint of one or_step step at the state P (= P_n) of a grid
 * without air layers (n_air = 0): from
 * lam = dJ/dP_{n+1} computes lam_out = dJ/dP_n, and adds this step's
 * sensitivities to grad[4] (a1, a11, a12, g) and to the per-face-cell
 * voltage sensitivities gv_lo, gv_hi (nx*ny each).  psi is the warm start of
 * the adjoint Poisson solve (in/out).  Returns the solve's status. */
int or_adjoint_step(const or_grid* G, const or_params* prm, const double* P, const double* lam,
                    double* lam_out, double* psi, double* grad, double* gv_lo, double* gv_hi,
                    int* iters);

/* Diagnostics of (P, phi): out[0..2] mean P, out[3] fraction of cells with
 * P_x > threshold, out[4] sum f(P), out[5] gradient energy, out[6]
 * -1/2 sum P.E(phi).  out has 7 entries. */
void or_diagnostics(const or_grid* G, const or_params* prm, const double* P, const double* phi,
                    double threshold, double* out);

/* Threads the oracle's loops run on: 1 for the serial build, the OpenMP
 * thread count for the OpenMP build. */
int or_threads(void);

#ifdef __cplusplus
}
#endif
#endif
