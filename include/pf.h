/*
 * pf.h -- C ABI of the GB300 time-domain ferroelectric phase-field step.
 *
 * The library advances the polarization field P of a ferroelectric film by
 * the time-dependent Ginzburg-Landau equation (Eq. TDGL of Ashraf &
 * Salahuddin, "A Massively Parallel Time Domain Phase Field Model for
 * Multi-domain Ferroelectric Device Simulation"), with the driving force made
 * of
 *   - the Landau bulk term (Eq. F_bulk),
 *   - the domain-wall gradient term G11 Lap P (Eqs. F_grad, dF_grad/dP),
 *   - the electric field E = -grad phi (Eqs. F_elec),
 * where phi solves the electrostatic Poisson problem div(eps grad phi) =
 * div P (Eqs. rho, Poisson) with periodic x/y and per-cell Dirichlet
 * (electrode) or Neumann (open surface) z faces (Section Electrostatics
 * Calculation).  Time stepping is explicit forward Euler (Section Time
 * Integration) or the paper's predictor-corrector.  Each Poisson solve is
 * warm-started (Section Numerical Performance): by default from a polynomial
 * extrapolation of the last potentials, with PF_FLAG_WARM_LAST from the last
 * potential as in the paper.  The paper's finite-element
 * elastic solve is not part of this library: a fixed homogeneous misfit
 * strain is assumed folded into a1, a11, a12.
 *
 * Discretisation: cell-centred unknowns on an nx*ny*nz grid of spacing dx,
 * linear index (z*ny + y)*nx + x (x fastest, the paper's natural ordering).
 * Interior face values are the mean of the two cells; at a Dirichlet face
 * phi_f = V and P_f = P_cell; at a Neumann face phi_f = phi_cell and P_f = 0;
 * P has zero normal flux at non-periodic z faces for the gradient term;
 * interior face permittivity is the harmonic mean of the two cells.
 *
 * Memory: every device buffer is owned by the caller (for example torch
 * tensors).  The library allocates no device memory and keeps only a small
 * pinned host mirror of its solver scalars.  All calls are issued on the CUDA
 * stream given to pf_create.  pf_step_async returns without waiting (when the
 * steps run as CUDA graphs, the default); the other calls that report solver
 * results (pf_step, pf_step_wait, pf_solve_potential, pf_adjoint_step,
 * pf_diagnostics, pf_true_residual) wait for their work, because the
 * statistics they return live on the device.  Calls return a pf_status and
 * never abort; the message of the last failure is available from
 * pf_last_error.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_ctx pf_ctx;

typedef enum {
  PF_OK = 0,
  PF_ERR_ARG = 1,        /* invalid argument (sizes, pointers, enum values) */
  PF_ERR_CUDA = 2,       /* a CUDA runtime call failed; see pf_last_error */
  PF_ERR_NOCONV = 3,     /* a Poisson solve hit poisson_maxit (state stays valid) */
  PF_ERR_NONFINITE = 4,  /* NaN or Inf detected in the solver scalars */
  PF_ERR_TIMEOUT = 5,    /* reserved: a bounded device wait gave up */
  PF_ERR_STATE = 6,      /* call out of order (e.g. pf_step before pf_bind) */
  PF_ERR_NOTIMPL = 7     /* entry point declared but not available */
} pf_status;

enum { PF_FP64 = 0, PF_FP32 = 1 };              /* storage and arithmetic type of fields */
enum { PF_PCG_JACOBI = 0, PF_PCG_MG = 1 };      /* Poisson preconditioner */
enum { PF_ZLO = 0, PF_ZHI = 1 };                /* z faces: z = -1/2 and z = nz - 1/2 */
enum { PF_NEUMANN = 0, PF_DIRICHLET = 1 };      /* per-(x,y) face type */
enum { PF_EULER = 0, PF_HEUN = 1 };             /* time integrator (Section Time Integration) */

typedef struct {
  int32_t nx, ny, nz;        /* grid cells (Section Grid); each >= 1 */
  double dx;                 /* grid spacing (reduced units) */
  double a1, a11, a12;       /* Landau coefficients, Eq. F_bulk */
  double g;                  /* gradient coefficient G11, Eq. dF_grad/dP */
  double L;                  /* mobility multiplying -dF/dP in Eq. TDGL */
  double dt;                 /* time step */
  int32_t precision;         /* PF_FP64 or PF_FP32 (FP32 fields; dots compensated, reduced in FP64) */
  int32_t solver;            /* PF_PCG_JACOBI or PF_PCG_MG */
  double poisson_rtol;       /* stop when ||b - A phi||_2 / ||b||_2 < rtol (recursive residual) */
  int32_t poisson_maxit;     /* iteration cap per solve (>= 1) */
  int32_t periodic_z;        /* 1: z periodic too (masks ignored; zero-mean potential) */
  int32_t has_eps;           /* 1: a cell permittivity field is bound; 0: eps = 1 */
  int32_t flags;             /* PF_FLAG_* bits (0 = defaults) */
  int32_t integrator;        /* PF_EULER (0) or PF_HEUN (the paper's predictor-corrector) */
  int32_t poisson_every;     /* solve the potential on every k-th step only (0 or 1: every step) */
  int32_t n_air;             /* top layers that are air (0 <= n_air < nz; needs periodic_z = 0) */
  int32_t extrap_order;      /* highest order of the extrapolated start (see PF_FLAG_WARM_LAST):
                                1 linear, 2 quadratic, 3 cubic; 0: automatic: cubic when
                                poisson_rtol <= 5e-7, quadratic above, linear while the thermal
                                noise is on (a start inherits the previous solves' residuals
                                times the weights' magnitudes, 3, 7 and 15, and the noise
                                roughens the potential series) */
  int32_t reserved[2];       /* must be zero */
} pf_params;

/* pf_params.integrator (Section Time Integration), with R(P) = L(-df/dP +
 * g Lap P + E) and E the field of the potential of P:
 *   PF_EULER  P_{n+1} = P_n + dt R(P_n);
 *   PF_HEUN   the predictor-corrector the paper prints as "velocity Verlet":
 *             P^p = P_n + dt R(P_n), P_{n+1} = P_n + dt (R(P_n) + R(P^p))/2;
 *             two Poisson solves per step (the second warm-started from the
 *             first), computed as P_{n+1} = (P_n + P^p + dt R(P^p))/2.
 * pf_params.n_air = m > 0 (Section Results, the open-circuit device: air on
 * top of the film): planes z >= nz - m are air.  Their P is set to zero by
 * every update (give zero initial values there), their permittivity is the
 * caller's eps field (has_eps), and the film's top surface is free for the
 * gradient term (no z+ neighbour in the Laplacian, no wall energy across it).
 * The Poisson problem spans film and air.  No adjoint step (PF_ERR_NOTIMPL).
 * pf_params.poisson_every = k > 1 (Section Numerical Performance: long-range
 * terms every 5 steps): the potential is solved only on steps whose index
 * (counted from pf_bind) is a multiple of k; the other steps, both Heun
 * stages included, use the last potential solved. */

/* pf_params.flags:
 *   PF_FLAG_NO_GRAPHS  launch every kernel from the host instead of running
 *                      each step as one CUDA graph (profilers cannot see
 *                      kernels inside graphs that contain conditional nodes);
 *   PF_FLAG_ADJOINT    reserve workspace for pf_adjoint_step (one more scalar
 *                      field, the adjoint potential, and one face array);
 *   PF_FLAG_WARM_LAST  start every Poisson solve of pf_step from the last
 *                      potential, as the paper does (Section Numerical
 *                      Performance).  Without it, forward-Euler runs (which
 *                      solve every step, or every poisson_every-th: equally
 *                      spaced in time either way) start solve k from a
 *                      polynomial extrapolation of the last potentials, up to
 *                      the order extrap_order of pf_params (cubic:
 *                      4 phi_{k-1} - 6 phi_{k-2} + 4 phi_{k-3} - phi_{k-4};
 *                      lower orders, then constant, for the first solves after
 *                      pf_bind, pf_solve_potential or a pf_set_bc that changes
 *                      an electrode layout; voltage changes keep the
 *                      history): the same stopping test, a closer start,
 *                      fewer iterations.  Costs three more fields of
 *                      workspace.  In FP32 (unless the problem is singular)
 *                      the library also keeps, in two more fields, the part
 *                      of each solution that the FP32 phi cannot hold, and
 *                      extrapolates from that compensated potential: without
 *                      it the rounding of phi alone would leave a start
 *                      residual above a 1e-7 tolerance on large films.  phi
 *                      is still the solution rounded to FP32.
 *   PF_FLAG_PLAIN_FP32 store the FP32 polarization state plainly.  Without it,
 *                      FP32 forward-Euler contexts (not created with
 *                      PF_FLAG_ADJOINT) keep the state as the compensated
 *                      pair P + P_lo: P_lo (3N more FP32 values of workspace)
 *                      holds the part of each updated value that the FP32 P
 *                      cannot hold, and every step adds its increment to the
 *                      pair exactly (TwoSum).  Plain FP32 loses the
 *                      increments that fall below half an ulp of P, which near
 *                      equilibrium is most of them: on the 256 x 256 x 64
 *                      strip film the plain state drifts to a relative error
 *                      of 4e-4 against FP64 in 5000 steps.  The driving force
 *                      is still evaluated in FP32 from P; P is what the
 *                      caller reads.  pf_bind zeroes P_lo; a caller that
 *                      overwrites P between calls should bind again. */
enum { PF_FLAG_NO_GRAPHS = 1, PF_FLAG_ADJOINT = 2, PF_FLAG_WARM_LAST = 4, PF_FLAG_PLAIN_FP32 = 8 };

typedef struct {
  int32_t steps_done;        /* steps completed by this call */
  int32_t last_iters;        /* Poisson iterations of the last solve */
  int64_t total_iters;       /* Poisson iterations summed over this call */
  double last_relres;        /* recursive ||r||/||b|| at the end of the last solve */
  int32_t nonconverged;      /* solves of this call that hit poisson_maxit */
  int32_t status;            /* pf_status of this call */
  int64_t kernel_launches;   /* kernels this call launched (including ones that
                                returned at entry because the solve had finished) */
  int64_t graph_steps;       /* steps of this call run as one CUDA graph each (a
                                device-driven Krylov loop, no host round trip);
                                the others ran host-driven (profiling on, or
                                graphs unavailable) */
  int32_t max_iters;         /* most Poisson iterations of one solve in this call */
  int32_t solves;            /* Poisson solves finished in this call */
} pf_step_info;

/* Per-kernel device-time statistics collected while profiling is on (see
 * pf_profile_enable).  Times come from CUDA events recorded on the context's
 * stream between consecutive launches; bytes are the algorithmic bytes each
 * kernel must move (reads + writes of whole fields, halos and masks not
 * counted), summed over the launches that did work. */
typedef struct {
  char name[32];             /* kernel family, e.g. "cg_p", "tdgl" */
  int64_t launches;          /* launches that did work */
  int64_t idle_launches;     /* launches that returned at entry */
  double total_ms;           /* device time of the working launches */
  double bytes;              /* algorithmic bytes of the working launches */
} pf_kernel_stat;

/* Bytes of device workspace needed for these parameters (0 on invalid
 * parameters).  The workspace holds the second polarization buffer, the
 * Krylov vectors, the multigrid hierarchy, the boundary masks and the
 * reduction scratch. */
size_t pf_workspace_bytes(const pf_params* params);

/* Validate params and create a context bound to a CUDA stream (a
 * cudaStream_t, or NULL for the legacy default stream).  Host only: no
 * kernel is launched and no device memory is allocated.  The context must be
 * used from one host thread at a time. */
pf_status pf_create(const pf_params* params, void* cuda_stream, pf_ctx** out);

/* Attach caller-owned device buffers (borrowed, never freed by the library):
 *   P         3*N elements, component-major (Px block, Py block, Pz block),
 *             each block in the linear cell order; double for PF_FP64,
 *             float for PF_FP32.  Read and updated in place by pf_step.
 *   phi       N elements of the same type: the potential.  Its contents are
 *             the initial guess of the first solve (zero is a valid start).
 *   eps       N elements of the same type (cell permittivity, > 0) when
 *             params.has_eps = 1, else ignored and may be NULL.
 *   workspace at least pf_workspace_bytes(params) bytes, 256-byte aligned.
 * All pointers must be device pointers of the current device, with P, phi
 * and eps 16-byte aligned.  Resets both z faces to Neumann at 0 V. */
pf_status pf_bind(pf_ctx* ctx, void* P, void* phi, const void* eps, void* workspace,
                  size_t workspace_bytes);

/* Set the electrical boundary of one z face (Section Electrostatics
 * Calculation): type_xy[y*nx + x] is PF_DIRICHLET (electrode held at
 * volts_xy[y*nx + x]) or PF_NEUMANN (open surface, zero normal field).
 * Host arrays of nx*ny entries, copied before the call returns.  volts_xy
 * may be NULL (0 V).  Ignored when periodic_z = 1. */
pf_status pf_set_bc(pf_ctx* ctx, int32_t face, const int8_t* type_xy, const double* volts_xy);

/* Advance nsteps steps of the chosen integrator.  A forward-Euler step n
 * solves A phi = b(P_n) from the current phi (or its extrapolation, see
 * PF_FLAG_WARM_LAST) as initial guess, then updates
 *   P <- P - dt L (df/dP - g Lap P - E),  E = -grad phi.
 * On return P = P_nsteps and phi is the last potential solved: with Euler
 * and poisson_every <= 1 the potential of P_{nsteps-1}, with Heun that of the
 * last predicted state.  pf_step is pf_step_async followed by pf_step_wait:
 * it blocks the host until the work is done, because info (iterations,
 * residuals, non-convergence) is read back from the device.  A solve that
 * hits poisson_maxit does not stop the run: the step completes with the
 * unconverged potential and the call returns PF_ERR_NOCONV with
 * info->nonconverged counting such solves.  info may be NULL. */
pf_status pf_step(pf_ctx* ctx, int32_t nsteps, pf_step_info* info);

/* Enqueue nsteps steps on the context's stream and return.  When the steps
 * run as CUDA graphs (the default: no PF_FLAG_NO_GRAPHS, profiling off) the
 * host does not wait: each step's Krylov loop is driven from the device, and
 * forward-Euler steps that all solve the potential go out as pairs inside one
 * persistent graph launch (a device-counted while loop), however many there
 * are.
 * Host-driven steps poll the convergence flag and so block while issuing.
 * Calls accumulate: their solver statistics stay on the device until
 * pf_step_wait.  Until then the other entry points of this context (except
 * pf_step, which joins the pending work) return PF_ERR_STATE.  P and phi hold
 * the state of the last enqueued step once the stream reaches that point. */
pf_status pf_step_async(pf_ctx* ctx, int32_t nsteps);

/* Wait for the work of the pf_step_async calls since the last wait, and
 * report it in info (may be NULL) as pf_step does; returns the status
 * pf_step would have returned for all those steps. */
pf_status pf_step_wait(pf_ctx* ctx, pf_step_info* info);

/* Same as pf_step but P and phi live in host memory: both are copied to the
 * device before every step and copied back after it (pinned host memory
 * makes the copies asynchronous).  This is the end-to-end entry for callers
 * that keep the state on the host.  The solver history (the extrapolation
 * ring and, in FP32, the compensated remainders of phi and P) stays in the
 * device workspace between steps. */
pf_status pf_step_host(pf_ctx* ctx, void* P_host, void* phi_host, int32_t nsteps,
                       pf_step_info* info);

/* Solve the Poisson problem for the current P only (no P update; Eqs. rho
 * and Poisson), starting from the bound phi.  Restarts the extrapolation
 * history of pf_step: its next solve starts from this potential. */
pf_status pf_solve_potential(pf_ctx* ctx, pf_step_info* info);

/* Reverse-mode (discrete adjoint) step of one forward-Euler TDGL + Poisson
 * step (Eq. TDGL, Eqs. rho and Poisson, Section Time Integration), taken at
 * the state P_n held in the bound P buffer.
 *
 * The forward step is P_{n+1} = P_n + dt L (-df/dP + g Lap P_n + E), with E
 * the field of the potential solved from P_n.  Given lam_in = dJ/dP_{n+1}
 * this writes lam_out = dJ/dP_n, obtained from one Poisson solve for the
 * adjoint potential (A psi = -div lam_in, electrodes at 0 V; same solver,
 * rtol and maxit as the forward solve, warm-started from the previous
 * adjoint step's psi, which pf_bind zeroes), and ADDS this step's
 * contribution lam_in . dP_{n+1}/dtheta to
 *   grad_params[0..3]  for theta = a1, a11, a12, g;
 *   grad_volts         (NULL to skip) for theta = each face voltage:
 *                      grad_volts[m] for volts of face PF_ZLO at m = y*nx + x,
 *                      grad_volts[nx*ny + m] for face PF_ZHI; entries of
 *                      Neumann face cells are left unchanged.
 * Summing over the steps in reverse order gives the gradient of J with
 * respect to the initial state (the last lam_out) and to the parameters.
 *
 * lam_in, lam_out: device, 3*nx*ny*nz values of the context precision,
 *   component-major like P, 16-byte aligned; lam_out must not overlap lam_in
 *   or the bound buffers.  grad_params (4 doubles) and grad_volts
 *   (2*nx*ny doubles): device, accumulated in place.
 * Needs a context created with PF_FLAG_ADJOINT (else PF_ERR_STATE).
 * Returns PF_ERR_NOCONV / PF_ERR_NONFINITE like pf_solve_potential; info
 * (may be NULL) reports the adjoint solve. */
pf_status pf_adjoint_step(pf_ctx* ctx, const void* lam_in, void* lam_out, double* grad_params,
                          double* grad_volts, pf_step_info* info);

/* Run diagnostics of the bound state (P, phi), one pass over the grid; waits
 * for the result.  out (host, 7 doubles):
 *   out[0..2]  mean P_x, P_y, P_z (polarization of P-V loops);
 *   out[3]     fraction of cells with P_x > threshold (switched domains,
 *              compared in FP64);
 *   out[4]     sum over cells of the Landau density f(P) (Eq. F_bulk);
 *   out[5]     gradient energy (g/2) sum over interior faces |P_nb - P_c|^2/dx^2
 *              (Eq. F_grad; z faces of a non-periodic film excluded);
 *   out[6]     -1/2 sum over cells P . E(phi), E = -grad phi from face values
 *              with the face voltages (Eq. F_elec).
 * Energies are sums over cells (multiply by dx^3 for a volume integral).
 * With the electrodes at 0 V and phi the potential of P (pf_solve_potential
 * first), out[4] + out[5] + out[6] is the discrete free energy that the TDGL
 * step descends.  Sums are reduced in a fixed order (reproducible). */
pf_status pf_diagnostics(pf_ctx* ctx, double threshold, double* out);

/* True residual of the stored potential: out[0] = ||b(P) - A phi||_2,
 * out[1] = ||b(P)||_2 and out[2] = ||b(P) - A phi_c||_2 (host, 3 doubles),
 * every operation in FP64 whatever the storage precision, for the bound phi
 * and the current face voltages (Eqs. rho and Poisson with the face rules
 * above; b projected to zero mean when no electrode exists).  The solver
 * stops on its recursive residual; out[0] is the residual of the potential
 * as stored (in FP32 mode, after rounding to FP32).  phi_c is the
 * compensated potential of an FP32 time series after a pf_step (phi plus the
 * remainder the FP32 phi cannot hold, see PF_FLAG_WARM_LAST): the solution
 * the Krylov loop converged.  Without one, out[2] = out[0].  P: device, 3N
 * values of the context precision, or NULL for the bound state (the
 * potential after pf_step belongs to the state before the last update, so
 * pass that state to check the last solve).  Blocks. */
pf_status pf_true_residual(pf_ctx* ctx, const void* P, double* out);

/* Turn per-kernel timing on (1) or off (0); turning it on clears the
 * counters.  While on, every launch is bracketed by CUDA events on the
 * context's stream (no extra synchronisation: the events are read at the
 * points where the host already waits). */
pf_status pf_profile_enable(pf_ctx* ctx, int32_t enable);

/* Copy up to max kernel statistics into out; returns how many families
 * exist (may exceed max), or -1 on a NULL context. */
int32_t pf_profile_read(const pf_ctx* ctx, pf_kernel_stat* out, int32_t max);

/* Size of the device array behind pf_solve_potential_noalloc. */
#define PF_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The Poisson solve of pf_solve_potential for callers that cannot allocate
 * device memory: real-time loops that must not stall on the allocator
 * (cudaMalloc and cudaFree can synchronize the whole device), and processes
 * whose device memory is reserved up front by another allocator (a fixed
 * pool, or a framework that owns every byte).  The paper has no counterpart:
 * it is a deployment variant.
 *   - No context and no workspace: every intermediate vector lives in one
 *     file-scope __device__ array of PF_NOALLOC_SCRATCH_BYTES (32 MiB) that
 *     every GPU loading the library keeps until the process exits; the call
 *     itself allocates nothing (no cudaMalloc/cudaFree, no allocating library
 *     routine).  Grids that need more scratch than the array holds (about
 *     800k cells in FP64, 1.6M in FP32) are rejected with PF_ERR_ARG.
 *   - params as for pf_create, restricted to solver = PF_PCG_JACOBI and
 *     has_eps = 0.  P (3N, input) and phi (N: initial guess in, potential out)
 *     are device (or managed) pointers of the current device, 16-byte
 *     aligned, in the precision of params; other pointers give PF_ERR_ARG.
 *     type_lo/type_hi (nx*ny int8, PF_NEUMANN or PF_DIRICHLET) and
 *     volt_lo/volt_hi (nx*ny double) are host arrays as in pf_set_bc; NULL
 *     means open face / 0 V.
 *   - Blocks until the solve is done (it polls the convergence flag and
 *     reads the solver scalars back); info as for pf_solve_potential.  So it
 *     must not be called while its stream, or the legacy stream, is being
 *     captured into a CUDA graph: it checks and returns PF_ERR_STATE.  On
 *     failure pf_last_error(NULL) holds the message.
 *   - Every call looks up the array's device address in the current device's
 *     context (cudaGetSymbolAddress, which allocates nothing).
 *   - Every call on a device shares the array: calls that overlap on the GPU
 *     (other streams, other host threads) race.  The array keeps the last
 *     call's contents; each call rewrites what it reads. */
pf_status pf_solve_potential_noalloc(const pf_params* params, void* cuda_stream, const void* P, void* phi,
                                     const int8_t* type_lo, const double* volt_lo, const int8_t* type_hi,
                                     const double* volt_hi, pf_step_info* info);

/* Thermal random force of Eq. TDGL (the paper's zeta_i(r, t): zero mean,
 * Gaussian variance).  With sigma > 0 every step adds sigma sqrt(dt) g to
 * each component of each cell's P, after the deterministic update
 * (Euler-Maruyama; the predictor-corrector adds the same increment in both
 * stages, so the corrected state carries it once).  g is standard normal:
 * components 0..2 of the Box-Muller transform of the Philox4x32-10 block
 * (Salmon et al. 2011) with counter (cell index, step index since pf_bind)
 * and key seed -- the same stream for any tiling, graph or host-driven
 * launch and any split of the steps over calls.  sigma = 0 (the default)
 * turns it off.  Contexts with noise have no adjoint step (PF_ERR_NOTIMPL). */
pf_status pf_set_noise(pf_ctx* ctx, double sigma, uint64_t seed);

/* ------------------------------------------------------------------ tiling
 * Tiling of the fine-grid plane-march kernels (Poisson right-hand side, CG
 * operator, TDGL update, diagnostics, adjoint): the hook the autotuner uses.
 * The paper has no counterpart (its code tiles by MPI subdomain). */
typedef struct {
  int32_t vx;                /* cells per thread along x: 1, or 16 bytes of cells (4 in
                                FP32, 2 in FP64; then nx must be a multiple of it).
                                A block is 16 x 16 threads: tiles of 16 vx x 16 columns */
  int32_t tz;                /* z planes per tile (z-block depth), 1 .. 64 */
  int32_t blocks_per_sm;     /* resident blocks per SM the grid is sized for
                                (0: as many as fit); tiles are handed out dynamically */
  int32_t mg_whole;          /* multigrid sweeps: 0 (default) runs the pre-smoother, the
                                prolongation sweep and the coarse levels' second post-sweep
                                of a level of >= 2^25 cells (2^23 with eps) whose z faces
                                are not periodic as two launches, the interior planes with
                                the face code compiled out and the two face slabs of 2
                                planes; in FP32 without eps the finest level's interior
                                then also fuses pre-smoother + residual + restriction, and
                                prolongation sweep + second post-sweep.  1 runs every sweep
                                as one launch over the whole level.  Results are identical
                                either way, except that the fused post-sweeps sum r.z in
                                another order (FP32 results agree within the solve
                                tolerance). */
} pf_tiling;

/* Current tiling (the default picks vx = 16 bytes when nx allows it and the
 * deepest tz that still gives about three tiles per resident block). */
pf_status pf_get_tiling(const pf_ctx* ctx, pf_tiling* out);

/* Replace the tiling; results are unchanged up to the order of the reduction
 * sums (dot products and norms are summed per tile).  Drops captured graphs. */
pf_status pf_set_tiling(pf_ctx* ctx, const pf_tiling* tiling);

/* ------------------------------------------------------------------- batch
 * Many independent films advanced together: a batch step is a CUDA graph
 * holding, per film, its whole time step (its device-driven Krylov loops
 * included) as an independent branch, so small films run concurrently and
 * fill the GPU; a multi-step call of forward-Euler films that solve every
 * step is ONE persistent graph launch (pairs of batch steps in a
 * device-counted while loop).  Before the branches one kernel applies the
 * films' electrode voltage ramps; after them one kernel records the
 * polarization-voltage loops (the switching observable of Section Results).
 * The films keep their own contexts, buffers and boundary masks; the batch
 * borrows them.  All films must use the same CUDA stream, integrator and
 * poisson_every, and be at the same step since pf_bind.  The paper runs one
 * film per job; the batch is this library's throughput mode. */
typedef struct pf_batch pf_batch;

/* Device workspace of a batch of nfilms films keeping up to max_records loop
 * records (0 on invalid arguments). */
size_t pf_batch_workspace_bytes(int32_t nfilms, int64_t max_records);

/* Create a batch over films[0 .. nfilms-1] (bound contexts, borrowed: keep
 * them alive until pf_batch_destroy).  workspace: device, 256-byte aligned,
 * pf_batch_workspace_bytes bytes, owned by the caller.  A loop record is
 * taken after every record_every-th batch step (>= 1).  No ramps at first. */
pf_status pf_batch_create(pf_ctx* const* films, int32_t nfilms, void* workspace, size_t workspace_bytes,
                          int64_t max_records, int32_t record_every, pf_batch** out);

/* Drive face PF_ZLO or PF_ZHI of film i by a triangular voltage ramp: during
 * batch step s (counted from pf_batch_create) every electrode cell of that
 * face is at V(s) = amplitude * tri(s / period), with tri the unit triangle
 * wave (tri(0) = 0, tri(1/4) = 1, tri(3/4) = -1, period 1).  period in steps
 * (> 0); period = 0 removes the ramp (the face keeps its last voltages).  One
 * ramped face per film. */
pf_status pf_batch_set_ramp(pf_batch* batch, int32_t film, int32_t face, double amplitude, double period);

/* Advance every film by nsteps steps (blocks until done).  info (may be
 * NULL) sums the films' solver statistics (last_iters, last_relres: the
 * largest over the films); the result is the worst film status
 * (PF_ERR_NONFINITE before PF_ERR_NOCONV before PF_OK). */
pf_status pf_batch_step(pf_batch* batch, int32_t nsteps, pf_step_info* info);

/* Statistics of film i over the last pf_batch_step call. */
pf_status pf_batch_film_info(const pf_batch* batch, int32_t film, pf_step_info* info);

/* Copy the loop records to host memory: out[(r * nfilms + i) * 4 + k] for
 * record r of film i, k = 0: the ramp voltage V(s) applied during the
 * recorded step s (0 without a ramp), k = 1..3: mean P_x, P_y, P_z after
 * it.  At most max_out records are copied; *nrecords receives the number
 * stored (records beyond the batch's max_records are not kept). */
pf_status pf_batch_read_loops(pf_batch* batch, double* out, int64_t max_out, int64_t* nrecords);

/* Release the batch (not the films or the workspace).  Safe on NULL. */
pf_status pf_batch_destroy(pf_batch* batch);

/* Message of the last failing call on this batch ("" if none); with batch =
 * NULL, the message of the last failing pf_batch_create. */
const char* pf_batch_last_error(const pf_batch* batch);

/* Release the context (not the bound buffers).  Safe on NULL. */
pf_status pf_destroy(pf_ctx* ctx);

/* Message of the last failing call on this context ("" if none); with
 * ctx = NULL, the message of the last failing pf_create in this process. */
const char* pf_last_error(const pf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
