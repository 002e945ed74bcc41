// Internal interface between the C ABI (pf_api.cu) and the kernel launchers.
#pragma once

#include <functional>

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pf.h"
#include "pf_common.cuh"

namespace pf {

constexpr int MAX_GRID = 4096;   // reduction partials are sized for this many blocks
constexpr int MAX_NV = 8;        // values reduced per block or tile
constexpr int MG_MAX_LEVELS = 24;
constexpr int MG_MAX_COARSE = 1024;   // cells of the coarsest multigrid level (one block)
constexpr int MG_TAIL_CELLS = 4096;   // levels at most this large run in the one-block V-cycle tail
constexpr int MG_TAIL_LEVELS = 16;
constexpr int MG_TAIL_SMEM = 192 * 1024;   // shared-memory limit of the tail's level arrays (bytes)
// A multigrid sweep over a large level whose z faces are not periodic runs as
// two launches: the interior planes [b, nz - b), compiled without the face
// code (fewer registers, more resident blocks), and the two face slabs of b
// planes (the pre-smoother's face code also covers the planes next to a face,
// hence b = 2).  Split: the pre-smoother, the prolongation sweep and the second
// post-sweep below the finest level (the finest one also reduces r.z).  The
// second launch costs about 10 us, which a level pays back from about 2^25
// cells (measured: a 2^27-cell level gains, a 2^24-cell one loses), or from
// 2^23 with a permittivity field, whose face code costs more registers.
constexpr int MG_SPLIT_B = 2;
constexpr long long MG_SPLIT_CELLS = 1LL << 25;
constexpr long long MG_SPLIT_CELLS_EPS = 1LL << 23;
inline bool mg_split_level(long long n, int nz, int periodic_z, int eps) {
  return !periodic_z && nz >= 2 * MG_SPLIT_B + 2 && n >= (eps ? MG_SPLIT_CELLS_EPS : MG_SPLIT_CELLS);
}

struct LaunchCfg {
  int grid;            // simple per-cell kernels (TX x TY blocks over tiles)
  dim3 block;
  MarchCfg march;      // plane-march kernels (MTX x MTY blocks)
  int flat_grid;       // flat vector kernels (FLAT_THREADS blocks, grid-stride)
  cudaStream_t stream;
};

// Compensated potential of an FP32 time series (see k_cg_finish_comp): hi is the
// bound phi, lo the rest of the start (the part of the last solution hi cannot
// hold plus the extrapolation increment), ring the differences of the last
// solutions.  lo == nullptr: off.
template <typename T>
struct Comp {
  T* hi;
  T* lo;
  T* ring[3];
  long long* nsolve;   // solves in the history
  int kcap;            // 1 + the highest extrapolation order
};

// Device views of one context's buffers, typed by the storage precision.
template <typename T>
struct Dev {
  T* phi;            // the Krylov iterate: the potential, or its correction when cp.lo is set
  const T* eps;      // nullptr when eps = 1
  T* invd;           // 1/diag(A), only when eps is bound
  T* r;
  T* p0;
  T* p1;
  T* q;
  T* z;              // preconditioned residual (multigrid mode)
  Bc<T> bc;
  double* part;
  Scalars* S;
  Comp<T> cp;
  unsigned short* plo;   // remainder of a compensated FP32 polarization state (3N bf16), or nullptr
};

// One multigrid level as the kernels see it.
template <typename T>
struct MgView {
  Geo g;              // nx, ny, nz, nxy, n, periodic_z of this level
  T ax, ay, az;       // 1/hx^2, 1/hy^2, 1/hz^2
  int fx, fy, fz;     // coarsening factor to the next level (1 or 2)
  const int8_t* tlo;  // z-face electrode masks of this level
  const int8_t* thi;
  T* f;               // right-hand side (level 0: the CG residual r)
  T* e;               // correction (level 0: z = M^-1 r)
  T* et;              // second buffer of the Jacobi sweeps
  const T* eps;       // cell permittivity of this level (nullptr: eps = 1)
  const T* invd;      // 1/diag of this level's operator (with eps only)
  MarchCfg mc;
  int split;          // 1: its split sweeps run as interior + face-slab launches (mg_split_level)
};

// The small levels of the V-cycle (lv[0] .. lv[nl - 1], the last one the
// coarsest) handled by one block.
template <typename T>
struct MgTail {
  MgView<T> lv[MG_TAIL_LEVELS];
  int off[MG_TAIL_LEVELS];   // shared-memory offset (elements) of level k's f, e, e_tmp
  int nl;
  int smem_elems;            // 3 x the cells of all tail levels
};

template <typename T>
void launch_rhs_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P);
template <typename T>
void launch_rhs(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, cudaGraphConditionalHandle cond,
                int use_cond);
// mg = 1: the search direction is built from z (multigrid-preconditioned
// CG) instead of r/diag, and k_cg_r leaves r.z and beta to the V-cycle.
// second = 1: the second iteration of a compensated multigrid solve (x still
// 0, not staged; needs eps = 1).
template <typename T>
void launch_cg_p(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int mg, int first = 0, int second = 0);
template <typename T>
void launch_cg_r(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int mg, cudaGraphConditionalHandle cond,
                 int use_cond);
template <typename T>
void launch_cg_finish(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int singular);
template <typename T>
void launch_sub_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d);
// Thermal random force of one TDGL launch: amp = sigma sqrt(dt) (0: off),
// the Philox key, the device step counter, and whether this launch (the
// last update of a step) advances the counter.
struct Noise {
  double amp;
  unsigned long long seed;
  long long* step;
  int advance;
};

// coef = {a1, a11, a12, g, dt*L}.  corr = 1: predictor-corrector corrector
// (P is the predicted state; Pn holds P_n on entry and P_{n+1} on exit).
template <typename T>
void launch_tdgl(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, T* Pn, const double* coef,
                 int corr, const Noise& nz);
template <typename T>
void launch_invdiag(const LaunchCfg& L, const Geo& g, const Dev<T>& d);
// Extrapolated initial guess of a time step's solve (see k_extrap; FP32 time
// series form theirs in k_cg_finish).
template <typename T>
void launch_extrap(const LaunchCfg& L, long long n, T* phi, T* const ring[3], long long* nsolve, unsigned* ticket,
                   int kcap);
// Adjoint update (pf_adjoint.cu): lam_out from lam, the adjoint potential psi
// and the state P; adds the parameter sensitivities to grad[4] and, when
// gv_lo/gv_hi are non-NULL, the face-voltage sensitivities.
template <typename T>
void launch_tdgl_adj(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* lam, T* lam_out, const T* psi,
                     const T* P, const double* coef, double* grad, double* gv_lo, double* gv_hi);

// Diagnostics (pf_diag.cu): out[0..6] = sums of P_x, P_y, P_z, [P_x > thr],
// f(P), the squared face differences of P, and P.E(phi); coef = {a1, a11, a12, thr}.
template <typename T>
void launch_diag(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, const double* coef, double* out);

// Persistent step loops (pf_kernels.cu): the count of loop bodies left, and
// the body's last kernel (counts down, sets the while condition).
void launch_loop_set(long long* left, long long n, cudaStream_t st);
void launch_loop_next(long long* left, cudaGraphConditionalHandle h, cudaStream_t st);

// True residual (pf_diag.cu): out[0] = ||b(P) - A phi||^2, out[1] = ||b(P)||^2,
// out[2] = the first for the compensated potential when d.cp.lo is set (else
// equal to out[0]), in FP64 (b projected to zero mean when singular).  out:
// device, 3 doubles.
// Blocks the host between its two passes when singular.
template <typename T>
void launch_true_residual(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, int singular, double* out);

// One film of a batch as the batch kernels see it (device table).
struct BatchFilm {
  const void* P[2];        // the film's two polarization buffers (3N each)
  void* volt;              // voltages of the ramped z face (nullptr: no ramp)
  long long n, nxy;
  double amp, period;      // V(s) = amp tri(s / period), s = batch step
  int fp32;
  int pad;
};

// Device state of a batch (in the batch workspace).
struct BatchState {
  long long step;          // batch steps completed
  long long records;       // loop records written (or dropped beyond max_records)
  long long record_every;
  long long max_records;
  unsigned ticket;
  unsigned pad;
};

constexpr int BATCH_REC_BLOCKS = 16;   // blocks per film of the loop record

void launch_batch_ramp(const BatchFilm* films, int nfilms, long long max_nxy, const BatchState* bs,
                       cudaStream_t st);
void launch_batch_record(const BatchFilm* films, int nfilms, int buf, BatchState* bs, double* part, double* hist,
                         cudaStream_t st);

// Tiling of a plane-march launch on an nx x ny x nz grid: the deepest z
// chunk that still gives about three tiles per resident block.
// Resident plane-march blocks (MTX x MTY threads) per SM for this precision.
int march_blocks_per_sm(int fp32, int eps);

inline MarchCfg march_cfg(int nx, int ny, int nz, int resident, bool even_tz, int word) {
  MarchCfg m{};
  const int v = 16 / word;
  m.vx = nx % v == 0 ? v : 1;
  const int bx = MTX * m.vx;
  m.tiles_x = (nx + bx - 1) / bx;
  m.tiles_y = (ny + MTY - 1) / MTY;
  const long long cols = (long long)m.tiles_x * m.tiles_y;
  m.tz = even_tz ? 2 : 1;
  for (int tz : {32, 16, 8, 4, 2}) {
    if (cols * ((nz + tz - 1) / tz) >= 3LL * resident) {
      m.tz = tz;
      break;
    }
  }
  m.ntiles = cols * ((nz + m.tz - 1) / m.tz);
  m.grid = (int)std::min<long long>(m.ntiles, std::min(MAX_GRID, resident));
  return m;
}

// Grid geometry and launch shapes of the fine level for these parameters
// (shared by the context-based entry points and the allocation-free solve).
inline void setup_launch(const pf_params* p, int nsm, cudaStream_t stream, Geo& g, LaunchCfg& L) {
  g = Geo{};
  g.nx = p->nx;
  g.ny = p->ny;
  g.nz = p->nz;
  g.periodic_z = p->periodic_z;
  g.zair = p->nz - p->n_air;
  g.nxy = (long long)g.nx * g.ny;
  g.n = g.nxy * g.nz;
  g.ih = 1.0 / p->dx;
  g.ih2 = g.ih * g.ih;
  g.tiles_x = (g.nx + TX - 1) / TX;
  g.tiles_y = (g.ny + TY - 1) / TY;
  const long long cols = (long long)g.tiles_x * g.tiles_y;
  g.tz = 1;
  for (int tz : {16, 8, 4, 2}) {
    if (cols * ((g.nz + tz - 1) / tz) >= 4LL * nsm) {
      g.tz = tz;
      break;
    }
  }
  g.tiles_z = (g.nz + g.tz - 1) / g.tz;
  g.ntiles = cols * g.tiles_z;
  L = LaunchCfg{};
  const int fp32 = p->precision == PF_FP32;
  const int resident = nsm * march_blocks_per_sm(fp32, p->has_eps);
  L.march = march_cfg(g.nx, g.ny, g.nz, resident, false, fp32 ? 4 : 8);
  const long long nvec = (g.n + 3) / 4;
  L.flat_grid = (int)std::max<long long>(
      1, std::min<long long>((nvec + FLAT_THREADS - 1) / FLAT_THREADS, std::min(MAX_GRID, 4 * nsm)));
  L.block = dim3(TX, TY, 1);
  L.grid = (int)std::min<long long>(g.ntiles, std::min(MAX_GRID, 8 * nsm));
  L.stream = stream;
}

// Record the message returned by pf_last_error(NULL) (fixed buffer, no allocation).
void set_global_error(const char* what, const char* detail = nullptr);


// Multigrid V-cycle pieces (pf_mg.cu).
template <typename T>
int launch_mg_pre(const LaunchCfg& L, const MgView<T>& lv, Scalars* S);
template <typename T>
int launch_mg_rr(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S);
// Pre-smoother and residual of a split FP32 level as one fused pass over its
// interior planes (plus the face slabs' own kernels); returns the launches, 0
// when the level does not qualify (then nothing was launched).
// mark(i) is called after the i-th of its launches (0 .. 2; the profiler's marks).
template <typename T>
int launch_mg_prr(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S,
                  const std::function<void(int)>& mark);
// Whether the finest level's post-sweeps run fused (launch_mg_pp); then the
// V-cycle keeps the pre-smoothed correction out of z (in z_tmp) and uses ep
// (the CG's q, dead between the residual update and the next search
// direction) for e'.
template <typename T>
bool mg_fused_post(const MgView<T>& lv);
// Prolongation sweep + second post-sweep of the finest level, fused on its
// interior (lv.e: the pre-smoothed correction, ep: e', z: the result; r.z and
// beta as k_mg_post2); returns the launches, 0 when not eligible.
template <typename T>
int launch_mg_pp(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, T* ep, T* z, double* part,
                 Scalars* S, const std::function<void(int)>& mark);
template <typename T>
void launch_mg_coarse(const LaunchCfg& L, const MgView<T>& cv, int singular, Scalars* S);
template <typename T>
void launch_mg_tail(const LaunchCfg& L, const MgTail<T>& t, int singular, Scalars* S);
template <typename T>
int launch_mg_post1(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S);
template <typename T>
int launch_mg_post2(const LaunchCfg& L, const MgView<T>& lv, int last, double* part, Scalars* S);
template <typename T>
int mg_blocks_per_sm();
// Permittivity of a coarse level (the mean of the fine children, into ceps)
// and 1/diag of its operator (into cinvd).
template <typename T>
void launch_mg_eps_level(const LaunchCfg& L, const MgView<T>& fine, const MgView<T>& coarse, T* ceps, T* cinvd);

}  // namespace pf
