// Internal interface between the C ABI (pf_api.cu) and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pf_common.cuh"

namespace pf {

constexpr int MAX_GRID = 4096;   // reduction partials are sized for this many blocks
constexpr int MAX_NV = 4;        // values reduced per block
constexpr int MG_MAX_LEVELS = 24;
constexpr int MG_MAX_COARSE = 1024;   // cells of the coarsest multigrid level (one block)

struct LaunchCfg {
  int grid;            // simple per-cell kernels (TX x TY blocks over tiles)
  dim3 block;
  MarchCfg march;      // plane-march kernels (MTX x MTY blocks)
  int flat_grid;       // flat vector kernels (FLAT_THREADS blocks, grid-stride)
  cudaStream_t stream;
};

// Device views of one context's buffers, typed by the storage precision.
template <typename T>
struct Dev {
  T* phi;
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
  MarchCfg mc;
};

template <typename T>
void launch_rhs_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P);
template <typename T>
void launch_rhs(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, cudaGraphConditionalHandle cond,
                int use_cond);
// mg = 1: the search direction is built from z (multigrid-preconditioned
// CG) instead of r/diag, and k_cg_r leaves r.z and beta to the V-cycle.
template <typename T>
void launch_cg_p(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int mg);
template <typename T>
void launch_cg_r(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int mg, cudaGraphConditionalHandle cond,
                 int use_cond);
template <typename T>
void launch_cg_finish(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int singular);
template <typename T>
void launch_sub_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d);
// coef = {a1, a11, a12, g, dt*L}
template <typename T>
void launch_tdgl(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, T* Pn, const double* coef);
template <typename T>
void launch_invdiag(const LaunchCfg& L, const Geo& g, const Dev<T>& d);

// Resident 512-thread plane-march blocks per SM for this precision.
int march_blocks_per_sm(int fp32, int eps);

// Multigrid V-cycle pieces (pf_mg.cu).
template <typename T>
void launch_mg_pre(const LaunchCfg& L, const MgView<T>& lv, Scalars* S);
template <typename T>
void launch_mg_rr(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S);
template <typename T>
void launch_mg_coarse(const LaunchCfg& L, const MgView<T>& cv, int singular, Scalars* S);
template <typename T>
void launch_mg_post1(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S);
template <typename T>
void launch_mg_post2(const LaunchCfg& L, const MgView<T>& lv, int last, double* part, Scalars* S);
template <typename T>
int mg_blocks_per_sm();

}  // namespace pf
