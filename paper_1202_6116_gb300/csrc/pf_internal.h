// Internal interface between the C ABI (pf_api.cu) and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pf_common.cuh"

namespace pf {

constexpr int MAX_GRID = 4096;   // reduction partials are sized for this many blocks
constexpr int MAX_NV = 4;        // values reduced per block

struct LaunchCfg {
  int grid;
  dim3 block;
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
  Bc<T> bc;
  InvDiagTable<T> tab;
  double* part;
  Scalars* S;
};

template <typename T>
void launch_rhs_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P);
template <typename T>
void launch_rhs(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, cudaGraphConditionalHandle cond,
                int use_cond);
template <typename T>
void launch_cg_p(const LaunchCfg& L, const Geo& g, const Dev<T>& d);
template <typename T>
void launch_cg_r(const LaunchCfg& L, const Geo& g, const Dev<T>& d, cudaGraphConditionalHandle cond,
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

}  // namespace pf
