// Kernels of the TDGL + Poisson step (sm_103a).
//
//   (the right-hand side and TDGL kernels live in pf_step.cu, the CG
//   iteration kernels in pf_cg.cu, the multigrid V-cycle in pf_mg.cu)
//   k_cg_finish  last deferred x update / zero solution, mean of x
//   k_sub_mean   x -= mean(x)                           (singular problems)
//   k_invdiag    1/diag(A) when a permittivity field is bound
//   k_extrap     initial guess of a time step's Poisson solve extrapolated
//                from the last three solutions
//
// All reductions use the last-block pattern of pf_common.cuh: deterministic,
// and no block ever waits on another.  The CG scalars (alpha, beta, the
// convergence flag) never leave the device; kernels of a finished solve
// return at entry.
#include "pf_common.cuh"
#include "pf_internal.h"

namespace pf {

// ----------------------------------------------------------- stencil helpers

__device__ __forceinline__ long long zm_index(const Geo& g, long long c, int z) {
  if (z > 0) return c - g.nxy;
  if (g.periodic_z) return c + (long long)(g.nz - 1) * g.nxy;
  return -1;
}

__device__ __forceinline__ long long zp_index(const Geo& g, long long c, int z) {
  if (z < g.nz - 1) return c + g.nxy;
  if (g.periodic_z) return c - (long long)(g.nz - 1) * g.nxy;
  return -1;
}

template <typename T>
__device__ __forceinline__ T hmean(T a, T b) {
  return T(2) * a * b / (a + b);
}

struct Nbr {
  long long c, xm, xp, ym, yp, zm, zp;   // zm/zp = -1 at a boundary face
  long long xy, xym, xyp, xmy, xpy;      // face-mask indices of the cell and its x/y neighbours
};

__device__ __forceinline__ Nbr neighbours(const Geo& g, int x, int y, int z) {
  Nbr n;
  const int xm = (x == 0) ? g.nx - 1 : x - 1, xp = (x == g.nx - 1) ? 0 : x + 1;
  const int ym = (y == 0) ? g.ny - 1 : y - 1, yp = (y == g.ny - 1) ? 0 : y + 1;
  n.xy = (long long)y * g.nx + x;
  n.xmy = (long long)y * g.nx + xm;
  n.xpy = (long long)y * g.nx + xp;
  n.xym = (long long)ym * g.nx + x;
  n.xyp = (long long)yp * g.nx + x;
  const long long zo = (long long)z * g.nxy;
  n.c = zo + n.xy;
  n.xm = zo + n.xmy;
  n.xp = zo + n.xpy;
  n.ym = zo + n.xym;
  n.yp = zo + n.xyp;
  n.zm = zm_index(g, n.c, z);
  n.zp = zp_index(g, n.c, z);
  return n;
}

// ------------------------------------------------------------------ kernels

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_cg_finish(Geo g, T* __restrict__ x, const T* __restrict__ p0,
                                                        const T* __restrict__ p1, double* part, Scalars* S,
                                                        int singular) {
  const int zero = S->zero_x, pend = S->pending;
  const T alpha = T(S->alpha);
  const T* __restrict__ p = S->pbuf ? p1 : p0;
  Acc<T> ax;
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    TileCoord tc = tile_coord(g, t);
    if (!tc.active) continue;
    for (int z = tc.z0; z < tc.z1; ++z) {
      const long long c = (long long)z * g.nxy + (long long)tc.y * g.nx + tc.x;
      if (zero) {
        x[c] = T(0);
      } else if (pend) {
        const T xv = x[c] + alpha * p[c];
        x[c] = xv;
        ax.add(xv, T(1));
      } else {
        ax.add(x[c], T(1));
      }
    }
    ax.flush();
  }
  double v[1] = {ax.value()};
  if (publish_partials<1>(v, part, &S->ticket)) {
    double out[1];
    gather_partials<1>(part, gridDim.x, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      S->mean_x = singular ? out[0] / (double)g.n : 0.0;
      S->pending = 0;
      S->total_iters += S->iter;
      S->last_iters = S->iter;
      if (S->status != 0) S->nonconv += 1;
      S->ticket = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_sub_mean(Geo g, T* __restrict__ x, const Scalars* S) {
  const T m = T(S->mean_x);
  for (long long i = blockIdx.x * (long long)NTHREADS + threadIdx.x + threadIdx.y * blockDim.x; i < g.n;
       i += (long long)gridDim.x * NTHREADS)
    x[i] -= m;
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_invdiag(Geo g, Bc<T> bc, const T* __restrict__ eps,
                                                      T* __restrict__ invd) {
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    TileCoord tc = tile_coord(g, t);
    if (!tc.active) continue;
    for (int z = tc.z0; z < tc.z1; ++z) {
      Nbr n = neighbours(g, tc.x, tc.y, z);
      const T ec = eps[n.c];
      T acc = T(0);
      acc += hmean(ec, eps[n.xm]);
      acc += hmean(ec, eps[n.xp]);
      acc += hmean(ec, eps[n.ym]);
      acc += hmean(ec, eps[n.yp]);
      if (n.zm >= 0) acc += hmean(ec, eps[n.zm]);
      else if (bc.tlo[n.xy]) acc += T(2) * ec;
      if (n.zp >= 0) acc += hmean(ec, eps[n.zp]);
      else if (bc.thi[n.xy]) acc += T(2) * ec;
      invd[n.c] = T(1) / (acc * T(g.ih2));
    }
  }
}

// Initial guess of solve number k of a time series (k = *nsolve): the
// quadratic extrapolation 3 (phi_1 - phi_2) + phi_3 of the last three
// solutions (phi_1 = phi, the last; phi_2 = h1; phi_3 = h2), linear 2 phi_1 -
// phi_2 for the third solve, the last solution for the second and the given
// phi for the first.  The history shifts (h2 <- h1, h1 <- phi) and the last
// block to finish advances the count (every block reads it first).
// Streams phi, h1, h2 once: read 3 words, write 3 words per cell.
template <typename T>
__device__ __forceinline__ T extrap_guess(long long k, T f, T a, T b) {
  if (k <= 1) return f;
  if (k == 2) return f + (f - a);
  return T(3) * (f - a) + b;
}

template <typename T>
__global__ void __launch_bounds__(FLAT_THREADS) k_extrap(long long n, T* __restrict__ phi, T* __restrict__ h1,
                                                        T* __restrict__ h2, long long* nsolve, unsigned* ticket) {
  using V = typename Vec16<T>::type;
  constexpr int NV = 16 / sizeof(T);
  __shared__ bool last;
  const long long k = *nsolve;
  const long long stride = (long long)gridDim.x * FLAT_THREADS;
  const long long nvec = n / NV;
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < nvec; i += stride) {
    V fv = reinterpret_cast<const V*>(phi)[i];
    const V av = reinterpret_cast<const V*>(h1)[i];
    const V bv = reinterpret_cast<const V*>(h2)[i];
    V gv;
    const T* f = reinterpret_cast<const T*>(&fv);
    const T* a = reinterpret_cast<const T*>(&av);
    const T* b = reinterpret_cast<const T*>(&bv);
    T* gs = reinterpret_cast<T*>(&gv);
#pragma unroll
    for (int j = 0; j < NV; ++j) gs[j] = extrap_guess(k, f[j], a[j], b[j]);
    reinterpret_cast<V*>(h2)[i] = av;
    reinterpret_cast<V*>(h1)[i] = fv;
    reinterpret_cast<V*>(phi)[i] = gv;
  }
  for (long long i = nvec * NV + blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += stride) {
    const T f = phi[i], a = h1[i], b = h2[i];
    h2[i] = a;
    h1[i] = f;
    phi[i] = extrap_guess(k, f, a, b);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    *ticket = 0u;
    *nsolve = k + 1;
    __threadfence();
  }
}

// ---------------------------------------------------------------- launchers

template <typename T>
void launch_cg_finish(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int singular) {
  k_cg_finish<T><<<L.grid, L.block, 0, L.stream>>>(g, d.phi, d.p0, d.p1, d.part, d.S, singular);
}

template <typename T>
void launch_sub_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d) {
  k_sub_mean<T><<<L.grid, L.block, 0, L.stream>>>(g, d.phi, d.S);
}

template <typename T>
void launch_invdiag(const LaunchCfg& L, const Geo& g, const Dev<T>& d) {
  k_invdiag<T><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, d.eps, d.invd);
}

template <typename T>
void launch_extrap(const LaunchCfg& L, long long n, T* phi, T* h1, T* h2, long long* nsolve, unsigned* ticket) {
  k_extrap<T><<<L.flat_grid, FLAT_THREADS, 0, L.stream>>>(n, phi, h1, h2, nsolve, ticket);
}

#define PF_INSTANTIATE(T)                                                                                   \
  template void launch_extrap<T>(const LaunchCfg&, long long, T*, T*, T*, long long*, unsigned*);          \
  template void launch_cg_finish<T>(const LaunchCfg&, const Geo&, const Dev<T>&, int);                      \
  template void launch_sub_mean<T>(const LaunchCfg&, const Geo&, const Dev<T>&);                            \
  template void launch_invdiag<T>(const LaunchCfg&, const Geo&, const Dev<T>&);

PF_INSTANTIATE(float)
PF_INSTANTIATE(double)

}  // namespace pf
