// Kernels of the TDGL + Poisson step (sm_103a).
//
//   (the right-hand side and TDGL kernels live in pf_step.cu, the CG
//   iteration kernels in pf_cg.cu, the multigrid V-cycle in pf_mg.cu)
//   k_cg_finish  last deferred x update / zero solution, mean of x (or the
//                correction folded into a compensated potential)
//   k_sub_mean   x -= mean(x)                           (singular problems)
//   k_invdiag    1/diag(A) when a permittivity field is bound
//   k_extrap     initial guess of a time step's Poisson solve extrapolated
//                from the last four solutions
//   k_extrap_comp  the same for FP32 time series, on a compensated potential
//                (FP32 pair hi + lo) and the differences of past solutions
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

// (s, e) with s = fl(a + b) and s + e = a + b exactly (Knuth's TwoSum; the
// _rn intrinsics keep the compiler from contracting or reordering it).
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

// COMP (FP32 time series): x is the correction to the compensated start
// hi + lo.  The solution becomes hi + lo + x (TwoSum, so lo keeps what hi
// cannot hold), and the ring slot of this solve (holding the extrapolation
// increment c) gains x, giving the difference D_k = phi_k - phi_{k-1}.
// Per cell: read x, p, hi, lo, the slot; write hi, lo, the slot.
template <typename T, bool COMP>
__global__ void __launch_bounds__(NTHREADS) k_cg_finish(Geo g, T* __restrict__ x, const T* __restrict__ p0,
                                                        const T* __restrict__ p1, double* part, Scalars* S,
                                                        int singular, Comp<T> cp) {
  const int zero = S->zero_x, pend = S->pending;
  const T alpha = T(S->alpha);
  const T* __restrict__ p = S->pbuf ? p1 : p0;
  T* __restrict__ slot = nullptr;
  if constexpr (COMP) slot = cp.ring[(*cp.nsolve + 2) % 3];   // solve k = nsolve - 1
  Acc<T> ax;
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    TileCoord tc = tile_coord(g, t);
    if (!tc.active) continue;
    for (int z = tc.z0; z < tc.z1; ++z) {
      const long long c = (long long)z * g.nxy + (long long)tc.y * g.nx + tc.x;
      if constexpr (COMP) {
        const T hi = cp.hi[c], lo = cp.lo[c], inc = slot[c];
        if (zero) {                     // phi_k = 0
          cp.hi[c] = T(0);
          cp.lo[c] = T(0);
          slot[c] = (inc - lo) - hi;
        } else {
          const T dx = pend ? x[c] + alpha * p[c] : x[c];
          const float2 sl = two_sum(hi, lo + dx);
          cp.hi[c] = sl.x;
          cp.lo[c] = sl.y;
          slot[c] = inc + dx;
        }
        continue;
      }
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
      if (S->iter == 0) S->zero_solves += 1;
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

// Initial guess of solve number k of a time series (k = *nsolve): the cubic
// extrapolation 4 phi_1 - 6 phi_2 + 4 phi_3 - phi_4 of the last four
// solutions (phi_1 = phi, the last one; the three before it sit in a ring of
// history fields, phi_j of solve number m in slot m mod 3).  Solves 1 to 3
// take the orders their history allows: the given phi, the last solution,
// then the linear and quadratic extrapolations.  phi_1 goes into the slot of
// phi_4 once that has been read, so the ring never moves.  The last block to
// finish advances the count (every block reads it first).
// Streams phi and the ring once: read 4 words, write 2 words per cell.
// The guess is formed from the differences of consecutive solutions (exact
// in floating point when they are close) plus one final rounding.
template <typename T>
__device__ __forceinline__ T extrap_guess(long long k, T f1, T f2, T f3, T f4) {
  if (k <= 1) return f1;
  const T d1 = f1 - f2;
  if (k == 2) return f1 + d1;
  const T d2 = f2 - f3;
  if (k == 3) return f1 + (T(2) * d1 - d2);
  const T d3 = f3 - f4;
  return f1 + (T(3) * (d1 - d2) + d3);
}

template <typename T>
__global__ void __launch_bounds__(FLAT_THREADS) k_extrap(long long n, T* __restrict__ phi, T* __restrict__ s0,
                                                        T* __restrict__ s1, T* __restrict__ s2,
                                                        long long* nsolve, unsigned* ticket) {
  using V = typename Vec16<T>::type;
  constexpr int NV = 16 / sizeof(T);
  __shared__ bool last;
  const long long k = *nsolve;
  T* const ring[3] = {s0, s1, s2};
  // phi_2, phi_3 and phi_4 (= the slot phi_1 goes to) of solve k; only the
  // ones solve k reads are ever dereferenced
  T* const h2 = ring[(k + 1) % 3];
  T* const h3 = ring[k % 3];
  T* const h4 = ring[(k + 2) % 3];
  const long long stride = (long long)gridDim.x * FLAT_THREADS;
  const long long nvec = n / NV;
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < nvec; i += stride) {
    V v1 = reinterpret_cast<const V*>(phi)[i], v2{}, v3{}, v4{};
    if (k >= 2) v2 = reinterpret_cast<const V*>(h2)[i];
    if (k >= 3) v3 = reinterpret_cast<const V*>(h3)[i];
    if (k >= 4) v4 = reinterpret_cast<const V*>(h4)[i];
    V gv;
    const T* f1 = reinterpret_cast<const T*>(&v1);
    const T* f2 = reinterpret_cast<const T*>(&v2);
    const T* f3 = reinterpret_cast<const T*>(&v3);
    const T* f4 = reinterpret_cast<const T*>(&v4);
    T* gs = reinterpret_cast<T*>(&gv);
#pragma unroll
    for (int j = 0; j < NV; ++j) gs[j] = extrap_guess(k, f1[j], f2[j], f3[j], f4[j]);
    if (k >= 1) reinterpret_cast<V*>(h4)[i] = v1;
    reinterpret_cast<V*>(phi)[i] = gv;
  }
  for (long long i = nvec * NV + blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += stride) {
    const T f1 = phi[i], f2 = k >= 2 ? h2[i] : T(0), f3 = k >= 3 ? h3[i] : T(0), f4 = k >= 4 ? h4[i] : T(0);
    if (k >= 1) h4[i] = f1;
    phi[i] = extrap_guess(k, f1, f2, f3, f4);
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

// Compensated form for FP32 time series (non-singular problems).  Rounding
// the potential to FP32 leaves a residual of order u |A| |phi|, well above a
// 1e-7 tolerance on large films, and the extrapolation above would add its
// weights' worth of it to every start.  Here the last solution is the pair
// hi + lo (lo: the part hi cannot hold), and the ring holds the differences
// D_m = phi_m - phi_{m-1} of consecutive solutions (slot m mod 3), small
// beside phi and so nearly exact in FP32.  The start of solve k is
// phi_{k-1} + c with the increment
//   c = 0 (k <= 1), D1 (k = 2), 2 D1 - D2 (k = 3), 3 (D1 - D2) + D3 (k >= 4)
// (D_j = D_{k-j}; the same linear, quadratic and cubic extrapolations as
// above), added to the pair by TwoSum.  c goes into the slot of D_{k-3} once
// that has been read; k_cg_finish adds the solve's correction x to it, which
// makes it D_k.  Solve 0 keeps hi and drops a stale lo.  x starts at 0.
// Per cell at k >= 4: read hi, lo and 3 differences; write hi, lo, c and x.
__device__ __forceinline__ float extrap_inc(long long k, float d1, float d2, float d3) {
  if (k <= 1) return 0.0f;
  if (k == 2) return d1;
  if (k == 3) return 2.0f * d1 - d2;
  return 3.0f * (d1 - d2) + d3;
}

__global__ void __launch_bounds__(FLAT_THREADS) k_extrap_comp(long long n, Comp<float> cp, float* __restrict__ x,
                                                             long long* nsolve, unsigned* ticket) {
  __shared__ bool last;
  const long long k = *nsolve;
  const float* const r1 = cp.ring[(k + 2) % 3];   // D_{k-1}
  const float* const r2 = cp.ring[(k + 1) % 3];   // D_{k-2}
  float* const r3 = cp.ring[k % 3];               // D_{k-3}, then c
  const long long stride = (long long)gridDim.x * FLAT_THREADS;
  const long long nvec = n / 4;
  auto one = [&](float& hi, float& lo, float d1, float d2, float d3) -> float {
    if (k == 0) {
      lo = 0.0f;
      return 0.0f;
    }
    const float c = extrap_inc(k, d1, d2, d3);
    const float2 sl = two_sum(hi, lo + c);
    hi = sl.x;
    lo = sl.y;
    return c;
  };
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < nvec; i += stride) {
    float4 h = reinterpret_cast<const float4*>(cp.hi)[i];
    float4 l = make_float4(0.f, 0.f, 0.f, 0.f), a = l, b = l, e = l;
    if (k >= 1) l = reinterpret_cast<const float4*>(cp.lo)[i];
    if (k >= 2) a = reinterpret_cast<const float4*>(r1)[i];
    if (k >= 3) b = reinterpret_cast<const float4*>(r2)[i];
    if (k >= 4) e = reinterpret_cast<const float4*>(r3)[i];
    float4 c;
    c.x = one(h.x, l.x, a.x, b.x, e.x);
    c.y = one(h.y, l.y, a.y, b.y, e.y);
    c.z = one(h.z, l.z, a.z, b.z, e.z);
    c.w = one(h.w, l.w, a.w, b.w, e.w);
    if (k >= 1) reinterpret_cast<float4*>(cp.hi)[i] = h;
    reinterpret_cast<float4*>(cp.lo)[i] = l;
    reinterpret_cast<float4*>(r3)[i] = c;
    reinterpret_cast<float4*>(x)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (long long i = nvec * 4 + blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += stride) {
    float h = cp.hi[i], l = k >= 1 ? cp.lo[i] : 0.0f;
    const float c = one(h, l, k >= 2 ? r1[i] : 0.0f, k >= 3 ? r2[i] : 0.0f, k >= 4 ? r3[i] : 0.0f);
    if (k >= 1) cp.hi[i] = h;
    cp.lo[i] = l;
    r3[i] = c;
    x[i] = 0.0f;
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
  if constexpr (std::is_same<T, float>::value) {
    if (d.cp.lo) {
      k_cg_finish<T, true><<<L.grid, L.block, 0, L.stream>>>(g, d.phi, d.p0, d.p1, d.part, d.S, 0, d.cp);
      return;
    }
  }
  k_cg_finish<T, false><<<L.grid, L.block, 0, L.stream>>>(g, d.phi, d.p0, d.p1, d.part, d.S, singular, d.cp);
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
void launch_extrap(const LaunchCfg& L, long long n, T* phi, T* const ring[3], long long* nsolve, unsigned* ticket) {
  k_extrap<T><<<L.flat_grid, FLAT_THREADS, 0, L.stream>>>(n, phi, ring[0], ring[1], ring[2], nsolve, ticket);
}

void launch_extrap_comp(const LaunchCfg& L, long long n, const Comp<float>& cp, float* x, long long* nsolve,
                        unsigned* ticket) {
  k_extrap_comp<<<L.flat_grid, FLAT_THREADS, 0, L.stream>>>(n, cp, x, nsolve, ticket);
}

#define PF_INSTANTIATE(T)                                                                                   \
  template void launch_extrap<T>(const LaunchCfg&, long long, T*, T* const[3], long long*, unsigned*);     \
  template void launch_cg_finish<T>(const LaunchCfg&, const Geo&, const Dev<T>&, int);                      \
  template void launch_sub_mean<T>(const LaunchCfg&, const Geo&, const Dev<T>&);                            \
  template void launch_invdiag<T>(const LaunchCfg&, const Geo&, const Dev<T>&);

PF_INSTANTIATE(float)
PF_INSTANTIATE(double)

}  // namespace pf
