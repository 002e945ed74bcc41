// Kernels of the TDGL + Poisson step (sm_103a).
//
//   (the right-hand side and TDGL kernels live in pf_step.cu, the CG
//   iteration kernels in pf_cg.cu, the multigrid V-cycle in pf_mg.cu)
//   k_cg_finish  last deferred x update / zero solution, mean of x
//   k_cg_finish_comp  the same for an FP32 time series: the compensated
//                potential and the next solve's extrapolated start
//   k_sub_mean   x -= mean(x)                           (singular problems)
//   k_invdiag    1/diag(A) when a permittivity field is bound
//   k_extrap     initial guess of a time step's Poisson solve extrapolated
//                from the last four solutions
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

// Increment of the extrapolated start of solve k over phi_{k-1}, from the
// differences d_j = phi_{k-j} - phi_{k-j-1} of the last solutions: constant
// (k <= 1), linear, quadratic, then cubic,
//   c = d1,  2 d1 - d2,  3 (d1 - d2) + d3,
// the increments of 2 phi_1 - phi_2, 3 phi_1 - 3 phi_2 + phi_3 and
// 4 phi_1 - 6 phi_2 + 4 phi_3 - phi_4 (phi_j = phi_{k-j}).
__device__ __forceinline__ float extrap_inc(long long k, float d1, float d2, float d3) {
  if (k <= 1) return 0.0f;
  if (k == 2) return d1;
  if (k == 3) return 2.0f * d1 - d2;
  return 3.0f * (d1 - d2) + d3;
}

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
      if (S->iter == 0) S->zero_solves += 1;
      S->total_iters += S->iter;
      S->last_iters = S->iter;
      S->solves += 1;
      if (S->iter > S->max_iters) S->max_iters = S->iter;
    if (S->iter < 2) S->short_solves += 1;
      if (S->status != 0) S->nonconv += 1;
      S->ticket = 0;
    }
  }
}

// COMP: the compensated potential of an FP32 time series (non-singular
// problems, extrapolated starts).  Rounding the potential to FP32 leaves a
// residual of order u |A| |phi|, above a 1e-7 tolerance on large films, and an
// extrapolation of rounded potentials would carry its weights' worth of it
// into every start.  So solve k starts from the pair hi + s, where hi is the
// bound phi (phi_{k-1} rounded to FP32) and s = lo + c_k holds the part of
// phi_{k-1} that hi cannot (lo) plus the extrapolation increment c_k; x is
// the correction the Krylov loop finds.  The ring holds the differences
// D_m = phi_m - phi_{m-1}, small beside phi and so nearly exact in FP32, in
// slot m mod 3; slot k holds c_k during solve k.  This kernel ends solve k:
//   phi_k = hi + s + x       -> (hi, lo) by TwoSum; phi = hi
//   D_k = c_k + x            -> slot k
//   c_{k+1} from D_k, D_{k-1}, D_{k-2} -> slot k + 1 (D_{k-2} read first)
//   s = lo + c_{k+1}, x = 0 (the next solve's start), and the count k + 1.
// A reset history starts with s = 0, slot 0 = 0, x = 0 and k = 0.
// x is not zeroed for the next solve: the solver state says when it is still
// 0 (unwritten since the start, S->xzero), and then it is not read.
// Per cell: read x (when written), p, hi, s and three slots; write hi, s and
// two slots (flat, 16-byte vectors).
__device__ __forceinline__ void finish_comp_cell(bool zero, long long k, int kcap, float dx, float& hi, float& sv,
                                                 float& ck, float d1, float& dm2) {
  float nlo, dk;
  if (zero) {                     // phi_k = 0 = phi_{k-1} + D_k, phi_{k-1} = hi + s - c_k
    dk = (ck - sv) - hi;
    hi = 0.0f;
    nlo = 0.0f;
  } else {
    const float2 sl = two_sum(hi, sv + dx);
    hi = sl.x;
    nlo = sl.y;
    dk = ck + dx;
  }
  const float cn = extrap_inc(k + 1 < kcap ? k + 1 : kcap, dk, d1, dm2);
  sv = nlo + cn;
  ck = dk;
  dm2 = cn;
}

__global__ void __launch_bounds__(FLAT_THREADS) k_cg_finish_comp(long long n, float* __restrict__ x,
                                                                const float* __restrict__ p0,
                                                                const float* __restrict__ p1, Scalars* S,
                                                                Comp<float> cp) {
  __shared__ bool last;
  const bool zero = S->zero_x;
  const int pend = S->pending;
  const int xz = S->xzero;
  const float alpha = float(S->alpha);
  const float* __restrict__ p = S->pbuf ? p1 : p0;
  const long long k = *cp.nsolve;
  float* const rk = cp.ring[k % 3];         // c_k, then D_k
  float* const r1 = cp.ring[(k + 2) % 3];   // D_{k-1}
  float* const r2 = cp.ring[(k + 1) % 3];   // D_{k-2}, then c_{k+1}
  const long long stride = (long long)gridDim.x * FLAT_THREADS;
  const long long nvec = n / 4;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < nvec; i += stride) {
    float4 xv = xz ? z4 : reinterpret_cast<const float4*>(x)[i];
    if (pend) {
      const float4 pv = reinterpret_cast<const float4*>(p)[i];
      xv.x += alpha * pv.x;
      xv.y += alpha * pv.y;
      xv.z += alpha * pv.z;
      xv.w += alpha * pv.w;
    }
    float4 h = reinterpret_cast<const float4*>(cp.hi)[i];
    float4 sv = reinterpret_cast<const float4*>(cp.lo)[i];
    float4 c = reinterpret_cast<const float4*>(rk)[i];
    const float4 a = k >= 1 ? reinterpret_cast<const float4*>(r1)[i] : z4;
    float4 b = k >= 2 ? reinterpret_cast<const float4*>(r2)[i] : z4;
    finish_comp_cell(zero, k, cp.kcap, xv.x, h.x, sv.x, c.x, a.x, b.x);
    finish_comp_cell(zero, k, cp.kcap, xv.y, h.y, sv.y, c.y, a.y, b.y);
    finish_comp_cell(zero, k, cp.kcap, xv.z, h.z, sv.z, c.z, a.z, b.z);
    finish_comp_cell(zero, k, cp.kcap, xv.w, h.w, sv.w, c.w, a.w, b.w);
    reinterpret_cast<float4*>(cp.hi)[i] = h;
    reinterpret_cast<float4*>(cp.lo)[i] = sv;
    reinterpret_cast<float4*>(rk)[i] = c;
    reinterpret_cast<float4*>(r2)[i] = b;
  }
  for (long long i = nvec * 4 + blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += stride) {
    const float xi = xz ? 0.0f : x[i];
    const float dx = pend ? xi + alpha * p[i] : xi;
    float h = cp.hi[i], sv = cp.lo[i], c = rk[i], b = k >= 2 ? r2[i] : 0.0f;
    finish_comp_cell(zero, k, cp.kcap, dx, h, sv, c, k >= 1 ? r1[i] : 0.0f, b);
    cp.hi[i] = h;
    cp.lo[i] = sv;
    rk[i] = c;
    r2[i] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    S->mean_x = 0.0;
    S->pending = 0;
    if (S->iter == 0) S->zero_solves += 1;
    S->total_iters += S->iter;
    S->last_iters = S->iter;
    S->solves += 1;
    if (S->iter > S->max_iters) S->max_iters = S->iter;
    if (S->iter < 2) S->short_solves += 1;
    if (S->status != 0) S->nonconv += 1;
    S->ticket = 0;
    *cp.nsolve = k + 1;
    __threadfence();
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

// Initial guess of solve number k of a time series (k = *nsolve), FP64 and
// singular FP32 problems: the cubic extrapolation 4 phi_1 - 6 phi_2 + 4 phi_3
// - phi_4 of the last four solutions (phi_1 = phi, the last one; the three
// before it sit in a ring of history fields, phi_j of solve number m in slot
// m mod 3).  Solves 1 to 3 take the orders their history allows: the given
// phi, the last solution, then the linear and quadratic extrapolations; kcap
// (1 + the highest order asked for) caps the order.  phi_1 goes into the slot
// of phi_4 once that has been read, so the ring never moves.  The last block
// to finish advances the count (every block reads it first).
// Streams phi and the ring once: read at most 4 words, write 2 words per cell.
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
                                                        long long* nsolve, unsigned* ticket, int kcap) {
  using V = typename Vec16<T>::type;
  constexpr int NV = 16 / sizeof(T);
  __shared__ bool last;
  const long long k = *nsolve;
  const long long ke = k < kcap ? k : kcap;   // the order: ke - 1 (at most the requested one)
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
    if (ke >= 2) v2 = reinterpret_cast<const V*>(h2)[i];
    if (ke >= 3) v3 = reinterpret_cast<const V*>(h3)[i];
    if (ke >= 4) v4 = reinterpret_cast<const V*>(h4)[i];
    V gv;
    const T* f1 = reinterpret_cast<const T*>(&v1);
    const T* f2 = reinterpret_cast<const T*>(&v2);
    const T* f3 = reinterpret_cast<const T*>(&v3);
    const T* f4 = reinterpret_cast<const T*>(&v4);
    T* gs = reinterpret_cast<T*>(&gv);
#pragma unroll
    for (int j = 0; j < NV; ++j) gs[j] = extrap_guess(ke, f1[j], f2[j], f3[j], f4[j]);
    if (k >= 1) reinterpret_cast<V*>(h4)[i] = v1;
    reinterpret_cast<V*>(phi)[i] = gv;
  }
  for (long long i = nvec * NV + blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < n; i += stride) {
    const T f1 = phi[i], f2 = ke >= 2 ? h2[i] : T(0), f3 = ke >= 3 ? h3[i] : T(0), f4 = ke >= 4 ? h4[i] : T(0);
    if (k >= 1) h4[i] = f1;
    phi[i] = extrap_guess(ke, f1, f2, f3, f4);
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
      k_cg_finish_comp<<<L.flat_grid, FLAT_THREADS, 0, L.stream>>>(g.n, d.phi, d.p0, d.p1, d.S, d.cp);
      return;
    }
  }
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
void launch_extrap(const LaunchCfg& L, long long n, T* phi, T* const ring[3], long long* nsolve, unsigned* ticket,
                   int kcap) {
  k_extrap<T><<<L.flat_grid, FLAT_THREADS, 0, L.stream>>>(n, phi, ring[0], ring[1], ring[2], nsolve, ticket, kcap);
}

#define PF_INSTANTIATE(T)                                                                                   \
  template void launch_extrap<T>(const LaunchCfg&, long long, T*, T* const[3], long long*, unsigned*, int); \
  template void launch_cg_finish<T>(const LaunchCfg&, const Geo&, const Dev<T>&, int);                      \
  template void launch_sub_mean<T>(const LaunchCfg&, const Geo&, const Dev<T>&);                            \
  template void launch_invdiag<T>(const LaunchCfg&, const Geo&, const Dev<T>&);

PF_INSTANTIATE(float)
PF_INSTANTIATE(double)

// ------------------------------------------------------- persistent step loops
// A whole multi-step call can run as ONE graph launch: a conditional while
// node whose body holds two time steps (one from each polarization buffer)
// and, last, k_loop_next, which counts the bodies down and sets the loop
// condition.  k_loop_set writes the count before the launch.
__global__ void k_loop_set(long long* left, long long n) { *left = n; }

__global__ void k_loop_next(long long* left, cudaGraphConditionalHandle h) {
  const long long v = *left - 1;
  *left = v;
  cudaGraphSetConditional(h, v > 0 ? 1u : 0u);
}

void launch_loop_set(long long* left, long long n, cudaStream_t st) { k_loop_set<<<1, 1, 0, st>>>(left, n); }

void launch_loop_next(long long* left, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_loop_next<<<1, 1, 0, st>>>(left, h);
}

}  // namespace pf
