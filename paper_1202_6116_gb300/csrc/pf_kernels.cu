// Kernels of the TDGL + Poisson step (sm_103a).
//
//   k_rhs_mean   sum of b = -div P + Dirichlet terms (singular problems only)
//   k_rhs        r0 = b - A phi, ||b||^2, ||r||^2, r.z   (Eqs. rho, Poisson)
//   k_cg_p       p = z + beta p (z = r / diag on the fly, halo included),
//                q = A p, deferred x += alpha p, p.q  -> alpha
//   k_cg_r       r -= alpha q, ||r||^2, r.z            -> beta, convergence
//   k_cg_finish  last deferred x update / zero solution, mean of x
//   k_sub_mean   x -= mean(x)                           (singular problems)
//   k_tdgl       forward-Euler TDGL update (Eqs. F_bulk, dF_grad/dP, F_elec, TDGL)
//   k_invdiag    1/diag(A) when a permittivity field is bound
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

// 1/diag(A) at cell (xy, z) for eps = 1.
template <typename T>
__device__ __forceinline__ T inv_diag_unit(const Geo& g, const Bc<T>& bc, const InvDiagTable<T>& tab,
                                           long long xy, int z) {
  if (g.periodic_z) return tab.v[6];
  int k = 4;
  k += (z > 0) ? 1 : 2 * (int)bc.tlo[xy];
  k += (z < g.nz - 1) ? 1 : 2 * (int)bc.thi[xy];
  return tab.v[k];
}

template <typename T, bool EPS>
__device__ __forceinline__ T inv_diag(const Geo& g, const Bc<T>& bc, const InvDiagTable<T>& tab,
                                      const T* __restrict__ invd, long long c, long long xy, int z) {
  if (EPS) return invd[c];
  return inv_diag_unit(g, bc, tab, xy, z);
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

// ------------------------------------------------------------ Poisson pieces

// b = -div P + (2 eps_c V / dx^2 per Dirichlet face), face values of P per
// the boundary kinds (mean inside, P_cell at an electrode, 0 at an open face).
template <typename T, bool EPS>
__device__ __forceinline__ T rhs_at(const Geo& g, const Bc<T>& bc, const T* __restrict__ P,
                                    const T* __restrict__ eps, const Nbr& n, int z) {
  const T* Px = P;
  const T* Py = P + g.n;
  const T* Pz = P + 2 * g.n;
  const T h = T(0.5);
  T div = T(0), dir = T(0);
  const T pxc = Px[n.c], pyc = Py[n.c], pzc = Pz[n.c];
  div += -(h * (pxc + Px[n.xm]));
  div += h * (pxc + Px[n.xp]);
  div += -(h * (pyc + Py[n.ym]));
  div += h * (pyc + Py[n.yp]);
  const T ec = EPS ? eps[n.c] : T(1);
  if (n.zm >= 0) {
    div += -(h * (pzc + Pz[n.zm]));
  } else if (bc.tlo[n.xy]) {
    div += -pzc;
    dir += T(2) * ec * bc.vlo[n.xy];
  }
  if (n.zp >= 0) {
    div += h * (pzc + Pz[n.zp]);
  } else if (bc.thi[n.xy]) {
    div += pzc;
    dir += T(2) * ec * bc.vhi[n.xy];
  }
  return -div * T(g.ih) + dir * T(g.ih2);
}

// (A v)_c with homogeneous boundary data: sum over faces of eps_f (v_c - v_nb),
// 2 eps_c v_c at an electrode face, nothing at an open face; / dx^2.
// vn[0..5] are the neighbour values (x-, x+, y-, y+, z-, z+).
template <typename T, bool EPS>
__device__ __forceinline__ T apply_at(const Geo& g, const Bc<T>& bc, const T* __restrict__ eps,
                                      const Nbr& n, T vc, const T (&vn)[6]) {
  T acc = T(0);
  if (EPS) {
    const T ec = eps[n.c];
    acc += hmean(ec, eps[n.xm]) * (vc - vn[0]);
    acc += hmean(ec, eps[n.xp]) * (vc - vn[1]);
    acc += hmean(ec, eps[n.ym]) * (vc - vn[2]);
    acc += hmean(ec, eps[n.yp]) * (vc - vn[3]);
    if (n.zm >= 0) acc += hmean(ec, eps[n.zm]) * (vc - vn[4]);
    else if (bc.tlo[n.xy]) acc += T(2) * ec * vc;
    if (n.zp >= 0) acc += hmean(ec, eps[n.zp]) * (vc - vn[5]);
    else if (bc.thi[n.xy]) acc += T(2) * ec * vc;
  } else {
    acc += vc - vn[0];
    acc += vc - vn[1];
    acc += vc - vn[2];
    acc += vc - vn[3];
    if (n.zm >= 0) acc += vc - vn[4];
    else if (bc.tlo[n.xy]) acc += T(2) * vc;
    if (n.zp >= 0) acc += vc - vn[5];
    else if (bc.thi[n.xy]) acc += T(2) * vc;
  }
  return acc * T(g.ih2);
}

// ------------------------------------------------------------------ kernels

template <typename T, bool EPS>
__global__ void __launch_bounds__(NTHREADS) k_rhs_mean(Geo g, Bc<T> bc, const T* __restrict__ P,
                                                       const T* __restrict__ eps, double* part,
                                                       Scalars* S) {
  Acc<T> acc;
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    TileCoord tc = tile_coord(g, t);
    if (!tc.active) continue;
    for (int z = tc.z0; z < tc.z1; ++z) {
      Nbr n = neighbours(g, tc.x, tc.y, z);
      acc.add(rhs_at<T, EPS>(g, bc, P, eps, n, z), T(1));
    }
    acc.flush();
  }
  double v[1] = {acc.value()};
  if (publish_partials<1>(v, part, &S->ticket)) {
    double out[1];
    gather_partials<1>(part, gridDim.x, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      S->mean_b = out[0] / (double)g.n;
      S->ticket = 0;
    }
  }
}

template <typename T, bool EPS>
__global__ void __launch_bounds__(NTHREADS) k_rhs(Geo g, Bc<T> bc, const T* __restrict__ P,
                                                  const T* __restrict__ phi, const T* __restrict__ eps,
                                                  const T* __restrict__ invd, InvDiagTable<T> tab,
                                                  T* __restrict__ r, double* part, Scalars* S,
                                                  cudaGraphConditionalHandle cond, int use_cond) {
  const T mb = T(S->mean_b);
  Acc<T> abb, arr, arz;
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    TileCoord tc = tile_coord(g, t);
    if (!tc.active) continue;
    for (int z = tc.z0; z < tc.z1; ++z) {
      Nbr n = neighbours(g, tc.x, tc.y, z);
      const T b = rhs_at<T, EPS>(g, bc, P, eps, n, z) - mb;
      const T vc = phi[n.c];
      const T vn[6] = {phi[n.xm], phi[n.xp], phi[n.ym], phi[n.yp],
                       n.zm >= 0 ? phi[n.zm] : T(0), n.zp >= 0 ? phi[n.zp] : T(0)};
      const T rv = b - apply_at<T, EPS>(g, bc, eps, n, vc, vn);
      const T zv = rv * inv_diag<T, EPS>(g, bc, tab, invd, n.c, n.xy, z);
      r[n.c] = rv;
      abb.add(b, b);
      arr.add(rv, rv);
      arz.add(rv, zv);
    }
    abb.flush();
    arr.flush();
    arz.flush();
  }
  double v[3] = {abb.value(), arr.value(), arz.value()};
  if (publish_partials<3>(v, part, &S->ticket)) {
    double out[3];
    gather_partials<3>(part, gridDim.x, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const double bb = out[0], rr = out[1], rz = out[2];
      S->bb = bb;
      S->rr = rr;
      S->rz = rz;
      S->iter = 0;
      S->first = 1;
      S->pending = 0;
      S->status = 0;
      S->alpha = 0.0;
      S->beta = 0.0;
      if (!isfinite(bb) || !isfinite(rr)) {
        S->nonfinite = 1;
        S->zero_x = 0;
        S->done = 1;
        S->last_rel = rr;
      } else if (bb == 0.0) {
        S->zero_x = 1;
        S->done = 1;
        S->last_rel = 0.0;
      } else {
        const double rel = sqrt(rr) / sqrt(bb);
        S->zero_x = 0;
        S->last_rel = rel;
        S->done = (rel < S->rtol) ? 1 : 0;
      }
      S->ticket = 0;
      if (use_cond) cudaGraphSetConditional(cond, S->done ? 0u : 1u);
    }
  }
}

// p_new = r/diag + beta p_old at cell i (p_new = r/diag on the first iteration).
template <typename T>
__device__ __forceinline__ T pnew_at(const T* __restrict__ r, const T* __restrict__ pold, long long i,
                                     T inv, T beta, int first) {
  const T zv = r[i] * inv;
  return first ? zv : zv + beta * pold[i];
}

template <typename T, bool EPS>
__global__ void __launch_bounds__(NTHREADS) k_cg_p(Geo g, Bc<T> bc, const T* __restrict__ eps,
                                                   const T* __restrict__ invd, InvDiagTable<T> tab,
                                                   const T* __restrict__ r, T* p0, T* p1,
                                                   T* __restrict__ q, T* __restrict__ x, double* part,
                                                   Scalars* S) {
  if (S->done) return;
  const int first = S->first;
  const T beta = first ? T(0) : T(S->beta);
  const T alpha = T(S->alpha);
  const int pb = S->pbuf;
  const T* __restrict__ pold = pb ? p1 : p0;
  T* __restrict__ pnew = pb ? p0 : p1;
  Acc<T> apq;
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    TileCoord tc = tile_coord(g, t);
    if (!tc.active) continue;
    for (int z = tc.z0; z < tc.z1; ++z) {
      Nbr n = neighbours(g, tc.x, tc.y, z);
      const T pc = pnew_at(r, pold, n.c, inv_diag<T, EPS>(g, bc, tab, invd, n.c, n.xy, z), beta, first);
      T vn[6];
      vn[0] = pnew_at(r, pold, n.xm, inv_diag<T, EPS>(g, bc, tab, invd, n.xm, n.xmy, z), beta, first);
      vn[1] = pnew_at(r, pold, n.xp, inv_diag<T, EPS>(g, bc, tab, invd, n.xp, n.xpy, z), beta, first);
      vn[2] = pnew_at(r, pold, n.ym, inv_diag<T, EPS>(g, bc, tab, invd, n.ym, n.xym, z), beta, first);
      vn[3] = pnew_at(r, pold, n.yp, inv_diag<T, EPS>(g, bc, tab, invd, n.yp, n.xyp, z), beta, first);
      if (n.zm >= 0) {
        const int zz = (z > 0) ? z - 1 : g.nz - 1;
        vn[4] = pnew_at(r, pold, n.zm, inv_diag<T, EPS>(g, bc, tab, invd, n.zm, n.xy, zz), beta, first);
      } else {
        vn[4] = T(0);
      }
      if (n.zp >= 0) {
        const int zz = (z < g.nz - 1) ? z + 1 : 0;
        vn[5] = pnew_at(r, pold, n.zp, inv_diag<T, EPS>(g, bc, tab, invd, n.zp, n.xy, zz), beta, first);
      } else {
        vn[5] = T(0);
      }
      const T qv = apply_at<T, EPS>(g, bc, eps, n, pc, vn);
      if (!first) x[n.c] += alpha * pold[n.c];
      pnew[n.c] = pc;
      q[n.c] = qv;
      apq.add(pc, qv);
    }
    apq.flush();
  }
  double v[1] = {apq.value()};
  if (publish_partials<1>(v, part, &S->ticket)) {
    double out[1];
    gather_partials<1>(part, gridDim.x, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const double pq = out[0];
      S->pq = pq;
      S->iter += 1;
      S->pbuf = pb ^ 1;
      S->first = 0;
      if (!(pq > 0.0)) {               // breakdown (or NaN): stop with the current iterate
        if (!isfinite(pq)) S->nonfinite = 1;
        S->alpha = 0.0;
        S->pending = 0;
        S->status = 3;
        S->done = 1;
      } else {
        S->alpha = S->rz / pq;
      }
      S->ticket = 0;
    }
  }
}

template <typename T, bool EPS>
__global__ void __launch_bounds__(NTHREADS) k_cg_r(Geo g, Bc<T> bc, const T* __restrict__ invd,
                                                   InvDiagTable<T> tab, T* __restrict__ r,
                                                   const T* __restrict__ q, double* part, Scalars* S,
                                                   cudaGraphConditionalHandle cond, int use_cond) {
  if (S->done) return;
  const T alpha = T(S->alpha);
  Acc<T> arr, arz;
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    TileCoord tc = tile_coord(g, t);
    if (!tc.active) continue;
    for (int z = tc.z0; z < tc.z1; ++z) {
      const long long xy = (long long)tc.y * g.nx + tc.x;
      const long long c = (long long)z * g.nxy + xy;
      const T rv = r[c] - alpha * q[c];
      r[c] = rv;
      const T zv = rv * inv_diag<T, EPS>(g, bc, tab, invd, c, xy, z);
      arr.add(rv, rv);
      arz.add(rv, zv);
    }
    arr.flush();
    arz.flush();
  }
  double v[2] = {arr.value(), arz.value()};
  if (publish_partials<2>(v, part, &S->ticket)) {
    double out[2];
    gather_partials<2>(part, gridDim.x, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const double rr = out[0], rz = out[1];
      const double rel = sqrt(rr) / sqrt(S->bb);
      S->rr = rr;
      S->last_rel = rel;
      if (!isfinite(rr)) {
        S->nonfinite = 1;
        S->status = 3;
        S->pending = 0;
        S->done = 1;
      } else if (rel < S->rtol) {
        S->pending = 1;
        S->done = 1;
      } else if (S->iter >= S->maxit) {
        S->pending = 1;
        S->status = 3;
        S->done = 1;
      } else {
        S->beta = rz / S->rz;
        S->rz = rz;
      }
      S->ticket = 0;
      if (use_cond) cudaGraphSetConditional(cond, S->done ? 0u : 1u);
    }
  }
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

// Forward-Euler TDGL update of one cell (Eq. TDGL with Eqs. F_bulk,
// dF_grad/dP and F_elec): P' = P + dt L (-df/dP + g Lap P + E).
template <typename T>
struct Coef {
  T a1, a11, a12, g, dtL;
};

template <typename T, bool EPS>
__global__ void __launch_bounds__(NTHREADS) k_tdgl(Geo g, Bc<T> bc, const T* __restrict__ P,
                                                   T* __restrict__ Pn, const T* __restrict__ phi,
                                                   Coef<T> k) {
  for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    TileCoord tc = tile_coord(g, t);
    if (!tc.active) continue;
    for (int z = tc.z0; z < tc.z1; ++z) {
      Nbr n = neighbours(g, tc.x, tc.y, z);
      T p[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) p[i] = P[i * g.n + n.c];
      // E = -grad phi from face values
      const T h = T(0.5);
      const T fc = phi[n.c];
      T E[3];
      E[0] = -(h * (fc + phi[n.xp]) - h * (fc + phi[n.xm])) * T(g.ih);
      E[1] = -(h * (fc + phi[n.yp]) - h * (fc + phi[n.ym])) * T(g.ih);
      T flo, fhi;
      if (n.zm >= 0) flo = h * (fc + phi[n.zm]);
      else flo = bc.tlo[n.xy] ? bc.vlo[n.xy] : fc;
      if (n.zp >= 0) fhi = h * (fc + phi[n.zp]);
      else fhi = bc.thi[n.xy] ? bc.vhi[n.xy] : fc;
      E[2] = -(fhi - flo) * T(g.ih);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, l = (i + 2) % 3;
        const T hi_ = T(2) * k.a1 * p[i] + T(4) * k.a11 * p[i] * p[i] * p[i] +
                      T(2) * k.a12 * p[i] * (p[j] * p[j] + p[l] * p[l]);
        const T* Pi = P + i * g.n;
        T lap = T(0);
        lap += Pi[n.xm] - p[i];
        lap += Pi[n.xp] - p[i];
        lap += Pi[n.ym] - p[i];
        lap += Pi[n.yp] - p[i];
        if (n.zm >= 0) lap += Pi[n.zm] - p[i];
        if (n.zp >= 0) lap += Pi[n.zp] - p[i];
        lap *= T(g.ih2);
        Pn[i * g.n + n.c] = p[i] + k.dtL * (-hi_ + k.g * lap + E[i]);
      }
    }
  }
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

// ---------------------------------------------------------------- launchers

template <typename T>
void launch_rhs_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P) {
  if (d.eps) k_rhs_mean<T, true><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, P, d.eps, d.part, d.S);
  else k_rhs_mean<T, false><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, P, d.eps, d.part, d.S);
}

template <typename T>
void launch_rhs(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, cudaGraphConditionalHandle cond,
                int use_cond) {
  if (d.eps)
    k_rhs<T, true><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, P, d.phi, d.eps, d.invd, d.tab, d.r, d.part,
                                                      d.S, cond, use_cond);
  else
    k_rhs<T, false><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, P, d.phi, d.eps, d.invd, d.tab, d.r, d.part,
                                                       d.S, cond, use_cond);
}

template <typename T>
void launch_cg_p(const LaunchCfg& L, const Geo& g, const Dev<T>& d) {
  if (d.eps)
    k_cg_p<T, true><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, d.eps, d.invd, d.tab, d.r, d.p0, d.p1, d.q,
                                                       d.phi, d.part, d.S);
  else
    k_cg_p<T, false><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, d.eps, d.invd, d.tab, d.r, d.p0, d.p1, d.q,
                                                        d.phi, d.part, d.S);
}

template <typename T>
void launch_cg_r(const LaunchCfg& L, const Geo& g, const Dev<T>& d, cudaGraphConditionalHandle cond,
                 int use_cond) {
  if (d.eps)
    k_cg_r<T, true><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, d.invd, d.tab, d.r, d.q, d.part, d.S, cond,
                                                       use_cond);
  else
    k_cg_r<T, false><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, d.invd, d.tab, d.r, d.q, d.part, d.S, cond,
                                                        use_cond);
}

template <typename T>
void launch_cg_finish(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int singular) {
  k_cg_finish<T><<<L.grid, L.block, 0, L.stream>>>(g, d.phi, d.p0, d.p1, d.part, d.S, singular);
}

template <typename T>
void launch_sub_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d) {
  k_sub_mean<T><<<L.grid, L.block, 0, L.stream>>>(g, d.phi, d.S);
}

template <typename T>
void launch_tdgl(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, T* Pn, const double* coef) {
  Coef<T> k{T(coef[0]), T(coef[1]), T(coef[2]), T(coef[3]), T(coef[4])};
  if (d.eps) k_tdgl<T, true><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, P, Pn, d.phi, k);
  else k_tdgl<T, false><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, P, Pn, d.phi, k);
}

template <typename T>
void launch_invdiag(const LaunchCfg& L, const Geo& g, const Dev<T>& d) {
  k_invdiag<T><<<L.grid, L.block, 0, L.stream>>>(g, d.bc, d.eps, d.invd);
}

#define PF_INSTANTIATE(T)                                                                                   \
  template void launch_rhs_mean<T>(const LaunchCfg&, const Geo&, const Dev<T>&, const T*);                   \
  template void launch_rhs<T>(const LaunchCfg&, const Geo&, const Dev<T>&, const T*,                         \
                              cudaGraphConditionalHandle, int);                                             \
  template void launch_cg_p<T>(const LaunchCfg&, const Geo&, const Dev<T>&);                                 \
  template void launch_cg_r<T>(const LaunchCfg&, const Geo&, const Dev<T>&, cudaGraphConditionalHandle, int);\
  template void launch_cg_finish<T>(const LaunchCfg&, const Geo&, const Dev<T>&, int);                      \
  template void launch_sub_mean<T>(const LaunchCfg&, const Geo&, const Dev<T>&);                            \
  template void launch_tdgl<T>(const LaunchCfg&, const Geo&, const Dev<T>&, const T*, T*, const double*);   \
  template void launch_invdiag<T>(const LaunchCfg&, const Geo&, const Dev<T>&);

PF_INSTANTIATE(float)
PF_INSTANTIATE(double)

}  // namespace pf
