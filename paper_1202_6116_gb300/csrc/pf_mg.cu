// Geometric multigrid V-cycle used as the CG preconditioner z = M^-1 r.
//
// Cell-centred hierarchy: each level halves every dimension that is even
// (2 x 2 x 2 cells -> 1), the operator is re-discretised on every level
// (per-direction spacings, so semi-coarsened levels stay consistent), a
// coarse z face is an electrode where any of its fine children is, and the
// error equation has homogeneous boundary data.  Transfers: restriction is
// the average of the children, prolongation is piecewise constant (its
// scaled transpose), smoothing is two Jacobi sweeps with the Chebyshev weights
// of mg_omega1/mg_omega2 before the coarse correction and the same two in
// reverse order after it (the adjoint smoother), so the V-cycle is a symmetric
// positive definite preconditioner.  The coarsest level (<= MG_MAX_COARSE cells) is
// solved by FP64 conjugate gradients inside one thread block.
//
// Per level and V-cycle (nu = 2):
//   k_mg_pre     e = two Jacobi sweeps from zero (the first sweep w1 f/diag
//                is formed on the fly, halo included)   reads f, writes e
//   k_mg_rr      r = f - A e and its restriction to the next level's rhs,
//                summed over 2 x 2 columns by warp shuffles and over 2 planes
//                in registers                            reads e, f, writes f_c
//   k_mg_post1   e' = e + P e_c, one Jacobi sweep        reads e, e_c, f, writes et
//   k_mg_post2   one Jacobi sweep (finest level: also r.z -> beta)
//                                                        reads et, f, writes e
#include "pf_internal.h"
#include "pf_march.cuh"

namespace pf {

constexpr int MG_D = 2;   // planes of cp.async look-ahead

// Jacobi weights of the two smoothing sweeps: the reciprocals of the roots of
// the degree-2 Chebyshev polynomial on [b/4, b], b = 1.9, which bound the
// spectrum of diag(A)^-1 A (in [0, 2] for this M-matrix) from below b/4 up,
// i.e. 1/lambda_k with lambda_k = (b + a)/2 + (b - a)/2 cos((2k - 1) pi / 4),
// a = b/4.  The pair damps the upper three quarters of the spectrum (the part
// the coarse grid cannot represent) by |(1 - w1 l)(1 - w2 l)| <= 0.35 on
// [b/4, 2]; weighted Jacobi with 6/7 twice leaves up to 0.51 there.  The
// pre-smoother applies w1 then w2, the post-smoother w2 then w1.
template <typename T>
__device__ __forceinline__ T mg_omega1() {
  return T(0.5912564121058501);
}
template <typename T>
__device__ __forceinline__ T mg_omega2() {
  return T(1.462658863889015);
}

// 1/diag of a level's operator at column xy of plane z.
template <typename T>
__device__ __forceinline__ T mg_inv(const MgView<T>& L, int xy, int z, T inv_int) {
  if (L.g.periodic_z || (z > 0 && z < L.g.nz - 1)) return inv_int;
  const int cz = (z > 0 ? 1 : 2 * (int)L.tlo[xy]) + (z < L.g.nz - 1 ? 1 : 2 * (int)L.thi[xy]);
  return T(1) / (T(2) * L.ax + T(2) * L.ay + T(cz) * L.az);
}

template <typename T>
__device__ __forceinline__ T mg_inv_int(const MgView<T>& L) {
  return T(1) / (T(2) * L.ax + T(2) * L.ay + T(2) * L.az);
}

// A v at a level with per-direction coefficients ax, ay, az = 1/h^2; the z
// face logic only on the planes next to a z face (bt).
template <typename T>
__device__ __forceinline__ T apply_aniso(const Stencil7<T>& s, int dlo, int dhi, T ax, T ay, T az, const bool bt) {
  const T sx = (s.c - s.xm) + (s.c - s.xp);
  const T sy = (s.c - s.ym) + (s.c - s.yp);
  T sz = T(0);
  if (bt) {
    if (s.zb >= 0) sz += s.c - s.zm;
    else if (dlo) sz += T(2) * s.c;
    if (s.za >= 0) sz += s.c - s.zp;
    else if (dhi) sz += T(2) * s.c;
  } else {
    sz = (s.c - s.zm) + (s.c - s.zp);
  }
  return ax * sx + ay * sy + az * sz;
}

template <typename T>
__device__ __forceinline__ T mg_inv_bt(const MgView<T>& L, int xy, int z, T inv_int, const bool bt) {
  return bt ? mg_inv(L, xy, z, inv_int) : inv_int;
}

template <typename T, int VX>
using MgPipeD0 = Pipe<T, void, MTX, MTY, VX, 1, 0, MG_D>;
template <typename T, int VX>
using MgPipeP = Pipe<T, void, MTX, MTY, VX, 1, 1, MG_D, 1>;
// stencil read straight from the staged planes (no field buffer)
template <typename T, int VX>
using MgPipeD = Pipe<T, void, MTX, MTY, VX, 1, 1, MG_D>;

// ------------------------------------------------------------------ kernels

// Two pre-smoothing sweeps from zero, read straight from the staged planes of
// f.  The first sweep is e1 = w1 diag^-1 f; the second e = e1 + w2 diag^-1 (f -
// A e1).  Away from the z faces the diagonal is one constant, so A e1 =
// w1 diag^-1 A f there; on the planes next to a z face and their neighbour
// planes e1 is formed per neighbour with its own diagonal.
template <typename T, int VX>
__global__ void __launch_bounds__(MTX* MTY) k_mg_pre(MgView<T> L, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  if (S->done) return;
  const T om1 = mg_omega1<T>(), om2 = mg_omega2<T>(), inv_int = mg_inv_int(L);
  const T w1 = om1 * inv_int;
  const T* hsrc[1] = {L.f};
  const T* osrc[1] = {nullptr};
  const int nx = L.g.nx, nz = L.g.nz;
  const bool zfaces = !L.g.periodic_z;
  TileGeo<MTX, MTY, VX> s;
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, 1>>& sr, const T (&)[1], const bool bt) -> T {
    const Stencil7<T> f = pick(sr, 0);
    const bool near = zfaces && (z == 1 || z == nz - 2);
    if (!bt && !near) {
      const T Ae1 = w1 * apply_aniso(f, 0, 0, L.ax, L.ay, L.az, false);
      return w1 * f.c + om2 * inv_int * (f.c - Ae1);
    }
    Stencil7<T> e1;
    const T ic = mg_inv(L, xy, z, inv_int);
    e1.c = om1 * ic * f.c;
    if (bt) {
      const int x = xy % nx, rb = xy - x;
      const int xm = rb + (x == 0 ? nx - 1 : x - 1), xp = rb + (x == nx - 1 ? 0 : x + 1);
      const int y = xy / nx;
      const int ym = (y == 0 ? L.g.ny - 1 : y - 1) * nx + x, yp = (y == L.g.ny - 1 ? 0 : y + 1) * nx + x;
      e1.xm = om1 * mg_inv(L, xm, z, inv_int) * f.xm;
      e1.xp = om1 * mg_inv(L, xp, z, inv_int) * f.xp;
      e1.ym = om1 * mg_inv(L, ym, z, inv_int) * f.ym;
      e1.yp = om1 * mg_inv(L, yp, z, inv_int) * f.yp;
    } else {
      e1.xm = w1 * f.xm;
      e1.xp = w1 * f.xp;
      e1.ym = w1 * f.ym;
      e1.yp = w1 * f.yp;
    }
    e1.zm = f.zb >= 0 ? om1 * mg_inv(L, xy, z - 1, inv_int) * f.zm : T(0);
    e1.zp = f.za >= 0 ? om1 * mg_inv(L, xy, z + 1, inv_int) * f.zp : T(0);
    e1.zb = f.zb;
    e1.za = f.za;
    const int dlo = (bt && f.zb < 0) ? (int)L.tlo[xy] : 0;
    const int dhi = (bt && f.za < 0) ? (int)L.thi[xy] : 0;
    const T Ae1 = apply_aniso(e1, dlo, dhi, L.ax, L.ay, L.az, bt);
    return e1.c + om2 * ic * (f.c - Ae1);
  };
  auto post = [&](int z, const T (&ov)[VX]) { store_n<T, VX>(L.e + (long long)z * L.g.nxy + s.xy, ov); };
  const TileSched ts{&S->sched_next, &S->sched_done};
  for (long long t = sched_take(ts, &tile_slot); t < L.mc.ntiles; t = sched_take(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(L.g, t, L.mc);
    march_direct<T, T, MTX, MTY, VX, 1, 0, MG_D>(L.g, s, smem, hsrc, osrc, emit, post);
  }
  sched_finish(ts);
}

// Residual and its restriction.  Children of one coarse cell: 2 planes (summed
// in registers across consecutive planes of the march), 2 rows (tile rows 2k,
// 2k+1 share a warp: lane ^ 16), 2 columns (inside the thread's vector, or
// lane ^ 1 when a thread owns one cell).
template <typename T, int VX>
__global__ void __launch_bounds__(MTX* MTY) k_mg_rr(MgView<T> L, MgView<T> C, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  static_assert(MTX == 16, "row pairs share a warp");
  if (S->done) return;
  const T* hsrc[1] = {L.e};
  const T* osrc[1] = {L.f};
  const T scale = T(1) / T(L.fx * L.fy * L.fz);
  TileGeo<MTX, MTY, VX> s;
  T racc[VX];
#pragma unroll
  for (int i = 0; i < VX; ++i) racc[i] = T(0);
  auto emit = [&](int xy, int, const Stencil7<Raw<T, 1>>& sr, const T (&o)[1], const bool bt) -> T {
    const Stencil7<T> st = pick(sr, 0);
    const bool B = bt;
    const int dlo = (B && st.zb < 0) ? (int)L.tlo[xy] : 0;
    const int dhi = (B && st.za < 0) ? (int)L.thi[xy] : 0;
    return o[0] - apply_aniso(st, dlo, dhi, L.ax, L.ay, L.az, bt);
  };
  auto post = [&](int z, const T (&rv)[VX]) {
#pragma unroll
    for (int i = 0; i < VX; ++i) racc[i] += rv[i];
    if ((z & (L.fz - 1)) != L.fz - 1) return;      // factors are 1 or 2
    T v[VX];
#pragma unroll
    for (int i = 0; i < VX; ++i) {
      v[i] = racc[i];
      racc[i] = T(0);
    }
    const unsigned m = __activemask();
    if (L.fy == 2) {
#pragma unroll
      for (int i = 0; i < VX; ++i) v[i] += __shfl_xor_sync(m, v[i], 16);
    }
    int cnt = VX;
    if (L.fx == 2) {
      if constexpr (VX >= 2) {
#pragma unroll
        for (int j = 0; j < VX / 2; ++j) v[j] = v[2 * j] + v[2 * j + 1];
        cnt = VX / 2;
      } else {
        v[0] += __shfl_xor_sync(m, v[0], 1);
      }
    }
    const bool lead_y = L.fy == 1 || (s.y & 1) == 0;
    const bool lead_x = VX >= 2 || L.fx == 1 || (s.x & 1) == 0;
    if (lead_y && lead_x) {
      T* dst = C.f + (long long)(z >> (L.fz - 1)) * C.g.nxy + (long long)(s.y >> (L.fy - 1)) * C.g.nx +
               (s.x >> (L.fx - 1));
      for (int j = 0; j < cnt; ++j) dst[j] = v[j] * scale;
    }
  };
  const TileSched ts{&S->sched_next, &S->sched_done};
  for (long long t = sched_take(ts, &tile_slot); t < L.mc.ntiles; t = sched_take(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(L.g, t, L.mc);
    march_direct<T, T, MTX, MTY, VX, 1, 1, MG_D>(L.g, s, smem, hsrc, osrc, emit, post);
  }
  sched_finish(ts);
}

// Prolongation + correction fused into the first post-smoothing sweep: the
// stencil field is e + e_c(parent), the parents staged with the fine planes
// and combined with e at each of the seven cells.
template <typename T, int VX>
__global__ void __launch_bounds__(MTX* MTY, sizeof(T) == 4 ? 3 : 2) k_mg_post1(MgView<T> L, MgView<T> C, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  if (S->done) return;
  const T om = mg_omega2<T>(), inv_int = mg_inv_int(L);
  const T* hsrc[1] = {L.e};
  const T* osrc[1] = {L.f};
  const ParentSrc<T> par{C.e, L.fx, L.fy, L.fz, C.g.nx, C.g.nxy};
  TileGeo<MTX, MTY, VX> s;
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, 2>>& sr, const T (&o)[1], const bool bt) -> T {
    Stencil7<T> st;
    st.c = sr.c.v[0] + sr.c.v[1];
    st.xm = sr.xm.v[0] + sr.xm.v[1];
    st.xp = sr.xp.v[0] + sr.xp.v[1];
    st.ym = sr.ym.v[0] + sr.ym.v[1];
    st.yp = sr.yp.v[0] + sr.yp.v[1];
    st.zm = sr.zm.v[0] + sr.zm.v[1];
    st.zp = sr.zp.v[0] + sr.zp.v[1];
    st.zb = sr.zb;
    st.za = sr.za;
    const bool B = bt;
    const int dlo = (B && st.zb < 0) ? (int)L.tlo[xy] : 0;
    const int dhi = (B && st.za < 0) ? (int)L.thi[xy] : 0;
    const T Ae = apply_aniso(st, dlo, dhi, L.ax, L.ay, L.az, bt);
    return st.c + om * mg_inv_bt(L, xy, z, inv_int, bt) * (o[0] - Ae);
  };
  auto post = [&](int z, const T (&ov)[VX]) { store_n<T, VX>(L.et + (long long)z * L.g.nxy + s.xy, ov); };
  const TileSched ts{&S->sched_next, &S->sched_done};
  for (long long t = sched_take(ts, &tile_slot); t < L.mc.ntiles; t = sched_take(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(L.g, t, L.mc);
    march_direct<T, T, MTX, MTY, VX, 1, 1, MG_D, 1>(L.g, s, smem, hsrc, osrc, emit, post, par);
  }
  sched_finish(ts);
}

// Last post-smoothing sweep.  On the finest level (LAST) it also forms
// r.z (f = r, e = z): the last block sets beta = (r.z)_new / (r.z)_old.
template <typename T, bool LAST, int VX>
__global__ void __launch_bounds__(MTX* MTY) k_mg_post2(MgView<T> L, double* part, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  if (S->done) return;
  const T om = mg_omega1<T>(), inv_int = mg_inv_int(L);
  const T* hsrc[1] = {L.et};
  const T* osrc[1] = {L.f};
  Acc<T> arz;
  TileGeo<MTX, MTY, VX> s;
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, 1>>& sr, const T (&o)[1], const bool bt) -> T {
    const Stencil7<T> st = pick(sr, 0);
    const bool B = bt;
    const int dlo = (B && st.zb < 0) ? (int)L.tlo[xy] : 0;
    const int dhi = (B && st.za < 0) ? (int)L.thi[xy] : 0;
    const T Ae = apply_aniso(st, dlo, dhi, L.ax, L.ay, L.az, bt);
    const T e = st.c + om * mg_inv_bt(L, xy, z, inv_int, bt) * (o[0] - Ae);
    if (LAST) arz.add(o[0], e);
    return e;
  };
  auto post = [&](int z, const T (&ov)[VX]) { store_n<T, VX>(L.e + (long long)z * L.g.nxy + s.xy, ov); };
  const TileSched ts{&S->sched_next, &S->sched_done};
  for (long long t = sched_take(ts, &tile_slot); t < L.mc.ntiles; t = sched_take(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(L.g, t, L.mc);
    arz = Acc<T>();
    march_direct<T, T, MTX, MTY, VX, 1, 1, MG_D>(L.g, s, smem, hsrc, osrc, emit, post);
    if (LAST) {
      double v[1] = {arz.value()};
      tile_partials<1, MTX * MTY>(v, part, t);
    }
  }
  sched_finish(ts);
  if (!LAST) return;
  if (last_block<MTX * MTY>(&S->ticket)) {
    double out[1];
    gather_partials<1, MTX * MTY>(part, L.mc.ntiles, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const double rz = out[0];
      if (!isfinite(rz)) {
        S->nonfinite = 1;
        S->status = 3;
        S->pending = 0;
        S->done = 1;
      } else {
        if (!S->first) S->beta = rz / S->rz;
        S->rz = rz;
      }
      S->ticket = 0;
    }
  }
}

// ------------------------------------------------------ coarsest-level solve

__device__ __forceinline__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();                 // red[] may still be read from the previous call
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];   // same order in every thread
  return s;
}

// Conjugate gradients on the coarsest level, FP64, one block, one cell per
// thread (n <= MG_MAX_COARSE <= blockDim.x), to a relative residual of 1e-12.
// With no electrode the level is singular: the right-hand side and the
// solution are projected to zero mean.  Every thread of the block calls it.
template <typename T>
__device__ __forceinline__ void mg_coarse_solve(const MgView<T>& C, const T* cf, T* ce, int singular, double* ps,
                                                double* red) {
  const int n = (int)C.g.n, tid = threadIdx.x;
  const bool on = tid < n;
  int x = 0, y = 0, z = 0;
  if (on) {
    x = tid % C.g.nx;
    y = (tid / C.g.nx) % C.g.ny;
    z = tid / (int)C.g.nxy;
  }
  const int xm = (x == 0 ? C.g.nx - 1 : x - 1) + (tid - x), xp = (x == C.g.nx - 1 ? 0 : x + 1) + (tid - x);
  const int rowo = z * (int)C.g.nxy;
  const int ym = rowo + (y == 0 ? C.g.ny - 1 : y - 1) * C.g.nx + x;
  const int yp = rowo + (y == C.g.ny - 1 ? 0 : y + 1) * C.g.nx + x;
  const int zb = z > 0 ? z - 1 : (C.g.periodic_z ? C.g.nz - 1 : -1);
  const int za = z < C.g.nz - 1 ? z + 1 : (C.g.periodic_z ? 0 : -1);
  const int zm = zb >= 0 ? zb * (int)C.g.nxy + y * C.g.nx + x : -1;
  const int zp = za >= 0 ? za * (int)C.g.nxy + y * C.g.nx + x : -1;
  const int xy = y * C.g.nx + x;
  const double ax = C.ax, ay = C.ay, az = C.az;
  const int dlo = (on && zb < 0) ? (int)C.tlo[xy] : 0;
  const int dhi = (on && za < 0) ? (int)C.thi[xy] : 0;
  auto apply = [&](const double* v) -> double {
    const double c = v[tid];
    double sz = 0.0;
    if (zm >= 0) sz += c - v[zm];
    else if (dlo) sz += 2.0 * c;
    if (zp >= 0) sz += c - v[zp];
    else if (dhi) sz += 2.0 * c;
    return ax * ((c - v[xm]) + (c - v[xp])) + ay * ((c - v[ym]) + (c - v[yp])) + az * sz;
  };
  double b = on ? (double)cf[tid] : 0.0;
  if (singular) b -= block_sum(b, red) / n;
  double xv = 0.0, r = b;
  double rr = block_sum(r * r, red);
  const double bb = rr;
  if (bb > 0.0) {
    double p = r;
    for (int it = 0; it < 4 * n + 20; ++it) {
      __syncthreads();             // ps[] may still be read from the previous iteration
      if (on) ps[tid] = p;
      __syncthreads();
      const double q = on ? apply(ps) : 0.0;
      const double pq = block_sum(p * q, red);
      if (!(pq > 0.0)) break;
      const double a = rr / pq;
      xv += a * p;
      r -= a * q;
      const double rrn = block_sum(r * r, red);
      if (rrn <= 1e-24 * bb) break;
      p = r + (rrn / rr) * p;
      rr = rrn;
    }
  }
  if (singular) xv -= block_sum(on ? xv : 0.0, red) / n;
  if (on) ce[tid] = (T)xv;
}

template <typename T>
__global__ void __launch_bounds__(MG_MAX_COARSE) k_mg_coarse(MgView<T> C, int singular, Scalars* S) {
  __shared__ double ps[MG_MAX_COARSE];
  __shared__ double red[32];
  if (S->done) return;
  mg_coarse_solve(C, C.f, C.e, singular, ps, red);
}

// ------------------------------------------------------------ the V-cycle tail

// A v at cell c of a small level, neighbours read from global memory.
template <typename T>
__device__ __forceinline__ T tail_apply(const MgView<T>& L, const T* v, int c, T& inv) {
  const int nx = L.g.nx, ny = L.g.ny, nz = L.g.nz, nxy = (int)L.g.nxy;
  const int x = c % nx, y = (c / nx) % ny, z = c / nxy;
  const int r0 = c - x, p0 = c - y * nx - x;
  const T vc = v[c];
  const T sx = (vc - v[r0 + (x == 0 ? nx - 1 : x - 1)]) + (vc - v[r0 + (x == nx - 1 ? 0 : x + 1)]);
  const T sy = (vc - v[p0 + (y == 0 ? ny - 1 : y - 1) * nx + x]) + (vc - v[p0 + (y == ny - 1 ? 0 : y + 1) * nx + x]);
  T sz = T(0);
  const int xy = y * nx + x;
  int cz = 2;
  if (z > 0) sz += vc - v[c - nxy];
  else if (L.g.periodic_z) sz += vc - v[c + (nz - 1) * nxy];
  else { cz += 2 * (int)L.tlo[xy] - 1; if (L.tlo[xy]) sz += T(2) * vc; }
  if (z < nz - 1) sz += vc - v[c + nxy];
  else if (L.g.periodic_z) sz += vc - v[c - (nz - 1) * nxy];
  else { cz += 2 * (int)L.thi[xy] - 1; if (L.thi[xy]) sz += T(2) * vc; }
  if (L.g.periodic_z) cz = 2;
  inv = T(1) / (T(2) * L.ax + T(2) * L.ay + T(cz) * L.az);
  return L.ax * sx + L.ay * sy + L.az * sz;
}

// The V-cycle below level k0 (all levels small) in one block: per level two
// pre-smoothing sweeps from zero, residual and restriction, the coarsest
// solve, then prolongation and two post-smoothing sweeps, each phase a loop
// over the level's cells followed by a block barrier.  Same operators,
// weights and transfers as the one-kernel-per-phase path above it.  Every
// level's f, e, e_tmp live in shared memory (t.off[k]: offset of level k's
// three arrays, in elements); the first level's f comes from and its e goes
// back to global memory.
template <typename T>
__global__ void __launch_bounds__(MG_MAX_COARSE) k_mg_tail(MgTail<T> t, int singular, Scalars* S) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  __shared__ double ps[MG_MAX_COARSE];
  __shared__ double red[32];
  if (S->done) return;
  T* sm = reinterpret_cast<T*>(tail_smem);
  auto F = [&](int k) { return sm + t.off[k]; };
  auto E = [&](int k) { return sm + t.off[k] + t.lv[k].g.n; };
  auto ET = [&](int k) { return sm + t.off[k] + 2 * t.lv[k].g.n; };
  const T om1 = mg_omega1<T>(), om2 = mg_omega2<T>();
  const int nt = blockDim.x;
  {
    const int n0 = (int)t.lv[0].g.n;
    T* f0 = F(0);
    for (int c = threadIdx.x; c < n0; c += nt) f0[c] = t.lv[0].f[c];
    __syncthreads();
  }
  for (int k = 0; k + 1 < t.nl; ++k) {
    const MgView<T>& L = t.lv[k];
    const MgView<T>& C = t.lv[k + 1];
    T *f = F(k), *e = E(k), *et = ET(k);
    const int n = (int)L.g.n;
    for (int c = threadIdx.x; c < n; c += nt) {
      T inv;
      tail_apply(L, f, c, inv);                        // only the diagonal is needed here
      et[c] = om1 * inv * f[c];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += nt) {
      T inv;
      const T Ae = tail_apply(L, et, c, inv);
      e[c] = et[c] + om2 * inv * (f[c] - Ae);
    }
    __syncthreads();
    const int nc = (int)C.g.n;
    const T scale = T(1) / T(L.fx * L.fy * L.fz);
    T* fc = F(k + 1);
    for (int cc = threadIdx.x; cc < nc; cc += nt) {
      const int X = cc % C.g.nx, Y = (cc / C.g.nx) % C.g.ny, Z = cc / (int)C.g.nxy;
      T acc = T(0);
      for (int dz = 0; dz < L.fz; ++dz)
        for (int dy = 0; dy < L.fy; ++dy)
          for (int dx = 0; dx < L.fx; ++dx) {
            const int c = ((Z * L.fz + dz) * L.g.ny + Y * L.fy + dy) * L.g.nx + X * L.fx + dx;
            T inv;
            acc += f[c] - tail_apply(L, e, c, inv);
          }
      fc[cc] = acc * scale;
    }
    __syncthreads();
  }
  mg_coarse_solve(t.lv[t.nl - 1], F(t.nl - 1), E(t.nl - 1), singular, ps, red);
  __syncthreads();
  for (int k = t.nl - 2; k >= 0; --k) {
    const MgView<T>& L = t.lv[k];
    const MgView<T>& C = t.lv[k + 1];
    T *f = F(k), *e = E(k), *et = ET(k);
    const T* ec = E(k + 1);
    const int n = (int)L.g.n;
    for (int c = threadIdx.x; c < n; c += nt) {
      const int x = c % L.g.nx, y = (c / L.g.nx) % L.g.ny, z = c / (int)L.g.nxy;
      e[c] += ec[((z >> (L.fz - 1)) * C.g.ny + (y >> (L.fy - 1))) * C.g.nx + (x >> (L.fx - 1))];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += nt) {
      T inv;
      const T Ae = tail_apply(L, e, c, inv);
      et[c] = e[c] + om2 * inv * (f[c] - Ae);
    }
    __syncthreads();
    T* eo = k == 0 ? t.lv[0].e : e;                    // the first level's result goes to global memory
    for (int c = threadIdx.x; c < n; c += nt) {
      T inv;
      const T Ae = tail_apply(L, et, c, inv);
      eo[c] = et[c] + om1 * inv * (f[c] - Ae);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- launchers

template <typename K>
static void smem_once(K kernel, size_t bytes, bool& flag) {
  if (!flag) {
    allow_smem(kernel, bytes);
    flag = true;
  }
}

// Grid of a multigrid launch: every tile of the level, at most as many
// blocks as this kernel keeps resident on the GPU (its own occupancy, so the
// lighter sweeps run more blocks per SM than the heavier ones).
template <class K>
static int mg_grid(K kernel, size_t bytes, long long ntiles, int& res) {
  if (res == 0) {
    int dev = 0, nsm = 1, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, MTX * MTY, bytes) != cudaSuccess) nb = 1;
    cudaGetLastError();
    res = std::max(1, nb) * std::max(1, nsm);
  }
  return (int)std::min<long long>(ntiles, std::min(res, MAX_GRID));
}

template <typename T, int VX>
static void pre_v(const LaunchCfg& L, const MgView<T>& lv, Scalars* S) {
  static bool f = false;
  static int res = 0;
  const size_t bytes = MgPipeD0<T, VX>::bytes();
  smem_once(k_mg_pre<T, VX>, bytes, f);
  const int grid = mg_grid(k_mg_pre<T, VX>, bytes, lv.mc.ntiles, res);
  k_mg_pre<T, VX><<<grid, dim3(MTX, MTY), bytes, L.stream>>>(lv, S);
}
template <typename T, int VX>
static void rr_v(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  static bool f = false;
  static int res = 0;
  const size_t bytes = MgPipeD<T, VX>::bytes();
  smem_once(k_mg_rr<T, VX>, bytes, f);
  const int grid = mg_grid(k_mg_rr<T, VX>, bytes, lv.mc.ntiles, res);
  k_mg_rr<T, VX><<<grid, dim3(MTX, MTY), bytes, L.stream>>>(lv, cv, S);
}
template <typename T, int VX>
static void post1_v(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  static bool f = false;
  static int res = 0;
  const size_t bytes = MgPipeP<T, VX>::bytes();
  smem_once(k_mg_post1<T, VX>, bytes, f);
  const int grid = mg_grid(k_mg_post1<T, VX>, bytes, lv.mc.ntiles, res);
  k_mg_post1<T, VX><<<grid, dim3(MTX, MTY), bytes, L.stream>>>(lv, cv, S);
}
template <typename T, bool LAST, int VX>
static void post2_v(const LaunchCfg& L, const MgView<T>& lv, double* part, Scalars* S) {
  static bool f = false;
  static int res = 0;
  const size_t bytes = MgPipeD<T, VX>::bytes();
  smem_once(k_mg_post2<T, LAST, VX>, bytes, f);
  const int grid = mg_grid(k_mg_post2<T, LAST, VX>, bytes, lv.mc.ntiles, res);
  k_mg_post2<T, LAST, VX><<<grid, dim3(MTX, MTY), bytes, L.stream>>>(lv, part, S);
}

constexpr int vec_of(size_t bytes) { return (int)(16 / bytes); }

template <typename T>
void launch_mg_pre(const LaunchCfg& L, const MgView<T>& lv, Scalars* S) {
  if (lv.mc.vx > 1) pre_v<T, vec_of(sizeof(T))>(L, lv, S);
  else pre_v<T, 1>(L, lv, S);
}

template <typename T>
void launch_mg_rr(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  if (lv.mc.vx > 1) rr_v<T, vec_of(sizeof(T))>(L, lv, cv, S);
  else rr_v<T, 1>(L, lv, cv, S);
}

template <typename T>
void launch_mg_coarse(const LaunchCfg& L, const MgView<T>& cv, int singular, Scalars* S) {
  const int threads = ((int)cv.g.n + 31) / 32 * 32;
  k_mg_coarse<T><<<1, threads, 0, L.stream>>>(cv, singular, S);
}

template <typename T>
void launch_mg_post1(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  if (lv.mc.vx > 1) post1_v<T, vec_of(sizeof(T))>(L, lv, cv, S);
  else post1_v<T, 1>(L, lv, cv, S);
}

template <typename T>
void launch_mg_post2(const LaunchCfg& L, const MgView<T>& lv, int last, double* part, Scalars* S) {
  constexpr int V = vec_of(sizeof(T));
  if (last) {
    if (lv.mc.vx > 1) post2_v<T, true, V>(L, lv, part, S);
    else post2_v<T, true, 1>(L, lv, part, S);
  } else {
    if (lv.mc.vx > 1) post2_v<T, false, V>(L, lv, part, S);
    else post2_v<T, false, 1>(L, lv, part, S);
  }
}

template <typename T>
void launch_mg_tail(const LaunchCfg& L, const MgTail<T>& t, int singular, Scalars* S) {
  static bool f = false;
  smem_once(k_mg_tail<T>, MG_TAIL_SMEM, f);
  k_mg_tail<T><<<1, MG_MAX_COARSE, (size_t)t.smem_elems * sizeof(T), L.stream>>>(t, singular, S);
}

template <typename T>
int mg_blocks_per_sm() {
  constexpr int V = vec_of(sizeof(T));
  allow_smem(k_mg_post1<T, V>, MgPipeP<T, V>::bytes());
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mg_post1<T, V>, MTX * MTY, MgPipeP<T, V>::bytes()) !=
      cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

#define PF_MG_INSTANTIATE(T)                                                           \
  template void launch_mg_pre<T>(const LaunchCfg&, const MgView<T>&, Scalars*);                  \
  template void launch_mg_rr<T>(const LaunchCfg&, const MgView<T>&, const MgView<T>&, Scalars*); \
  template void launch_mg_coarse<T>(const LaunchCfg&, const MgView<T>&, int, Scalars*);          \
  template void launch_mg_tail<T>(const LaunchCfg&, const MgTail<T>&, int, Scalars*);            \
  template void launch_mg_post1<T>(const LaunchCfg&, const MgView<T>&, const MgView<T>&, Scalars*); \
  template void launch_mg_post2<T>(const LaunchCfg&, const MgView<T>&, int, double*, Scalars*);        \
  template int mg_blocks_per_sm<T>();

PF_MG_INSTANTIATE(float)
PF_MG_INSTANTIATE(double)

}  // namespace pf
