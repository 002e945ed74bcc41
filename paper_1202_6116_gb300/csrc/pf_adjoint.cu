// Discrete adjoint of one forward-Euler TDGL step (Eq. TDGL with Eqs. F_bulk,
// dF_grad/dP, F_elec, rho and Poisson; Section Time Integration).
//
// The forward step is P' = P + dt L (-f'(P) + g Lap P + E(phi)), with
// A phi = -div P + B(V).  The face rules make the zero-voltage field operator
// E0 the transpose of div, and A and Lap are symmetric, so for a cotangent
// lam = dJ/dP' the transposed step is
//   lam_out = lam + dt L (-H(P) lam + g Lap lam + E0(psi)),  A psi = -div lam,
// H the 3x3 Hessian of the Landau density at each cell.  The adjoint
// potential psi comes from the same right-hand-side and Krylov kernels as the
// forward potential, run with the electrode voltages at zero; this file holds
// the update kernel, which also reduces the step's parameter sensitivities
//   d/da1  : -dt L sum lam . 2P
//   d/da11 : -dt L sum lam . 4P^3
//   d/da12 : -dt L sum lam_i 2P_i (P_j^2 + P_k^2)
//   d/dg   :  dt L sum lam . Lap P  (= dt L sum P . Lap lam, Lap symmetric)
// and, at every electrode face cell, the voltage sensitivity
//   bottom:  dt L (-psi_c 2 eps_c / dx^2 + lam_z,c / dx)
//   top:     dt L (-psi_c 2 eps_c / dx^2 - lam_z,c / dx).
// Algorithmic traffic per cell: reads lam (3), psi (1), P (3); writes lam_out (3).
#include "pf_internal.h"
#include "pf_march.cuh"

namespace pf {

constexpr int ADJ_D = 2;
constexpr int ADJ_NV = 4;

template <typename T, int VX>
using AdjPipe = Pipe<T, void, MTX, MTY, VX, 4, 3, ADJ_D>;

template <typename T>
struct AdjCoef {
  T a1, a11, a12, g, dtL;
};

template <typename T>
struct L3 {
  T x, y, z;
};

template <typename T, int VX>
__global__ void __launch_bounds__(MTX* MTY) k_tdgl_adj(Geo g, Bc<T> bc, const T* __restrict__ lam,
                                                      T* __restrict__ lam_out, const T* __restrict__ psi,
                                                      const T* __restrict__ P, const T* __restrict__ eps,
                                                      AdjCoef<T> k, double* __restrict__ grad,
                                                      double* __restrict__ gv_lo, double* __restrict__ gv_hi,
                                                      double* part, Scalars* S, MarchCfg mc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  const T h = T(0.5), ih = T(g.ih), ih2 = T(g.ih2);
  const T* hsrc[4] = {lam, lam + g.n, lam + 2 * g.n, psi};
  const T* osrc[3] = {P, P + g.n, P + 2 * g.n};
  Acc<T> acc[ADJ_NV];
  TileGeo<MTX, MTY, VX> s{};
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, 4>>& st, const T (&o)[3], const bool bt) -> L3<T> {
    // E0(psi): face values with every electrode at 0 V
    const T fc = st.c.v[3];
    T E[3];
    E[0] = -(h * (fc + st.xp.v[3]) - h * (fc + st.xm.v[3])) * ih;
    E[1] = -(h * (fc + st.yp.v[3]) - h * (fc + st.ym.v[3])) * ih;
    T flo, fhi;
    if (st.zb >= 0) flo = h * (fc + st.zm.v[3]);
    else flo = bc.tlo[xy] ? T(0) : fc;
    if (st.za >= 0) fhi = h * (fc + st.zp.v[3]);
    else fhi = bc.thi[xy] ? T(0) : fc;
    E[2] = -(fhi - flo) * ih;
    const T p[3] = {o[0], o[1], o[2]};
    const T l[3] = {st.c.v[0], st.c.v[1], st.c.v[2]};
    T out[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int j = (i + 1) % 3, m = (i + 2) % 3;
      const T pjk = p[j] * p[j] + p[m] * p[m];
      const T Hl = (T(2) * k.a1 + T(12) * k.a11 * p[i] * p[i] + T(2) * k.a12 * pjk) * l[i] +
                   T(4) * k.a12 * p[i] * (p[j] * l[j] + p[m] * l[m]);
      T lap = T(0);
      lap += st.xm.v[i] - l[i];
      lap += st.xp.v[i] - l[i];
      lap += st.ym.v[i] - l[i];
      lap += st.yp.v[i] - l[i];
      if (st.zb >= 0) lap += st.zm.v[i] - l[i];
      if (st.za >= 0) lap += st.zp.v[i] - l[i];
      lap *= ih2;
      out[i] = l[i] + k.dtL * (-Hl + k.g * lap + E[i]);
      acc[0].add(l[i], T(2) * p[i]);
      acc[1].add(l[i], T(4) * p[i] * p[i] * p[i]);
      acc[2].add(l[i], T(2) * p[i] * pjk);
      acc[3].add(p[i], lap);
    }
    if (bt) {
      const long long c = (long long)z * g.nxy + xy;
      const double dtL = (double)k.dtL;
      const double ec = eps ? (double)eps[c] : 1.0;
      const double qpsi = -(double)fc * 2.0 * ec * g.ih2;
      if (gv_lo && st.zb < 0 && bc.tlo[xy]) gv_lo[xy] += dtL * (qpsi + (double)l[2] * g.ih);
      if (gv_hi && st.za < 0 && bc.thi[xy]) gv_hi[xy] += dtL * (qpsi - (double)l[2] * g.ih);
    }
    return L3<T>{out[0], out[1], out[2]};
  };
  auto post = [&](int z, const L3<T> (&ov)[VX]) {
#pragma unroll
    for (int q = 0; q < ADJ_NV; ++q) acc[q].run();
    const long long c = (long long)z * g.nxy + s.xy;
    T a[VX], b[VX], d[VX];
#pragma unroll
    for (int i = 0; i < VX; ++i) {
      a[i] = ov[i].x;
      b[i] = ov[i].y;
      d[i] = ov[i].z;
    }
    store_n<T, VX>(lam_out + c, a);
    store_n<T, VX>(lam_out + g.n + c, b);
    store_n<T, VX>(lam_out + 2 * g.n + c, d);
  };
  const TileSched ts{&S->sched_next, &S->sched_done, mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(g, t, mc);
#pragma unroll
    for (int q = 0; q < ADJ_NV; ++q) acc[q] = Acc<T>();
    march_direct<T, L3<T>, MTX, MTY, VX, 4, 3, ADJ_D>(g, s, smem, hsrc, osrc, emit, post);
    double v[ADJ_NV];
#pragma unroll
    for (int q = 0; q < ADJ_NV; ++q) v[q] = acc[q].value();
    tile_partials<ADJ_NV, MTX * MTY>(v, part, t);
  }
  sched_finish(ts);
  if (!last_block<MTX * MTY>(&S->ticket)) return;
  double sum[ADJ_NV];
  gather_partials<ADJ_NV, MTX * MTY>(part, mc.ntiles, sum);
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
  const double dtL = (double)k.dtL;
  grad[0] += -dtL * sum[0];
  grad[1] += -dtL * sum[1];
  grad[2] += -dtL * sum[2];
  grad[3] += dtL * sum[3];
  S->ticket = 0;
}

template <typename T, int VX>
static void adj_t(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* lam, T* lam_out, const T* psi,
                  const T* P, const AdjCoef<T>& k, double* grad, double* gv_lo, double* gv_hi) {
  static bool once = false;
  const size_t bytes = AdjPipe<T, VX>::bytes();
  if (!once) {
    allow_smem(k_tdgl_adj<T, VX>, bytes);
    once = true;
  }
  k_tdgl_adj<T, VX><<<L.march.grid, dim3(MTX, MTY), bytes, L.stream>>>(
      g, d.bc, lam, lam_out, psi, P, d.eps, k, grad, gv_lo, gv_hi, d.part, d.S, L.march);
}

template <typename T>
void launch_tdgl_adj(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* lam, T* lam_out, const T* psi,
                     const T* P, const double* coef, double* grad, double* gv_lo, double* gv_hi) {
  const AdjCoef<T> k{T(coef[0]), T(coef[1]), T(coef[2]), T(coef[3]), T(coef[4])};
  constexpr int V = 16 / sizeof(T);
  if (L.march.vx == V) adj_t<T, V>(L, g, d, lam, lam_out, psi, P, k, grad, gv_lo, gv_hi);
  else adj_t<T, 1>(L, g, d, lam, lam_out, psi, P, k, grad, gv_lo, gv_hi);
}

template void launch_tdgl_adj<float>(const LaunchCfg&, const Geo&, const Dev<float>&, const float*, float*,
                                     const float*, const float*, const double*, double*, double*, double*);
template void launch_tdgl_adj<double>(const LaunchCfg&, const Geo&, const Dev<double>&, const double*, double*,
                                      const double*, const double*, const double*, double*, double*, double*);

}  // namespace pf
