// Run diagnostics of the current state (P, phi) in one plane-march pass:
//   mean P (the polarization of P-V loops), the fraction of cells with
//   P_x > threshold (switched domains), the Landau energy sum f(P)
//   (Eq. F_bulk), the gradient energy (g/2) sum over interior faces
//   |P_nb - P_c|^2 / dx^2 (Eq. F_grad) and -1/2 sum P . E(phi) with E from
//   face values and the face voltages (Eq. F_elec).
// Every cell adds its +x, +y and +z faces to the gradient energy (the +z face
// only where it is interior or periodic), so each face counts once.
// Sums: per-tile partials gathered in a fixed order; FP32 terms go through
// the compensated accumulator.  Traffic per cell: reads 4 words, writes none.
#include "pf_internal.h"
#include "pf_march.cuh"

namespace pf {

constexpr int DIAG_D = 2;
constexpr int DIAG_NV = 7;

template <typename T, int VX>
using DiagPipe = Pipe<T, void, MTX, MTY, VX, 4, 0, DIAG_D>;

template <typename T>
struct DiagCoef {
  T a1, a11, a12;
  double thr;          // compared with P_x in FP64
};

template <typename T, int VX>
__global__ void __launch_bounds__(MTX* MTY) k_diag(Geo g, Bc<T> bc, const T* __restrict__ P,
                                                  const T* __restrict__ phi, DiagCoef<T> k, double* out,
                                                  double* part, Scalars* S, MarchCfg mc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  const T h = T(0.5), ih = T(g.ih);
  const T* hsrc[4] = {P, P + g.n, P + 2 * g.n, phi};
  const T* osrc[1] = {nullptr};
  Acc<T> acc[DIAG_NV];
  TileGeo<MTX, MTY, VX> s{};
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, 4>>& st, const T (&)[1], bool) -> T {
    const T fc = st.c.v[3];
    T E[3];
    E[0] = -(h * (fc + st.xp.v[3]) - h * (fc + st.xm.v[3])) * ih;
    E[1] = -(h * (fc + st.yp.v[3]) - h * (fc + st.ym.v[3])) * ih;
    T flo, fhi;
    if (st.zb >= 0) flo = h * (fc + st.zm.v[3]);
    else flo = bc.tlo[xy] ? bc.vlo[xy] : fc;
    if (st.za >= 0) fhi = h * (fc + st.zp.v[3]);
    else fhi = bc.thi[xy] ? bc.vhi[xy] : fc;
    E[2] = -(fhi - flo) * ih;
    const T p[3] = {st.c.v[0], st.c.v[1], st.c.v[2]};
    const T x2 = p[0] * p[0], y2 = p[1] * p[1], z2 = p[2] * p[2];
    acc[0].add(p[0], T(1));
    acc[1].add(p[1], T(1));
    acc[2].add(p[2], T(1));
    acc[3].add((double)p[0] > k.thr ? T(1) : T(0), T(1));
    acc[4].add(k.a1, x2 + y2 + z2);
    acc[4].add(k.a11, x2 * x2 + y2 * y2 + z2 * z2);
    acc[4].add(k.a12, x2 * y2 + y2 * z2 + z2 * x2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T dxp = st.xp.v[i] - p[i], dyp = st.yp.v[i] - p[i];
      acc[5].add(dxp, dxp);
      acc[5].add(dyp, dyp);
      if (st.za >= 0 && (z + 1 < g.zair || g.zair == g.nz)) {     // no wall energy across the film/air face
        const T dzp = st.zp.v[i] - p[i];
        acc[5].add(dzp, dzp);
      }
      acc[6].add(p[i], E[i]);
    }
    return T(0);
  };
  auto post = [&](int, const T (&)[VX]) {
#pragma unroll
    for (int q = 0; q < DIAG_NV; ++q) acc[q].run();
  };
  const TileSched ts{&S->sched_next, &S->sched_done, mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(g, t, mc);
#pragma unroll
    for (int q = 0; q < DIAG_NV; ++q) acc[q] = Acc<T>();
    march_direct<T, T, MTX, MTY, VX, 4, 0, DIAG_D>(g, s, smem, hsrc, osrc, emit, post);
    double v[DIAG_NV];
#pragma unroll
    for (int q = 0; q < DIAG_NV; ++q) v[q] = acc[q].value();
    tile_partials<DIAG_NV, MTX * MTY>(v, part, t);
  }
  sched_finish(ts);
  if (!last_block<MTX * MTY>(&S->ticket)) return;
  double sum[DIAG_NV];
  gather_partials<DIAG_NV, MTX * MTY>(part, mc.ntiles, sum);
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
#pragma unroll
  for (int q = 0; q < DIAG_NV; ++q) out[q] = sum[q];
  S->ticket = 0;
}

template <typename T, int VX>
static void diag_t(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, const DiagCoef<T>& k,
                   double* out) {
  static bool once = false;
  const size_t bytes = DiagPipe<T, VX>::bytes();
  if (!once) {
    allow_smem(k_diag<T, VX>, bytes);
    once = true;
  }
  k_diag<T, VX><<<L.march.grid, dim3(MTX, MTY), bytes, L.stream>>>(g, d.bc, P, d.phi, k, out, d.part, d.S,
                                                                   L.march);
}

template <typename T>
void launch_diag(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, const double* coef, double* out) {
  const DiagCoef<T> k{T(coef[0]), T(coef[1]), T(coef[2]), coef[3]};
  constexpr int V = 16 / sizeof(T);
  if (L.march.vx == V) diag_t<T, V>(L, g, d, P, k, out);
  else diag_t<T, 1>(L, g, d, P, k, out);
}

template void launch_diag<float>(const LaunchCfg&, const Geo&, const Dev<float>&, const float*, const double*,
                                 double*);
template void launch_diag<double>(const LaunchCfg&, const Geo&, const Dev<double>&, const double*, const double*,
                                  double*);

// ------------------------------------------------------------ true residual
//
// ||b(P) - A phi||_2^2 and ||b(P)||_2^2 of a stored state, every operation in
// FP64 whatever the storage precision.  The Krylov loop stops on its
// recursive residual; this is the residual of the potential actually stored
// (in FP32 mode, after rounding to FP32).  b and A follow the face rules of k_rhs and
// apply_field (Eqs. rho, Poisson: face values of P are the mean inside, P_cell
// at an electrode, 0 at an open face; Dirichlet faces add 2 eps_c (phi_c - V)
// / dx^2, open faces nothing; interior face permittivity is the harmonic mean).
// Singular problems (no electrode) use b - mean(b), the system the solver
// solves: MEAN = true sums b alone.  One thread per cell, neighbours read from
// global memory (a diagnostic, not on the hot path).
// An FP32 time series also keeps the part of the last solution that the
// stored phi cannot hold (see k_cg_finish_comp: after solve k the remainder
// buffer holds that part plus the next start's increment c_{k+1}, which sits
// in ring slot (k + 1) mod 3).  With cp.lo set, the third sum is the residual
// of that compensated potential phi + (lo - c_{k+1}), formed in FP64.
template <typename T, bool EPS, bool MEAN>
__global__ void __launch_bounds__(256) k_true_res(Geo g, Bc<T> bc, const T* __restrict__ P, const T* __restrict__ phi,
                                                  const T* __restrict__ eps, Comp<T> cp, double mb, double* part,
                                                  unsigned* ticket, double* out) {
  constexpr int NV = MEAN ? 1 : 3;
  const long long ks = cp.lo ? *cp.nsolve : 0;
  const T* cn = ks >= 1 ? cp.ring[ks % 3] : nullptr;
  auto phic = [&](long long c) -> double {
    const double v = (double)phi[c];
    return cn ? v + ((double)cp.lo[c] - (double)cn[c]) : v;
  };
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const double ih = g.ih, ih2 = g.ih2;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.n; c += stride) {
    const int x = (int)(c % g.nx);
    const int y = (int)((c / g.nx) % g.ny);
    const int z = (int)(c / g.nxy);
    const long long xy = (long long)y * g.nx + x;
    const long long zo = c - xy;
    const long long nb[6] = {zo + (long long)y * g.nx + (x == 0 ? g.nx - 1 : x - 1),
                             zo + (long long)y * g.nx + (x == g.nx - 1 ? 0 : x + 1),
                             zo + (long long)(y == 0 ? g.ny - 1 : y - 1) * g.nx + x,
                             zo + (long long)(y == g.ny - 1 ? 0 : y + 1) * g.nx + x,
                             z > 0 ? c - g.nxy : (g.periodic_z ? c + (long long)(g.nz - 1) * g.nxy : -1),
                             z < g.nz - 1 ? c + g.nxy : (g.periodic_z ? c - (long long)(g.nz - 1) * g.nxy : -1)};
    const int dlo = nb[4] < 0 ? (int)bc.tlo[xy] : 0;
    const int dhi = nb[5] < 0 ? (int)bc.thi[xy] : 0;
    const double ec = EPS ? (double)eps[c] : 1.0;
    // b = -div P + Dirichlet terms, faces in the order x-, x+, y-, y+, z-, z+
    double div = 0.0;
    for (int a = 0; a < 3; ++a) {
      const T* Pa = P + a * g.n;
      const double pc = (double)Pa[c];
      const long long m = nb[2 * a], p = nb[2 * a + 1];
      double fm, fp;
      if (m >= 0) fm = 0.5 * (pc + (double)Pa[m]);
      else fm = dlo ? pc : 0.0;
      if (p >= 0) fp = 0.5 * (pc + (double)Pa[p]);
      else fp = dhi ? pc : 0.0;
      div += fp - fm;
    }
    double b = -div * ih - mb;
    if (dlo) b += 2.0 * ec * (double)bc.vlo[xy] * ih2;
    if (dhi) b += 2.0 * ec * (double)bc.vhi[xy] * ih2;
    if (MEAN) {
      acc[0] += b;
      continue;
    }
    const double fc = (double)phi[c], gc = phic(c);
    double Af = 0.0, Ag = 0.0;
    for (int f = 0; f < 6; ++f) {
      if (nb[f] >= 0) {
        const double en = EPS ? (double)eps[nb[f]] : 1.0;
        const double ef = EPS ? 2.0 * ec * en / (ec + en) : 1.0;
        Af += ef * (fc - (double)phi[nb[f]]);
        Ag += ef * (gc - phic(nb[f]));
      } else if ((f == 4 && dlo) || (f == 5 && dhi)) {
        Af += 2.0 * ec * fc;
        Ag += 2.0 * ec * gc;
      }
    }
    const double r = b - Af * ih2, rg = b - Ag * ih2;
    acc[0] += r * r;
    acc[1] += b * b;
    acc[NV - 1] += rg * rg;
  }
  if (!publish_partials<NV, 256>(acc, part, ticket)) return;
  double sum[NV];
  gather_partials<NV, 256>(part, gridDim.x, sum);
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = sum[k];
  *ticket = 0;
}

template <typename T, bool EPS>
static void true_res_t(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, int singular, double* out) {
  const int grid = std::max(1, std::min(L.flat_grid, MAX_GRID));
  double mb = 0.0;
  if (singular) {
    k_true_res<T, EPS, true><<<grid, 256, 0, L.stream>>>(g, d.bc, P, d.phi, d.eps, d.cp, 0.0, d.part, &d.S->ticket,
                                                         out);
    // the mean of b is read back by the host between the passes (a diagnostic)
    double sb = 0.0;
    if (cudaMemcpyAsync(&sb, out, sizeof(double), cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
        cudaStreamSynchronize(L.stream) != cudaSuccess)
      return;
    mb = sb / (double)g.n;
  }
  k_true_res<T, EPS, false><<<grid, 256, 0, L.stream>>>(g, d.bc, P, d.phi, d.eps, d.cp, mb, d.part, &d.S->ticket,
                                                        out);
}

template <typename T>
void launch_true_residual(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, int singular, double* out) {
  if (d.eps) true_res_t<T, true>(L, g, d, P, singular, out);
  else true_res_t<T, false>(L, g, d, P, singular, out);
}

template void launch_true_residual<float>(const LaunchCfg&, const Geo&, const Dev<float>&, const float*, int, double*);
template void launch_true_residual<double>(const LaunchCfg&, const Geo&, const Dev<double>&, const double*, int,
                                           double*);

}  // namespace pf
