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
  auto post = [&](int, const T (&)[VX]) {};
  const TileSched ts{&S->sched_next, &S->sched_done};
  for (long long t = sched_take(ts, &tile_slot); t < mc.ntiles; t = sched_take(ts, &tile_slot)) {
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

}  // namespace pf
