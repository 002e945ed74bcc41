// Jacobi-preconditioned CG iteration kernels (the hot loop of every solve).
//
//   k_cg_p  p_new = r/diag + beta p_old (formed on the fly, halo included),
//           q = A p_new, deferred x += alpha_prev p_old, partial p_new.q;
//           the last block turns p.q into alpha.            (2.5-D plane march)
//   k_cg_r  r -= alpha q, partial r.r and r.z (z = r/diag);  the last block
//           decides convergence and forms beta.              (flat, 16-byte vectors)
//
// Algorithmic traffic per iteration and cell: k_cg_p reads r, p_old, x and
// writes p_new, q, x (6 words); k_cg_r reads r, q and writes r (3 words).
#include "pf_internal.h"
#include "pf_march.cuh"

namespace pf {

constexpr int CG_D = 2;   // planes of cp.async look-ahead in k_cg_p
constexpr int CGD_D = 3;  // the same for its direct (multigrid) forms, whose stages are smaller

template <typename T, bool EPS, int VX>
using CgPipe = Pipe<T, typename FieldOf<T, EPS>::type, MTX, MTY, VX, EPS ? 4 : 2, 1, CG_D>;

// MG = false: z = r/diag (Jacobi), r is the staged input.  MG = true: z comes
// from the V-cycle and is the staged input.
// DIRECT (multigrid, eps = 1): the stencil of p = z + beta p_old is formed
// from the staged planes of z and p_old at each of the seven cells (no field
// buffer); otherwise p goes through the march's shared field buffer.
// FIRST (direct form, launched for a solve's first iteration only): p = z,
// and neither p_old nor x is read (1 word read, 2 written per cell).
// SECOND (direct form, launched for a compensated solve's second iteration
// only): the correction x is still 0, so the deferred update writes alpha
// p_old without staging or reading x (2 words read, 3 written per cell).
template <typename T, bool EPS, bool MG, int VX, bool DIRECT = false, bool FIRST = false, bool SECOND = false>
__global__ void __launch_bounds__(MTX* MTY, (sizeof(T) == 4 && !EPS) ? 3 : 2) k_cg_p(Geo g, Bc<T> bc, const T* __restrict__ eps,
                                                  const T* __restrict__ invd, const T* __restrict__ r, T* p0,
                                                  T* p1, T* __restrict__ q, T* __restrict__ x, double* part,
                                                  Scalars* S, MarchCfg mc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  using F = typename FieldOf<T, EPS>::type;
  constexpr int NH = EPS ? 4 : 2;          // r or z, p_old (, eps, 1/diag) with halo
  static_assert(!FIRST || DIRECT, "the first-iteration form is the direct one");
  static_assert(!SECOND || (DIRECT && !FIRST), "the second-iteration form is the direct one");
  if (S->done) return;
  const int first = FIRST ? 1 : S->first;
  // x still 0 (the correction of a compensated start, not written yet): the
  // deferred update writes alpha p_old and ignores the staged x
  const int xz = SECOND ? 1 : S->xzero;
  const T beta = first ? T(0) : T(S->beta);
  const T alpha = T(S->alpha);
  const int pb = S->pbuf;
  const T* pold = pb ? p1 : p0;
  T* __restrict__ pnew = pb ? p0 : p1;
  const T inv6 = T(1) / (T(6) * T(g.ih2));
  const T ih2 = T(g.ih2);
  Acc<T> apq;
  const T* hsrc[NH];
  hsrc[0] = r;
  hsrc[1] = pold;
  if constexpr (EPS) {
    hsrc[2] = eps;
    hsrc[3] = invd;
  }
  const T* osrc[1] = {x};
  struct Out {
    T x, p, q;
  };
  TileGeo<MTX, MTY, VX> s;

  auto val = [&](const T (&h)[NH], int xy, int z, int, int, const bool bt) -> F {
    T zz;
    if constexpr (MG) {
      zz = h[0];
    } else {
      T inv;
      if constexpr (EPS) inv = h[3];
      else inv = bt ? inv_diag_unit(g, bc, xy, z, inv6) : inv6;
      zz = h[0] * inv;
    }
    const T v = first ? zz : zz + beta * h[1];
    if constexpr (EPS) return F{v, h[2]};
    else return v;
  };
  auto emit = [&](int xy, int, const Stencil7<F>& st, const T (&h)[NH], const T (&o)[1], const bool bt) -> Out {
    const bool B = bt;
    const int dlo = (B && st.zb < 0) ? (int)bc.tlo[xy] : 0;
    const int dhi = (B && st.za < 0) ? (int)bc.thi[xy] : 0;
    const T qv = apply_bt(st, dlo, dhi, ih2, bt);
    const T pc = field_value<T>(st.c);
    apq.add(pc, qv);
    return Out{first ? o[0] : (xz ? alpha * h[1] : o[0] + alpha * h[1]), pc, qv};
  };
  auto post = [&](int z, const Out (&ov)[VX]) {
    apq.run();
    const long long c = (long long)z * g.nxy + s.xy;
    T xs[VX], ps[VX], qs[VX];
#pragma unroll
    for (int i = 0; i < VX; ++i) {
      xs[i] = ov[i].x;
      ps[i] = ov[i].p;
      qs[i] = ov[i].q;
    }
    if (!first) store_n<T, VX>(x + c, xs);
    store_n<T, VX>(pnew + c, ps);
    store_n<T, VX>(q + c, qs);
  };
  // direct form: p at a cell from the raw (z, p_old) pair
  auto pval = [&](const Raw<T, NH>& rw) -> T { return first ? rw.v[0] : rw.v[0] + beta * rw.v[1]; };
  auto emit_d = [&](int xy, int, const Stencil7<Raw<T, NH>>& sr, const T (&o)[1], const bool bt) -> Out {
    Stencil7<T> st;
    st.c = pval(sr.c);
    st.xm = pval(sr.xm);
    st.xp = pval(sr.xp);
    st.ym = pval(sr.ym);
    st.yp = pval(sr.yp);
    st.zm = pval(sr.zm);
    st.zp = pval(sr.zp);
    st.zb = sr.zb;
    st.za = sr.za;
    const bool B = bt;
    const int dlo = (B && st.zb < 0) ? (int)bc.tlo[xy] : 0;
    const int dhi = (B && st.za < 0) ? (int)bc.thi[xy] : 0;
    const T qv = apply_bt(st, dlo, dhi, ih2, bt);
    apq.add(st.c, qv);
    return Out{first ? o[0] : (xz ? alpha * sr.c.v[1] : o[0] + alpha * sr.c.v[1]), st.c, qv};
  };
  const TileSched ts{&S->sched_next, &S->sched_done, mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(g, t, mc);
    apq = Acc<T>();
    if constexpr (DIRECT && FIRST) {
      const T* const hs1[1] = {r};
      const T* const os1[1] = {nullptr};
      auto emit_f = [&](int xy, int, const Stencil7<Raw<T, 1>>& sr, const T (&)[1], const bool bt) -> Out {
        Stencil7<T> st = pick(sr, 0);
        const bool B = bt;
        const int dlo = (B && st.zb < 0) ? (int)bc.tlo[xy] : 0;
        const int dhi = (B && st.za < 0) ? (int)bc.thi[xy] : 0;
        const T qv = apply_bt(st, dlo, dhi, ih2, bt);
        apq.add(st.c, qv);
        return Out{T(0), st.c, qv};
      };
      march_direct<T, Out, MTX, MTY, VX, 1, 0, CGD_D>(g, s, smem, hs1, os1, emit_f, post);
    } else if constexpr (DIRECT) {
      static_assert(MG && !EPS, "the direct form is the multigrid search direction with eps = 1");
      if constexpr (SECOND) {          // x is not read: stage z and p_old alone
        const T* const os0[1] = {nullptr};
        march_direct<T, Out, MTX, MTY, VX, NH, 0, CGD_D>(g, s, smem, hsrc, os0, emit_d, post);
      } else {
        march_direct<T, Out, MTX, MTY, VX, NH, 1, CGD_D>(g, s, smem, hsrc, osrc, emit_d, post);
      }
    } else {
      march<T, F, Out, MTX, MTY, VX, NH, 1, CG_D>(g, s, smem, hsrc, osrc, val, emit, post);
    }
    double v[1] = {apq.value()};
    tile_partials<1, MTX * MTY>(v, part, t);
  }
  sched_finish(ts);
  if (last_block<MTX * MTY>(&S->ticket)) {
    double out[1];
    gather_partials<1, MTX * MTY>(part, mc.ntiles, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const double pq = out[0];
      S->pq = pq;
      S->iter += 1;
      S->pbuf = pb ^ 1;
      if (!first) S->xzero = 0;        // this launch wrote x
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

template <typename T, bool EPS, bool MG>
__global__ void __launch_bounds__(FLAT_THREADS) k_cg_r(Geo g, Bc<T> bc, const T* __restrict__ invd,
                                                      T* __restrict__ r, const T* __restrict__ q, double* part,
                                                      Scalars* S, cudaGraphConditionalHandle cond, int use_cond) {
  if (S->done) {
    // In a graph loop the condition must drop whatever finished the solve
    // (a breakdown in k_cg_p, a non-finite r.z in the V-cycle): every pass
    // of the loop body either counts an iteration or ends the loop.
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  using V = typename Vec16<T>::type;
  constexpr int NV = 16 / sizeof(T);
  const T alpha = T(S->alpha);
  const T inv6 = T(1) / (T(6) * T(g.ih2));
  Acc<T> arr, arz;
  const long long nvec = g.n / NV;
  const long long stride = (long long)gridDim.x * FLAT_THREADS;
  int cnt = 0;
  auto one = [&](long long e, T& rv, T qv) {
    rv = rv - alpha * qv;
    arr.add(rv, rv);
    if (!MG) arz.add(rv, rv * (EPS ? invd[e] : inv_flat(g, bc, e, inv6)));
  };
  for (long long i = blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; i < nvec; i += stride) {
    V rv = reinterpret_cast<const V*>(r)[i];
    const V qv = reinterpret_cast<const V*>(q)[i];
    T* rs = reinterpret_cast<T*>(&rv);
    const T* qs = reinterpret_cast<const T*>(&qv);
#pragma unroll
    for (int k = 0; k < NV; ++k) one(i * NV + k, rs[k], qs[k]);
    reinterpret_cast<V*>(r)[i] = rv;
    arr.run();
    arz.run();
    if (++cnt == 16) {
      arr.flush();
      arz.flush();
      cnt = 0;
    }
  }
  for (long long e = nvec * NV + blockIdx.x * (long long)FLAT_THREADS + threadIdx.x; e < g.n; e += stride) {
    T rv = r[e];
    one(e, rv, q[e]);
    r[e] = rv;
  }
  arr.flush();
  arz.flush();
  double v[2] = {arr.value(), arz.value()};
  if (publish_partials<2, FLAT_THREADS>(v, part, &S->ticket)) {
    double out[2];
    gather_partials<2, FLAT_THREADS>(part, gridDim.x, out);
    if (threadIdx.x == 0) {
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
      } else if (!MG) {
        S->beta = rz / S->rz;
        S->rz = rz;
      }
      S->ticket = 0;
      if (use_cond) cudaGraphSetConditional(cond, S->done ? 0u : 1u);
    }
  }
}

template <typename T, bool EPS, bool MG, int VX, bool FIRST, bool SECOND>
static void launch_cg_p_t(const LaunchCfg& L, const Geo& g, const Dev<T>& d) {
  constexpr bool DIRECT = MG && !EPS;
  using PD = Pipe<T, void, MTX, MTY, VX, FIRST ? 1 : 2, (FIRST || SECOND) ? 0 : 1, CGD_D>;
  const size_t bytes = DIRECT ? PD::bytes() : CgPipe<T, EPS, VX>::bytes();
  static bool once = false;
  if (!once) {
    allow_smem(k_cg_p<T, EPS, MG, VX, DIRECT, FIRST, SECOND>, bytes);
    once = true;
  }
  k_cg_p<T, EPS, MG, VX, DIRECT, FIRST, SECOND><<<L.march.grid, dim3(MTX, MTY), bytes, L.stream>>>(
      g, d.bc, d.eps, d.invd, MG ? d.z : d.r, d.p0, d.p1, d.q, d.phi, d.part, d.S, L.march);
}

template <typename T, bool EPS, bool MG, bool FIRST = false, bool SECOND = false>
static void launch_cg_p_v(const LaunchCfg& L, const Geo& g, const Dev<T>& d) {
  constexpr int V = 16 / sizeof(T);
  if (L.march.vx == V) launch_cg_p_t<T, EPS, MG, V, FIRST, SECOND>(L, g, d);
  else launch_cg_p_t<T, EPS, MG, 1, FIRST, SECOND>(L, g, d);
}

template <typename T>
void launch_cg_p(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int mg, int first, int second) {
  // with a permittivity field the multigrid form stages eps too (field-buffer
  // march; its first iteration reads the first-iteration flag of the solver)
  if (mg && d.eps) launch_cg_p_v<T, true, true>(L, g, d);
  else if (mg && first) launch_cg_p_v<T, false, true, true>(L, g, d);
  else if (mg && second) launch_cg_p_v<T, false, true, false, true>(L, g, d);
  else if (mg) launch_cg_p_v<T, false, true>(L, g, d);
  else if (d.eps) launch_cg_p_v<T, true, false>(L, g, d);
  else launch_cg_p_v<T, false, false>(L, g, d);
}

template <typename T>
void launch_cg_r(const LaunchCfg& L, const Geo& g, const Dev<T>& d, int mg, cudaGraphConditionalHandle cond,
                 int use_cond) {
  if (mg)
    k_cg_r<T, false, true><<<L.flat_grid, FLAT_THREADS, 0, L.stream>>>(g, d.bc, d.invd, d.r, d.q, d.part, d.S,
                                                                        cond, use_cond);
  else if (d.eps)
    k_cg_r<T, true, false><<<L.flat_grid, FLAT_THREADS, 0, L.stream>>>(g, d.bc, d.invd, d.r, d.q, d.part, d.S,
                                                                        cond, use_cond);
  else
    k_cg_r<T, false, false><<<L.flat_grid, FLAT_THREADS, 0, L.stream>>>(g, d.bc, d.invd, d.r, d.q, d.part, d.S,
                                                                         cond, use_cond);
}

template <typename T, bool EPS, int VX>
static int occ_cg_p() {
  const size_t bytes = CgPipe<T, EPS, VX>::bytes();
  allow_smem(k_cg_p<T, EPS, false, VX>, bytes);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_p<T, EPS, false, VX>, MTX * MTY, bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

int march_blocks_per_sm(int fp32, int eps) {
  if (fp32) return eps ? occ_cg_p<float, true, 4>() : occ_cg_p<float, false, 4>();
  return eps ? occ_cg_p<double, true, 2>() : occ_cg_p<double, false, 2>();
}

template void launch_cg_p<float>(const LaunchCfg&, const Geo&, const Dev<float>&, int, int, int);
template void launch_cg_p<double>(const LaunchCfg&, const Geo&, const Dev<double>&, int, int, int);
template void launch_cg_r<float>(const LaunchCfg&, const Geo&, const Dev<float>&, int, cudaGraphConditionalHandle,
                                 int);
template void launch_cg_r<double>(const LaunchCfg&, const Geo&, const Dev<double>&, int,
                                  cudaGraphConditionalHandle, int);

}  // namespace pf
