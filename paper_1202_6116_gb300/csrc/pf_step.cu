// Once-per-step kernels on the plane march: the Poisson right-hand side with
// the warm-start residual, and the forward-Euler TDGL update.
//
//   k_rhs   b = -div P + (Dirichlet terms) (Eqs. rho, Poisson; face values of P:
//           mean inside, P_cell at an electrode, 0 at an open face), the warm
//           start residual r0 = b - A phi (Section Numerical Performance), and
//           ||b||^2, ||r||^2, r.z.  An FP32 time series starts from the
//           compensated pair phi + s (r0 = b - A phi - A s, see
//           k_cg_finish_comp).  With MEAN = true it only sums b (the
//           zero-mean projection of singular problems).
//   k_tdgl  P' = P + dt L (-df/dP + g Lap P + E), E = -grad phi from face values
//           (Eq. TDGL with Eqs. F_bulk, dF_grad/dP, F_elec; Section Time Integration).
//           Planes z >= zair are air: P = 0 there, and the film's top plane has
//           no z+ neighbour in the Laplacian (free surface).
//           COMP = true (FP32 forward Euler): the state is the compensated
//           pair P + P_lo, P_lo the part of the exact sum that the FP32 P
//           cannot hold (own cells only, updated in place, stored as bf16:
//           it is at most half an FP32 ulp of P, so its 8-bit significand
//           still resolves increments down to about 2^-10 ulp of P).  The
//           increment dt R is added to the pair by TwoSum, so increments far
//           below half an FP32 ulp of P still accumulate instead of being
//           rounded away step after step.
//           CORR = true is the corrector of the predictor-corrector scheme: P is
//           the predicted state P^p, and the output overwrites the state P_n it
//           started from with (P_n + P^p + dt R(P^p)) / 2 = P_n + dt (R(P_n) +
//           R(P^p)) / 2 (each thread reads its own cells of P_n before writing).
//
// Both read P (3 components) and phi with their 6 neighbours; the neighbours
// come straight from the staged planes (march_direct).  Algorithmic traffic
// per cell: k_rhs reads 4 words (5 with a compensated start) and writes 1;
// k_tdgl reads 4 and writes 3 (compensated state: plus 3 half-words each way).
// An FP32 time series on whole 64 x 16 tiles runs k_rhs_w and k_tdgl_w: the
// same arithmetic on their own staging (each field with only the neighbours
// its term reads, halo copies spread over the block).
#include <cuda_bf16.h>

#include "pf_internal.h"
#include "pf_march.cuh"
#include "pf_rng.cuh"

namespace pf {

constexpr int STEP_D = 2;

// X: extra staged fields (the remainder of a compensated potential)
template <typename T, bool EPS, int VX, int X = 0>
using StepPipe = Pipe<T, void, MTX, MTY, VX, (EPS ? 5 : 4) + X, EPS ? 1 : 0, STEP_D>;

// Face values of P along the face normal (reading of the boundary kinds).
// Between two interior cells the face values (P_c + P_n)/2 of a component
// cancel their P_c: the pair of faces normal to x adds (P_x+ - P_x-)/2, which
// is formed directly (fewer operations and no rounding of P_c + P_n).
template <typename T, int NH>
__device__ __forceinline__ T divergence(const Stencil7<Raw<T, NH>>& s, int dlo, int dhi) {
  const T h = T(0.5);
  const T pzc = s.c.v[2];
  T div = h * (s.xp.v[0] - s.xm.v[0]);
  div += h * (s.yp.v[1] - s.ym.v[1]);
  if (s.zb >= 0 && s.za >= 0) return div + h * (s.zp.v[2] - s.zm.v[2]);
  if (s.zb >= 0) div += -(h * (pzc + s.zm.v[2]));
  else if (dlo) div += -pzc;
  if (s.za >= 0) div += h * (pzc + s.zp.v[2]);
  else if (dhi) div += pzc;
  return div;
}

// The last block to finish sums the tiles' partials in tile order and starts
// the solve: ||b||^2, ||r||^2 and r.z of the warm residual, the convergence
// test of the start (or, MEAN, the mean of b).  Called by every thread.
template <int NV, bool MEAN, bool COMP>
__device__ __forceinline__ void rhs_close(const Geo& g, double* part, Scalars* S, long long ntiles,
                                          cudaGraphConditionalHandle cond, int use_cond) {
  if (!last_block<MTX * MTY>(&S->ticket)) return;
  double out[NV];
  gather_partials<NV, MTX * MTY>(part, ntiles, out);
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
  if (MEAN) {
    S->mean_b = out[0] / (double)g.n;
    S->ticket = 0;
    return;
  }
  const double bb = out[0], rr = out[NV > 1 ? 1 : 0], rz = out[NV > 2 ? 2 : 0];
  S->bb = bb;
  S->rr = rr;
  S->rz = rz;
  S->iter = 0;
  S->first = 1;
  S->pending = 0;
  S->xzero = COMP ? 1 : 0;            // a compensated start's correction begins at 0, unwritten
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

// COMP: the start is the compensated pair phi + s (r0 = b - A phi - A s).
template <typename T, bool EPS, bool MEAN, int VX, bool COMP = false>
__global__ void __launch_bounds__(MTX* MTY) k_rhs(Geo g, Bc<T> bc, const T* __restrict__ P, const T* __restrict__ phi,
                                                 const T* __restrict__ lo, const T* __restrict__ eps,
                                                 const T* __restrict__ invd, T* __restrict__ r, double* part,
                                                 Scalars* S, MarchCfg mc, cudaGraphConditionalHandle cond,
                                                 int use_cond) {
  static_assert(!(COMP && MEAN), "the mean of b needs no start");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  constexpr int NH = (EPS ? 5 : 4) + (COMP ? 1 : 0);   // Px, Py, Pz, phi (, lo) (, eps)
  constexpr int IE = NH - 1;                           // eps, when staged
  constexpr int NO = EPS ? 1 : 0;     // (1/diag)
  constexpr int NV = MEAN ? 1 : 3;
  const T mb = MEAN ? T(0) : T(S->mean_b);
  const T inv6 = T(1) / (T(6) * T(g.ih2));
  const T ih = T(g.ih), ih2 = T(g.ih2);
  const T* hsrc[NH];
  hsrc[0] = P;
  hsrc[1] = P + g.n;
  hsrc[2] = P + 2 * g.n;
  hsrc[3] = phi;
  if constexpr (COMP) hsrc[4] = lo;
  if constexpr (EPS) hsrc[IE] = eps;
  const T* osrc[1] = {invd};
  Acc<T> abb, arr, arz;
  TileGeo<MTX, MTY, VX> s;
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, NH>>& st, const T (&o)[NO > 0 ? NO : 1], const bool bt) -> T {
    const bool B = bt;
    const int dlo = (B && st.zb < 0) ? (int)bc.tlo[xy] : 0;
    const int dhi = (B && st.za < 0) ? (int)bc.thi[xy] : 0;
    const T ec = EPS ? st.c.v[IE] : T(1);
    T dir = T(0);
    if (dlo) dir += T(2) * ec * bc.vlo[xy];
    if (dhi) dir += T(2) * ec * bc.vhi[xy];
    const T b = -divergence(st, dlo, dhi) * ih + dir * ih2 - mb;
    if (MEAN) {
      abb.add(b, T(1));
      return T(0);
    }
    auto Aof = [&](int i) -> T {
      if constexpr (EPS) {
        Stencil7<EpsVal<T>> se;
        auto ev = [&](const Raw<T, NH>& rw) { return EpsVal<T>{rw.v[i], rw.v[IE]}; };
        se.c = ev(st.c);
        se.xm = ev(st.xm);
        se.xp = ev(st.xp);
        se.ym = ev(st.ym);
        se.yp = ev(st.yp);
        se.zm = ev(st.zm);
        se.zp = ev(st.zp);
        se.zb = st.zb;
        se.za = st.za;
        return apply_bt(se, dlo, dhi, ih2, bt);
      } else {
        return apply_bt(pick(st, i), dlo, dhi, ih2, bt);
      }
    };
    T rv = b - Aof(3);
    if constexpr (COMP) rv -= Aof(4);
    T inv;
    if constexpr (EPS) inv = o[0];
    else inv = B ? inv_diag_unit(g, bc, xy, z, inv6) : inv6;
    abb.add(b, b);
    arr.add(rv, rv);
    arz.add(rv, rv * inv);
    return rv;
  };
  auto post = [&](int z, const T (&ov)[VX]) {
    abb.run();
    if (!MEAN) {
      arr.run();
      arz.run();
      store_n<T, VX>(r + (long long)z * g.nxy + s.xy, ov);
    }
  };
  const TileSched ts{&S->sched_next, &S->sched_done, mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(g, t, mc);
    abb = Acc<T>();
    arr = Acc<T>();
    arz = Acc<T>();
    march_direct<T, T, MTX, MTY, VX, NH, NO, STEP_D>(g, s, smem, hsrc, osrc, emit, post);
    double v[3] = {abb.value(), arr.value(), arz.value()};
    double (&vv)[NV] = *reinterpret_cast<double(*)[NV]>(v);
    tile_partials<NV, MTX * MTY>(vv, part, t);
  }
  sched_finish(ts);
  rhs_close<NV, MEAN, COMP>(g, part, S, mc.ntiles, cond, use_cond);
}

// k_rhs for a compensated FP32 start with eps = 1 on whole tiles of 64 x 16
// columns (nx a multiple of 64, ny of 16): the same outputs, sums and tile
// order, with each field staged with only the neighbours its term reads --
// phi and its remainder with the x and y halo of the 7-point operator, P_y
// with its halo rows, P_x with its halo columns, P_z at the own cells (its
// z neighbours come down the own column).  A stage is 23 680 bytes instead
// of the general march's 25 920, and there are fewer copies to issue.  The
// copies of plane v + 3 are issued after plane v's barrier, into the stage
// plane v - 1 had (every thread has finished it by then): plane v is read
// in-plane, plane v + 1 at the own cells, planes v + 2 and v + 3 are in
// flight.  Four stages, two blocks of 256 threads per SM.  On the
// 1024 x 1024 x 128 film, against this form: three stages (one plane in
// flight, three blocks per SM) 14 % slower, the copies issued before the
// barrier (one plane in flight) 4 %, the own column's current plane read back
// from its stage instead of carried 8 %.
constexpr int RW_RS = 72;                  // phi / lo / P_x rows: x0 - 4 .. x0 + 67 (x0 at column 4)
constexpr int RW_PHI = 0;                  // stage offsets (floats): phi, rows y0 - 1 .. y0 + 16
constexpr int RW_LO = RW_PHI + 18 * RW_RS; // remainder of the start, as phi
constexpr int RW_PY = RW_LO + 18 * RW_RS;  // P_y, rows y0 - 1 .. y0 + 16, columns x0 .. x0 + 63
constexpr int RW_PX = RW_PY + 18 * 64;     // P_x, rows y0 .. y0 + 15, as phi's columns
constexpr int RW_PZ = RW_PX + 16 * RW_RS;  // P_z, rows y0 .. y0 + 15, columns x0 .. x0 + 63
constexpr int RW_STAGE = RW_PZ + 16 * 64;
constexpr int RW_D = 2;                    // planes in flight beyond the two being read
constexpr int RW_NS = RW_D + 2;
constexpr size_t rhs_w_smem_bytes() { return (size_t)RW_NS * RW_STAGE * sizeof(float); }
static_assert(RW_LO % 4 == 0 && RW_PY % 4 == 0 && RW_PX % 4 == 0 && RW_PZ % 4 == 0 && RW_STAGE % 4 == 0,
              "16-byte aligned stage regions");

__global__ void __launch_bounds__(MTX* MTY, RW_D == 1 ? 3 : 2) k_rhs_w(Geo g, Bc<float> bc, const float* __restrict__ P,
                                                      const float* __restrict__ phi, const float* __restrict__ lo,
                                                      float* __restrict__ r, double* part, Scalars* S, MarchCfg mc,
                                                      cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  static_assert(MTX == 16 && MTY == 16, "tiles of 64 x 16 columns, four cells a thread");
  float* const stg = reinterpret_cast<float*>(smem);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long nxy = g.nxy;
  const float* const Px = P;
  const float* const Py = P + g.n;
  const float* const Pz = P + 2 * g.n;
  const float mb = float(S->mean_b);
  const float inv6 = 1.0f / (6.0f * float(g.ih2));
  const float ih = float(g.ih), ih2 = float(g.ih2);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * MTX;
  // own vector in each region of a stage
  const int o_phi = (ty + 1) * RW_RS + 4 + 4 * tx, o_py = (ty + 1) * 64 + 4 * tx;
  const int o_px = ty * RW_RS + 4 + 4 * tx, o_pz = ty * 64 + 4 * tx;
  auto load4 = [](const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  };
  // z of virtual plane v of a tile starting at z0 (v = 0: the plane below,
  // nt + 1: the plane above), -1 past a non-periodic face
  auto plane_of = [&](int z0, int v) {
    int z = z0 - 1 + v;
    if (z < 0) z = g.periodic_z ? z + nz : -1;
    else if (z >= nz) z = g.periodic_z ? z - nz : -1;
    return z;
  };
  Acc<float> abb, arr, arz;
  const TileSched ts{&S->sched_next, &S->sched_done, mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < mc.ntiles; t = sched_next(ts, &tile_slot)) {
    const TileGeo<MTX, MTY, 4> s = tile_geo<MTX, MTY, 4>(g, t, mc);
    const int x0 = s.x - 4 * tx, y0 = s.y - ty, z0 = s.z0, nt = s.z1 - s.z0;
    // The halo copies of a plane: 96 vectors (phi, lo and P_y, the rows
    // y0 - 1 and y0 + 16) by threads 0 .. 95, 96 cells (phi, lo and P_x, the
    // columns x0 - 1 and x0 + 64) by threads 96 .. 191; periodic x/y wrap in
    // the source.
    const float* hsrc = nullptr;
    int hdst = -1;
    bool hvec = false;
    if (tid < 96) {
      const int f = tid >> 5, bot = (tid >> 4) & 1, c = tid & 15;
      const int y = bot ? (y0 + 16 == ny ? 0 : y0 + 16) : (y0 == 0 ? ny - 1 : y0 - 1);
      hsrc = (f == 0 ? phi : f == 1 ? lo : Py) + (long long)y * nx + x0 + 4 * c;
      hdst = f == 2 ? RW_PY + bot * 17 * 64 + 4 * c : (f == 0 ? RW_PHI : RW_LO) + bot * 17 * RW_RS + 4 + 4 * c;
      hvec = true;
    } else if (tid < 192) {
      const int j = tid - 96, f = j >> 5, rgt = (j >> 4) & 1, row = j & 15;
      const int x = rgt ? (x0 + 64 == nx ? 0 : x0 + 64) : (x0 == 0 ? nx - 1 : x0 - 1);
      hsrc = (f == 0 ? phi : f == 1 ? lo : Px) + (long long)(y0 + row) * nx + x;
      hdst = (f == 2 ? RW_PX + row * RW_RS : (f == 0 ? RW_PHI : RW_LO) + (row + 1) * RW_RS) + (rgt ? 68 : 3);
    }
    auto issue = [&](int v) {
      const int z = v <= nt + 1 ? plane_of(z0, v) : -1;
      if (z >= 0) {
        float* st = stg + (v % RW_NS) * RW_STAGE;
        const long long zo = (long long)z * nxy, go = zo + s.xy;
        cp_async<16>(st + RW_PHI + o_phi, phi + go);
        cp_async<16>(st + RW_LO + o_phi, lo + go);
        cp_async<16>(st + RW_PZ + o_pz, Pz + go);
        if (v >= 1 && v <= nt) {
          cp_async<16>(st + RW_PY + o_py, Py + go);
          cp_async<16>(st + RW_PX + o_px, Px + go);
          if (hvec) cp_async<16>(st + hdst, hsrc + zo);
          else if (hdst >= 0) cp_async<4>(st + hdst, hsrc + zo);
        }
      }
      cp_commit();
    };
    abb = Acc<float>();
    arr = Acc<float>();
    arz = Acc<float>();
    // z carry of the own column: P_z, phi, lo at planes v - 1 and v (plane
    // v + 1 is read at the own cells of its stage)
    float zm[3][4], cc[3][4];
    for (int w = 0; w < RW_NS; ++w) issue(w);
    for (int v = 1; v <= nt; ++v) {
      cp_wait<RW_D - 1>();                 // planes <= v + 1 of this thread have landed
      __syncthreads();                     // ... of every thread, and plane v - 1 is no longer read
      const int zb = plane_of(z0, v - 1), za = plane_of(z0, v + 1);
      if (v == 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) zm[0][i] = zm[1][i] = zm[2][i] = 0.f;
        if (zb >= 0) {                     // stage 0: the plane below
          load4(stg + RW_PZ + o_pz, zm[0]);
          load4(stg + RW_PHI + o_phi, zm[1]);
          load4(stg + RW_LO + o_phi, zm[2]);
        }
        load4(stg + RW_STAGE + RW_PZ + o_pz, cc[0]);
        load4(stg + RW_STAGE + RW_PHI + o_phi, cc[1]);
        load4(stg + RW_STAGE + RW_LO + o_phi, cc[2]);
      }
      issue(v + RW_D + 1);                 // into the stage of plane v - 1 (plane 0 read just above)
      const float* sc = stg + (v % RW_NS) * RW_STAGE;
      const float* sa = stg + ((v + 1) % RW_NS) * RW_STAGE;
      const int z = z0 + v - 1;
      // own vector of carried field k at planes v (carried) and v + 1 (stage
      // offset off; 0 past a face), which becomes the carried plane
      auto own = [&](int off, int k, float (&c)[4], float (&p)[4]) {
#pragma unroll
        for (int i = 0; i < 4; ++i) c[i] = cc[k][i];
        if (za >= 0) load4(sa + off, p);
        else p[0] = p[1] = p[2] = p[3] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) cc[k][i] = p[i];
      };
      auto xends = [&](const float (&c)[4], int off, float& l, float& rr) {
        l = __shfl_up_sync(0xffffffffu, c[3], 1);
        rr = __shfl_down_sync(0xffffffffu, c[0], 1);
        if (tx == 0) l = sc[off - 1];
        if (tx == MTX - 1) rr = sc[off + 4];
      };
      auto plane = [&](const bool bt) {
        // electrode faces of cell i (read again where needed: fewer live registers)
        auto dlo = [&](int i) { return (bt && zb < 0) ? (int)bc.tlo[s.xy + i] : 0; };
        auto dhi = [&](int i) { return (bt && za < 0) ? (int)bc.thi[s.xy + i] : 0; };
        // b = -div P + Dirichlet terms (the general kernel's face rules)
        float rv[4], bv[4];
        {
          float pzc[4], pzp[4], px[4], pym[4], pyp[4], l, rr;
          own(RW_PZ + o_pz, 0, pzc, pzp);
          load4(sc + RW_PX + o_px, px);
          load4(sc + RW_PY + o_py - 64, pym);
          load4(sc + RW_PY + o_py + 64, pyp);
          xends(px, RW_PX + o_px, l, rr);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            Stencil7<Raw<float, 3>> sp;
            sp.c.v[2] = pzc[i];
            sp.xm.v[0] = i == 0 ? l : px[i - 1];
            sp.xp.v[0] = i == 3 ? rr : px[i + 1];
            sp.ym.v[1] = pym[i];
            sp.yp.v[1] = pyp[i];
            sp.zm.v[2] = zm[0][i];
            sp.zp.v[2] = pzp[i];
            sp.zb = bt ? zb : 0;
            sp.za = bt ? za : 0;
            const int dl = dlo(i), dh = dhi(i);
            float dir = 0.f;
            if (dl) dir += 2.f * bc.vlo[s.xy + i];
            if (dh) dir += 2.f * bc.vhi[s.xy + i];
            bv[i] = -divergence(sp, dl, dh) * ih + dir * ih2 - mb;
            rv[i] = bv[i];
            zm[0][i] = pzc[i];
          }
        }
        // r0 = b - A phi - A lo
#pragma unroll
        for (int k = 1; k < 3; ++k) {
          const int off = (k == 1 ? RW_PHI : RW_LO) + o_phi;
          float c[4], p[4], ym[4], yp[4], l, rr;
          own(off, k, c, p);
          load4(sc + off - RW_RS, ym);
          load4(sc + off + RW_RS, yp);
          xends(c, off, l, rr);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            Stencil7<float> q;
            q.c = c[i];
            q.xm = i == 0 ? l : c[i - 1];
            q.xp = i == 3 ? rr : c[i + 1];
            q.ym = ym[i];
            q.yp = yp[i];
            q.zm = zm[k][i];
            q.zp = p[i];
            q.zb = bt ? zb : 0;
            q.za = bt ? za : 0;
            rv[i] -= apply_bt(q, dlo(i), dhi(i), ih2, bt);
            zm[k][i] = c[i];
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float inv = bt ? inv_diag_unit(g, bc, s.xy + i, z, inv6) : inv6;
          abb.add(bv[i], bv[i]);
          arr.add(rv[i], rv[i]);
          arz.add(rv[i], rv[i] * inv);
        }
        abb.run();
        arr.run();
        arz.run();
        *reinterpret_cast<float4*>(r + (long long)z * nxy + s.xy) = make_float4(rv[0], rv[1], rv[2], rv[3]);
      };
      if (zb < 0 || za < 0) plane(true);
      else plane(false);
    }
    cp_wait<0>();
    double vals[3] = {abb.value(), arr.value(), arz.value()};
    tile_partials<3, MTX * MTY>(vals, part, t);
  }
  sched_finish(ts);
  rhs_close<3, false, true>(g, part, S, mc.ntiles, cond, use_cond);
}

template <typename T>
struct Coef {
  T c1, c11, c12, g, dtL;        // c1 = 2 a1, c11 = 4 a11, c12 = 2 a12 (exact scalings)
  T amp;                         // thermal random force: sigma sqrt(dt) (0: off)
  unsigned long long seed;
  long long* step;               // device step counter (steps since pf_bind)
  int advance;                   // 1: the last block advances the step counter
};

template <typename T>
struct P3 {
  T x, y, z;
};

// Compensated state of one cell after a step: the new P and its remainder.
template <typename T>
struct P6 {
  T x, y, z, lx, ly, lz;
};

// VX floats -> bf16 remainders (one 8-byte store for a 4-cell vector).
template <int VX>
__device__ __forceinline__ void store_bf16(unsigned short* p, const float (&v)[VX]) {
  unsigned short b[VX];
#pragma unroll
  for (int i = 0; i < VX; ++i) b[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v[i]));
  if constexpr (VX == 4) {
    *reinterpret_cast<uint2*>(p) = make_uint2((unsigned)b[0] | ((unsigned)b[1] << 16),
                                              (unsigned)b[2] | ((unsigned)b[3] << 16));
  } else {
#pragma unroll
    for (int i = 0; i < VX; ++i) p[i] = b[i];
  }
}

// VX bf16 values kept packed in registers (two per 32-bit word) and widened
// one at a time: a bf16 is the upper half of the float with the same value.
template <int VX>
struct Bf16x {
  unsigned w[(VX + 1) / 2];
};
template <int VX>
__device__ __forceinline__ Bf16x<VX> load_bf16x(const unsigned short* p) {
  Bf16x<VX> r;
  if constexpr (VX == 4) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    r.w[0] = u.x;
    r.w[1] = u.y;
  } else if constexpr (VX == 2) {
    r.w[0] = *reinterpret_cast<const unsigned*>(p);
  } else {
#pragma unroll
    for (int i = 0; i < (VX + 1) / 2; ++i) r.w[i] = 0u;
#pragma unroll
    for (int i = 0; i < VX; ++i) r.w[i >> 1] |= (unsigned)p[i] << ((i & 1) * 16);
  }
  return r;
}
template <int VX>
__device__ __forceinline__ float bf16x_at(const Bf16x<VX>& r, int i) {
  return __uint_as_float(((r.w[i >> 1] >> ((i & 1) * 16)) & 0xffffu) << 16);
}

// a + b = s + e exactly (TwoSum, Knuth): no condition on the magnitudes.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
  s = a + b;
  const T bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// dt L (-df/dP + g Lap P + E) at one cell from its stencil (P in v[0..2], phi
// in v[3]); zb / za < 0 mark a z face (Neumann P, the face value of phi).
template <typename T>
__device__ __forceinline__ void tdgl_inc(const Stencil7<Raw<T, 4>>& st, int xy, int z, const Geo& g,
                                         const Bc<T>& bc, const Coef<T>& k, T (&inc)[3]) {
  const T h = T(0.5), ih = T(g.ih), ih2 = T(g.ih2);
  // E = -grad phi from face values (mean inside, V at an electrode, phi_cell at an open face)
  const T fc = st.c.v[3];
  T E[3];
  E[0] = -(h * (st.xp.v[3] - st.xm.v[3])) * ih;      // the face values' phi_c cancels
  E[1] = -(h * (st.yp.v[3] - st.ym.v[3])) * ih;
  T flo, fhi;
  if (st.zb >= 0) flo = h * (fc + st.zm.v[3]);
  else flo = bc.tlo[xy] ? bc.vlo[xy] : fc;
  if (st.za >= 0) fhi = h * (fc + st.zp.v[3]);
  else fhi = bc.thi[xy] ? bc.vhi[xy] : fc;
  E[2] = -(fhi - flo) * ih;
  const T p[3] = {st.c.v[0], st.c.v[1], st.c.v[2]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, l = (i + 2) % 3;
    const T hi = k.c1 * p[i] + k.c11 * p[i] * p[i] * p[i] + k.c12 * p[i] * (p[j] * p[j] + p[l] * p[l]);
    T lap = T(0);
    lap += st.xm.v[i] - p[i];
    lap += st.xp.v[i] - p[i];
    lap += st.ym.v[i] - p[i];
    lap += st.yp.v[i] - p[i];
    if (st.zb >= 0) lap += st.zm.v[i] - p[i];
    if (st.za >= 0 && (z + 1 < g.zair || g.zair == g.nz)) lap += st.zp.v[i] - p[i];   // free surface under air
    lap *= ih2;
    inc[i] = k.dtL * (-hi + k.g * lap + E[i]);
  }
}

template <typename T, bool CORR, bool NOISE, int VX, bool COMP = false>
__global__ void __launch_bounds__(MTX* MTY, 2) k_tdgl(Geo g, Bc<T> bc, const T* __restrict__ P, T* __restrict__ Pn,
                                                  const T* __restrict__ phi, Coef<T> k, Scalars* S, MarchCfg mc,
                                                  unsigned short* __restrict__ Plo) {
  static_assert(!(COMP && CORR), "the compensated state is a forward-Euler mode");
  using Out = typename std::conditional<COMP, P6<T>, P3<T>>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  // every block reads the step before the last block to finish advances it
  const unsigned long long nstep = (unsigned long long)*k.step;
  const T* hsrc[4] = {P, P + g.n, P + 2 * g.n, phi};
  const T* osrc[1] = {nullptr};
  TileGeo<MTX, MTY, VX> s;
  // remainders of the own vector (COMP), packed: those of plane z are loaded
  // while plane z - 1 is stored, so their latency hides behind a plane of work
  Bf16x<VX> lraw[3];
  auto load_lo = [&](int z) {
    const long long c0 = (long long)z * g.nxy + s.xy;
#pragma unroll
    for (int i = 0; i < 3; ++i) lraw[i] = load_bf16x<VX>(Plo + i * g.n + c0);
  };
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, 4>>& st, const T (&)[1], bool) -> Out {
    T p[3] = {st.c.v[0], st.c.v[1], st.c.v[2]};
    T inc[3];
    tdgl_inc(st, xy, z, g, bc, k, inc);
    T gz[3] = {T(0), T(0), T(0)};
    if constexpr (NOISE && !CORR) gauss3<T>((unsigned long long)z * g.nxy + xy, nstep, k.seed, gz);
    if constexpr (COMP) {
      const int iv = xy - s.xy;                     // index inside the own vector
      T hv[3], lv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        T d = bf16x_at(lraw[i], iv) + inc[i];
        if constexpr (NOISE) d += k.amp * gz[i];
        two_sum(p[i], d, hv[i], lv[i]);
      }
      return Out{hv[0], hv[1], hv[2], lv[0], lv[1], lv[2]};
    } else {
      T out[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        out[i] = p[i] + inc[i];
        if constexpr (NOISE && !CORR) out[i] += k.amp * gz[i];
      }
      return Out{out[0], out[1], out[2]};
    }
  };
  auto post = [&](int z, const Out (&ov)[VX]) {
    const long long c = (long long)z * g.nxy + s.xy;
    if constexpr (COMP) {
      if (z + 1 < s.z1) load_lo(z + 1);          // the next plane's remainders (the own cells of plane z are done)
    }
    T a[VX], b[VX], d[VX];
    if (z >= g.zair) {                 // air layers carry no polarization
#pragma unroll
      for (int i = 0; i < VX; ++i) a[i] = b[i] = d[i] = T(0);
      store_n<T, VX>(Pn + c, a);
      store_n<T, VX>(Pn + g.n + c, b);
      store_n<T, VX>(Pn + 2 * g.n + c, d);
      if constexpr (COMP) {
        store_bf16<VX>(Plo + c, a);
        store_bf16<VX>(Plo + g.n + c, b);
        store_bf16<VX>(Plo + 2 * g.n + c, d);
      }
      return;
    }
    if constexpr (COMP) {
      T la[VX], lb[VX], ld[VX];
#pragma unroll
      for (int i = 0; i < VX; ++i) {
        la[i] = ov[i].lx;
        lb[i] = ov[i].ly;
        ld[i] = ov[i].lz;
      }
      store_bf16<VX>(Plo + c, la);
      store_bf16<VX>(Plo + g.n + c, lb);
      store_bf16<VX>(Plo + 2 * g.n + c, ld);
    }
#pragma unroll
    for (int i = 0; i < VX; ++i) {
      a[i] = ov[i].x;
      b[i] = ov[i].y;
      d[i] = ov[i].z;
    }
    if constexpr (CORR) {
      T ca[VX], cb[VX], cd[VX];
      load_n<T, VX>(Pn + c, ca);
      load_n<T, VX>(Pn + g.n + c, cb);
      load_n<T, VX>(Pn + 2 * g.n + c, cd);
#pragma unroll
      for (int i = 0; i < VX; ++i) {
        a[i] = T(0.5) * (ca[i] + a[i]);
        b[i] = T(0.5) * (cb[i] + b[i]);
        d[i] = T(0.5) * (cd[i] + d[i]);
      }
      if constexpr (NOISE) {
        // the predictor carried the increment amp g; the corrected state needs
        // it whole: (P_n + P^p + dt R(P^p)) / 2 holds half of it
#pragma unroll
        for (int i = 0; i < VX; ++i) {
          T gz[3];
          gauss3<T>((unsigned long long)c + i, nstep, k.seed, gz);
          const T half = T(0.5) * k.amp;
          a[i] += half * gz[0];
          b[i] += half * gz[1];
          d[i] += half * gz[2];
        }
      }
    }
    store_n<T, VX>(Pn + c, a);
    store_n<T, VX>(Pn + g.n + c, b);
    store_n<T, VX>(Pn + 2 * g.n + c, d);
  };
  const TileSched ts{&S->sched_next, &S->sched_done, mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(g, t, mc);
    if constexpr (COMP) {
      if (s.act) load_lo(s.z0);
    }
    march_direct<T, Out, MTX, MTY, VX, 4, 0, STEP_D>(g, s, smem, hsrc, osrc, emit, post);
  }
  // sched_finish, with the step counter advanced by the last block to finish
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    if (atomicAdd(ts.done, 1u) == gridDim.x - 1) {
      *ts.next = 0ull;
      *ts.done = 0u;
      if (k.advance) *k.step = (long long)nstep + 1;
      __threadfence();
    }
  }
}

// k_tdgl for the compensated FP32 forward-Euler state without noise on whole
// tiles of 64 x 16 columns (nx a multiple of 64, ny of 16): the same update
// cell by cell (tdgl_inc, then TwoSum with the remainder) on the same staged
// planes, with the halo copies shared evenly over the block (each thread one
// row vector or one column cell of one field, instead of the edge threads
// copying every field's halo) and no ragged-tile or inactive-thread logic.
// 1.6 % faster than k_tdgl on the 1024 x 1024 x 128 film.  (Issuing each
// plane's copies after the barrier, two planes in flight as in k_rhs_w, was
// 0.6 % slower here; reading the own column's current plane from its stage
// instead of carrying it, 7 %.)
constexpr int TW_RS = 72;                  // a staged row: x0 - 4 .. x0 + 67 (x0 at column 4)
constexpr int TW_F = 18 * TW_RS;           // one field of a stage: rows y0 - 1 .. y0 + 16
constexpr int TW_STAGE = 4 * TW_F;         // P_x, P_y, P_z, phi
constexpr int TW_D = 2;                    // planes of cp.async look-ahead
constexpr int TW_NS = TW_D + 2;
constexpr size_t tdgl_w_smem_bytes() { return (size_t)TW_NS * TW_STAGE * sizeof(float); }

__global__ void __launch_bounds__(MTX* MTY, 2) k_tdgl_w(Geo g, Bc<float> bc, const float* __restrict__ P,
                                                       float* __restrict__ Pn, const float* __restrict__ phi,
                                                       Coef<float> k, Scalars* S, MarchCfg mc,
                                                       unsigned short* __restrict__ Plo) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  static_assert(MTX == 16 && MTY == 16, "tiles of 64 x 16 columns, four cells a thread");
  float* const stg = reinterpret_cast<float*>(smem);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long nxy = g.nxy, n = g.n;
  // every block reads the step before the last block to finish advances it
  const unsigned long long nstep = (unsigned long long)*k.step;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * MTX;
  const int o = (ty + 1) * TW_RS + 4 + 4 * tx;     // own vector in a field of a stage
  auto field = [&](int f) -> const float* { return f < 3 ? P + f * n : phi; };
  auto load4 = [](const float* q, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(q);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  };
  auto plane_of = [&](int z0, int v) {
    int z = z0 - 1 + v;
    if (z < 0) z = g.periodic_z ? z + nz : -1;
    else if (z >= nz) z = g.periodic_z ? z - nz : -1;
    return z;
  };
  const TileSched ts{&S->sched_next, &S->sched_done, mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < mc.ntiles; t = sched_next(ts, &tile_slot)) {
    const TileGeo<MTX, MTY, 4> s = tile_geo<MTX, MTY, 4>(g, t, mc);
    const int x0 = s.x - 4 * tx, y0 = s.y - ty, z0 = s.z0, nt = s.z1 - s.z0;
    // halo copies of a plane: threads 0 .. 127 the row vectors y0 - 1 and
    // y0 + 16 of field tid / 32, threads 128 .. 255 the cells x0 - 1 and x0 + 64
    // of one row of field (tid - 128) / 32; periodic x/y wrap in the source
    const float* hsrc;
    int hdst;
    const bool hvec = tid < 128;
    if (hvec) {
      const int f = tid >> 5, bot = (tid >> 4) & 1, c = tid & 15;
      const int y = bot ? (y0 + 16 == ny ? 0 : y0 + 16) : (y0 == 0 ? ny - 1 : y0 - 1);
      hsrc = field(f) + (long long)y * nx + x0 + 4 * c;
      hdst = f * TW_F + bot * 17 * TW_RS + 4 + 4 * c;
    } else {
      const int j = tid - 128, f = j >> 5, rgt = (j >> 4) & 1, row = j & 15;
      const int x = rgt ? (x0 + 64 == nx ? 0 : x0 + 64) : (x0 == 0 ? nx - 1 : x0 - 1);
      hsrc = field(f) + (long long)(y0 + row) * nx + x;
      hdst = f * TW_F + (row + 1) * TW_RS + (rgt ? 68 : 3);
    }
    auto issue = [&](int v) {
      const int z = v <= nt + 1 ? plane_of(z0, v) : -1;
      if (z >= 0) {
        float* st = stg + (v % TW_NS) * TW_STAGE;
        const long long zo = (long long)z * nxy, go = zo + s.xy;
#pragma unroll
        for (int f = 0; f < 4; ++f) cp_async<16>(st + f * TW_F + o, field(f) + go);
        if (v >= 1 && v <= nt) {
          if (hvec) cp_async<16>(st + hdst, hsrc + zo);
          else cp_async<4>(st + hdst, hsrc + zo);
        }
      }
      cp_commit();
    };
    // remainders of the own vector, packed: those of plane z are loaded while
    // plane z - 1 is stored, so their latency hides behind a plane of work
    Bf16x<4> lraw[3];
    auto load_lo = [&](int z) {
      const long long c0 = (long long)z * nxy + s.xy;
#pragma unroll
      for (int i = 0; i < 3; ++i) lraw[i] = load_bf16x<4>(Plo + i * n + c0);
    };
    load_lo(z0);
    float zm[4][4], c[4][4];               // the own column's fields at planes v - 1 and v
    for (int w = 0; w < TW_NS - 1; ++w) issue(w);
    for (int v = 1; v <= nt; ++v) {
      issue(v + TW_D);                     // into the stage of plane v - 2: a thread still at plane
                                           // v - 1 reads those of planes v - 1 and v only
      cp_wait<TW_D - 1>();                 // planes <= v + 1 of this thread have landed
      __syncthreads();                     // ... and of every thread
      const int zb = plane_of(z0, v - 1), za = plane_of(z0, v + 1);
      if (v == 1) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (zb >= 0) load4(stg + f * TW_F + o, zm[f]);
          else zm[f][0] = zm[f][1] = zm[f][2] = zm[f][3] = 0.f;
          load4(stg + TW_STAGE + f * TW_F + o, c[f]);
        }
      }
      const float* sc = stg + (v % TW_NS) * TW_STAGE;
      const float* sa = stg + ((v + 1) % TW_NS) * TW_STAGE;
      const int z = z0 + v - 1;
      float zp[4][4], ym[4][4], yp[4][4], xl[4], xr[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float* q = sc + f * TW_F + o;
        if (za >= 0) load4(sa + f * TW_F + o, zp[f]);
        else zp[f][0] = zp[f][1] = zp[f][2] = zp[f][3] = 0.f;
        load4(q - TW_RS, ym[f]);
        load4(q + TW_RS, yp[f]);
        xl[f] = __shfl_up_sync(0xffffffffu, c[f][3], 1);
        xr[f] = __shfl_down_sync(0xffffffffu, c[f][0], 1);
        if (tx == 0) xl[f] = q[-1];
        if (tx == MTX - 1) xr[f] = q[4];
      }
      const bool bt = zb < 0 || za < 0;
      float a[4], b[4], d[4], la[4], lb[4], ld[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        Stencil7<Raw<float, 4>> st;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          st.c.v[f] = c[f][i];
          st.xm.v[f] = i == 0 ? xl[f] : c[f][i - 1];
          st.xp.v[f] = i == 3 ? xr[f] : c[f][i + 1];
          st.ym.v[f] = ym[f][i];
          st.yp.v[f] = yp[f][i];
          st.zm.v[f] = zm[f][i];
          st.zp.v[f] = zp[f][i];
        }
        st.zb = bt ? zb : 0;
        st.za = bt ? za : 0;
        float inc[3], hv[3], lv[3];
        tdgl_inc(st, s.xy + i, z, g, bc, k, inc);
#pragma unroll
        for (int f = 0; f < 3; ++f) two_sum(c[f][i], bf16x_at(lraw[f], i) + inc[f], hv[f], lv[f]);
        a[i] = hv[0]; b[i] = hv[1]; d[i] = hv[2];
        la[i] = lv[0]; lb[i] = lv[1]; ld[i] = lv[2];
      }
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          zm[f][i] = c[f][i];
          c[f][i] = zp[f][i];
        }
      if (z + 1 < s.z1) load_lo(z + 1);      // the next plane's remainders (the own cells of plane z are done)
      const long long cz = (long long)z * nxy + s.xy;
      if (z >= g.zair) {                     // air layers carry no polarization
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = b[i] = d[i] = la[i] = lb[i] = ld[i] = 0.f;
      }
      store_bf16<4>(Plo + cz, la);
      store_bf16<4>(Plo + n + cz, lb);
      store_bf16<4>(Plo + 2 * n + cz, ld);
      *reinterpret_cast<float4*>(Pn + cz) = make_float4(a[0], a[1], a[2], a[3]);
      *reinterpret_cast<float4*>(Pn + n + cz) = make_float4(b[0], b[1], b[2], b[3]);
      *reinterpret_cast<float4*>(Pn + 2 * n + cz) = make_float4(d[0], d[1], d[2], d[3]);
    }
    cp_wait<0>();
  }
  // sched_finish, with the step counter advanced by the last block to finish
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    if (atomicAdd(ts.done, 1u) == gridDim.x - 1) {
      *ts.next = 0ull;
      *ts.done = 0u;
      if (k.advance) *k.step = (long long)nstep + 1;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------- launchers

template <typename K>
static void smem_attr(K kernel, size_t bytes, bool& done) {
  if (!done) {
    allow_smem(kernel, bytes);
    done = true;
  }
}

// The whole-tile kernels (k_rhs_w, k_tdgl_w) take an FP32 time series when
// the march's tiles are whole 64 x 16 tiles.
static bool rhs_whole(const Geo& g, const MarchCfg& mc) { return mc.vx == 4 && g.nx % 64 == 0 && g.ny % MTY == 0; }

// Grid of a whole-tile kernel: its own occupancy (or the blocks per SM a
// tiling asked for, if fewer) on every SM, at most a block per tile.
template <class K>
static int own_grid(K kernel, size_t bytes, const MarchCfg& mc, int& occ, int& nsm) {
  if (occ == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, MTX * MTY, bytes) != cudaSuccess) occ = 1;
    cudaGetLastError();
    occ = std::max(occ, 1);
  }
  const int bps = mc.bps > 0 ? std::min(mc.bps, occ) : occ;
  return (int)std::min<long long>(mc.ntiles, std::min<long long>(MAX_GRID, (long long)bps * nsm));
}

static void rhs_w(const LaunchCfg& L, const Geo& g, const Dev<float>& d, const float* P, cudaGraphConditionalHandle cond,
                  int use_cond) {
  static bool f = false;
  static int occ = 0, nsm = 0;
  const size_t bytes = rhs_w_smem_bytes();
  smem_attr(k_rhs_w, bytes, f);
  const int grid = own_grid(k_rhs_w, bytes, L.march, occ, nsm);
  k_rhs_w<<<grid, dim3(MTX, MTY), bytes, L.stream>>>(g, d.bc, P, d.cp.hi, d.cp.lo, d.r, d.part, d.S, L.march, cond,
                                                     use_cond);
}

template <typename T, bool EPS, bool MEAN, int VX, bool COMP>
static void rhs_t(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, cudaGraphConditionalHandle cond,
                  int use_cond) {
  if constexpr (std::is_same<T, float>::value && !EPS && !MEAN && VX == 4 && COMP) {
    if (rhs_whole(g, L.march)) {
      rhs_w(L, g, d, P, cond, use_cond);
      return;
    }
  }
  static bool f = false;
  const size_t bytes = StepPipe<T, EPS, VX, COMP ? 1 : 0>::bytes();
  smem_attr(k_rhs<T, EPS, MEAN, VX, COMP>, bytes, f);
  k_rhs<T, EPS, MEAN, VX, COMP><<<L.march.grid, dim3(MTX, MTY), bytes, L.stream>>>(
      g, d.bc, P, COMP ? d.cp.hi : d.phi, d.cp.lo, d.eps, d.invd, d.r, d.part, d.S, L.march, cond, use_cond);
}

template <typename T, bool MEAN, bool COMP>
static void rhs_c(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, cudaGraphConditionalHandle cond,
                  int use_cond) {
  constexpr int V = 16 / sizeof(T);
  const bool vec = L.march.vx == V;
  if (d.eps) {
    if (vec) rhs_t<T, true, MEAN, V, COMP>(L, g, d, P, cond, use_cond);
    else rhs_t<T, true, MEAN, 1, COMP>(L, g, d, P, cond, use_cond);
  } else {
    if (vec) rhs_t<T, false, MEAN, V, COMP>(L, g, d, P, cond, use_cond);
    else rhs_t<T, false, MEAN, 1, COMP>(L, g, d, P, cond, use_cond);
  }
}

template <typename T, bool MEAN>
static void rhs_v(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, cudaGraphConditionalHandle cond,
                  int use_cond) {
  // compensated starts are FP32 only (FP64 potentials need no remainder)
  if constexpr (!MEAN && std::is_same<T, float>::value) {
    if (d.cp.lo) {
      rhs_c<T, false, true>(L, g, d, P, cond, use_cond);
      return;
    }
  }
  rhs_c<T, MEAN, false>(L, g, d, P, cond, use_cond);
}

template <typename T>
void launch_rhs_mean(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P) {
  rhs_v<T, true>(L, g, d, P, 0, 0);
}

template <typename T>
void launch_rhs(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, cudaGraphConditionalHandle cond,
                int use_cond) {
  rhs_v<T, false>(L, g, d, P, cond, use_cond);
}

template <typename T, bool CORR, bool NOISE, int VX, bool COMP>
static void tdgl_t(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, T* Pn, const Coef<T>& k) {
  static bool f = false;
  const size_t bytes = StepPipe<T, false, VX>::bytes();
  smem_attr(k_tdgl<T, CORR, NOISE, VX, COMP>, bytes, f);
  k_tdgl<T, CORR, NOISE, VX, COMP><<<L.march.grid, dim3(MTX, MTY), bytes, L.stream>>>(g, d.bc, P, Pn, d.phi, k, d.S,
                                                                                     L.march, d.plo);
}

template <typename T, bool CORR, bool NOISE>
static void tdgl_v(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, T* Pn, const Coef<T>& k) {
  constexpr int V = 16 / sizeof(T);
  // the compensated state exists for FP32 forward Euler (d.plo set)
  if constexpr (!CORR && std::is_same<T, float>::value) {
    if constexpr (!NOISE) {
      if (d.plo && rhs_whole(g, L.march)) {       // whole 64 x 16 tiles
        static bool f = false;
        static int occ = 0, nsm = 0;
        const size_t bytes = tdgl_w_smem_bytes();
        smem_attr(k_tdgl_w, bytes, f);
        const int grid = own_grid(k_tdgl_w, bytes, L.march, occ, nsm);
        k_tdgl_w<<<grid, dim3(MTX, MTY), bytes, L.stream>>>(g, d.bc, P, Pn, d.phi, k, d.S, L.march, d.plo);
        return;
      }
    }
    if (d.plo) {
      if (L.march.vx == V) tdgl_t<T, CORR, NOISE, V, true>(L, g, d, P, Pn, k);
      else tdgl_t<T, CORR, NOISE, 1, true>(L, g, d, P, Pn, k);
      return;
    }
  }
  if (L.march.vx == V) tdgl_t<T, CORR, NOISE, V, false>(L, g, d, P, Pn, k);
  else tdgl_t<T, CORR, NOISE, 1, false>(L, g, d, P, Pn, k);
}

template <typename T>
void launch_tdgl(const LaunchCfg& L, const Geo& g, const Dev<T>& d, const T* P, T* Pn, const double* coef,
                 int corr, const Noise& nz) {
  Coef<T> k{T(2) * T(coef[0]), T(4) * T(coef[1]), T(2) * T(coef[2]), T(coef[3]), T(coef[4]), T(nz.amp), nz.seed,
            nz.step, nz.advance};
  const bool noise = nz.amp != 0.0;
  if (corr) {
    if (noise) tdgl_v<T, true, true>(L, g, d, P, Pn, k);
    else tdgl_v<T, true, false>(L, g, d, P, Pn, k);
  } else {
    if (noise) tdgl_v<T, false, true>(L, g, d, P, Pn, k);
    else tdgl_v<T, false, false>(L, g, d, P, Pn, k);
  }
}

#define PF_STEP_INSTANTIATE(T)                                                                              \
  template void launch_rhs_mean<T>(const LaunchCfg&, const Geo&, const Dev<T>&, const T*);                  \
  template void launch_rhs<T>(const LaunchCfg&, const Geo&, const Dev<T>&, const T*,                        \
                              cudaGraphConditionalHandle, int);                                             \
  template void launch_tdgl<T>(const LaunchCfg&, const Geo&, const Dev<T>&, const T*, T*, const double*, int,  \
                               const Noise&);

PF_STEP_INSTANTIATE(float)
PF_STEP_INSTANTIATE(double)

}  // namespace pf
