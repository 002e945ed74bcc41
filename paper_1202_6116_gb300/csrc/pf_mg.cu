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
// With a permittivity field every level carries its own cell permittivity
// (level 0: the bound eps; a coarse cell: the mean of its children) and 1/diag
// of its operator (precomputed); faces weigh the harmonic mean of the two
// cells' eps, an electrode face 2 eps_c, as on the finest level.
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

// The interior 7-point operator (eps = 1) and the two pre-sweeps from zero,
// every operation rounded as written, with the fused multiply-adds spelled
// out (no contraction left to the compiler): the kernels that form them on
// the same cell -- the pre-smoother, the residual and their fused form on a
// split level -- then agree bit for bit.
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ T apply_int(T c, T xm, T xp, T ym, T yp, T zm, T zp, T ax, T ay, T az) {
  const T sx = rn_add(rn_sub(c, xm), rn_sub(c, xp));
  const T sy = rn_add(rn_sub(c, ym), rn_sub(c, yp));
  const T sz = rn_add(rn_sub(c, zm), rn_sub(c, zp));
  return rn_fma(ax, sx, rn_fma(ay, sy, rn_mul(az, sz)));
}

// e = e1 + w2 D^-1 (f - A e1), e1 = w1 D^-1 f, with D constant (w1 = omega1 / d,
// w2d = omega2 / d): A e1 = w1 A f.
template <typename T>
__device__ __forceinline__ T pre_int(T c, T xm, T xp, T ym, T yp, T zm, T zp, T ax, T ay, T az, T w1, T w2d) {
  const T Ae1 = rn_mul(w1, apply_int(c, xm, xp, ym, yp, zm, zp, ax, ay, az));
  return rn_fma(w2d, rn_sub(c, Ae1), rn_mul(w1, c));
}

template <typename T>
__device__ __forceinline__ T mg_inv_bt(const MgView<T>& L, int xy, int z, T inv_int, const bool bt) {
  return bt ? mg_inv(L, xy, z, inv_int) : inv_int;
}

// A v at a level with cell permittivities (v and eps carried together).
template <typename T>
__device__ __forceinline__ T apply_aniso_eps(const Stencil7<EpsVal<T>>& s, int dlo, int dhi, T ax, T ay, T az,
                                             const bool bt) {
  const T ec = s.c.e, vc = s.c.v;
  const T sx = hmean2(ec, s.xm.e) * (vc - s.xm.v) + hmean2(ec, s.xp.e) * (vc - s.xp.v);
  const T sy = hmean2(ec, s.ym.e) * (vc - s.ym.v) + hmean2(ec, s.yp.e) * (vc - s.yp.v);
  T sz = T(0);
  if (bt) {
    if (s.zb >= 0) sz += hmean2(ec, s.zm.e) * (vc - s.zm.v);
    else if (dlo) sz += T(2) * ec * vc;
    if (s.za >= 0) sz += hmean2(ec, s.zp.e) * (vc - s.zp.v);
    else if (dhi) sz += T(2) * ec * vc;
  } else {
    sz = hmean2(ec, s.zm.e) * (vc - s.zm.v) + hmean2(ec, s.zp.e) * (vc - s.zp.v);
  }
  return ax * sx + ay * sy + az * sz;
}

// Field kv with the permittivity of field ke, as one stencil.
template <typename T, int NF>
__device__ __forceinline__ Stencil7<EpsVal<T>> pick_eps(const Stencil7<Raw<T, NF>>& s, int kv, int ke) {
  Stencil7<EpsVal<T>> o;
  o.c = EpsVal<T>{s.c.v[kv], s.c.v[ke]};
  o.xm = EpsVal<T>{s.xm.v[kv], s.xm.v[ke]};
  o.xp = EpsVal<T>{s.xp.v[kv], s.xp.v[ke]};
  o.ym = EpsVal<T>{s.ym.v[kv], s.ym.v[ke]};
  o.yp = EpsVal<T>{s.yp.v[kv], s.yp.v[ke]};
  o.zm = EpsVal<T>{s.zm.v[kv], s.zm.v[ke]};
  o.zp = EpsVal<T>{s.zp.v[kv], s.zp.v[ke]};
  o.zb = s.zb;
  o.za = s.za;
  return o;
}

// Staged planes of the sweeps (E: with a permittivity field, eps staged with
// halo beside the field, 1/diag staged at the own cells -- and with halo in
// the pre-smoother, whose first sweep is formed at all seven cells).
template <typename T, int VX, bool E = false>
using MgPipeD0 = Pipe<T, void, MTX, MTY, VX, E ? 3 : 1, 0, MG_D>;
template <typename T, int VX, bool E = false>
using MgPipeP = Pipe<T, void, MTX, MTY, VX, E ? 2 : 1, E ? 2 : 1, MG_D, 1>;
template <typename T, int VX, bool E = false>
using MgPipeR = Pipe<T, void, MTX, MTY, VX, E ? 2 : 1, 1, MG_D>;
template <typename T, int VX, bool E = false>
using MgPipeD = Pipe<T, void, MTX, MTY, VX, E ? 2 : 1, E ? 2 : 1, MG_D>;

// ------------------------------------------------------------------ kernels

// Two pre-smoothing sweeps from zero, read straight from the staged planes of
// f.  The first sweep is e1 = w1 diag^-1 f; the second e = e1 + w2 diag^-1 (f -
// A e1).  Away from the z faces the diagonal is one constant, so A e1 =
// w1 diag^-1 A f there; on the planes next to a z face and their neighbour
// planes e1 is formed per neighbour with its own diagonal.
template <typename T, int VX, bool EPS, bool INT = false>
__global__ void __launch_bounds__(MTX* MTY, (sizeof(T) == 4 && !EPS) ? (INT ? 5 : 4) : 2) k_mg_pre(MgView<T> L, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  if (S->done) return;
  constexpr int NH = EPS ? 3 : 1;          // f (, eps, 1/diag)
  const T om1 = mg_omega1<T>(), om2 = mg_omega2<T>(), inv_int = mg_inv_int(L);
  const T w1 = rn_mul(om1, inv_int), w2d = rn_mul(om2, inv_int);
  const T* hsrc[NH];
  hsrc[0] = L.f;
  if constexpr (EPS) {
    hsrc[1] = L.eps;
    hsrc[2] = L.invd;
  }
  const T* osrc[1] = {nullptr};
  const int nx = L.g.nx, nz = L.g.nz;
  const bool zfaces = !L.g.periodic_z;
  TileGeo<MTX, MTY, VX> s;
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, NH>>& sr, const T (&)[1], const bool bt) -> T {
    const Stencil7<T> f = pick(sr, 0);
    if constexpr (EPS) {
      // first sweep e1 = w1 f / diag at all seven cells, then the second
      Stencil7<EpsVal<T>> e1 = pick_eps(sr, 0, 1);
      e1.c.v = om1 * sr.c.v[2] * f.c;
      e1.xm.v = om1 * sr.xm.v[2] * f.xm;
      e1.xp.v = om1 * sr.xp.v[2] * f.xp;
      e1.ym.v = om1 * sr.ym.v[2] * f.ym;
      e1.yp.v = om1 * sr.yp.v[2] * f.yp;
      e1.zm.v = f.zb >= 0 ? om1 * sr.zm.v[2] * f.zm : T(0);
      e1.zp.v = f.za >= 0 ? om1 * sr.zp.v[2] * f.zp : T(0);
      const int dlo = (bt && f.zb < 0) ? (int)L.tlo[xy] : 0;
      const int dhi = (bt && f.za < 0) ? (int)L.thi[xy] : 0;
      const T Ae1 = apply_aniso_eps(e1, dlo, dhi, L.ax, L.ay, L.az, bt);
      return e1.c.v + om2 * sr.c.v[2] * (f.c - Ae1);
    } else {
      const bool near = !INT && zfaces && (z == 1 || z == nz - 2);
      if (!bt && !near) return pre_int(f.c, f.xm, f.xp, f.ym, f.yp, f.zm, f.zp, L.ax, L.ay, L.az, w1, w2d);
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
    }
  };
  auto post = [&](int z, const T (&ov)[VX]) { store_n<T, VX>(L.e + (long long)z * L.g.nxy + s.xy, ov); };
  const TileSched ts{&S->sched_next, &S->sched_done, L.mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < L.mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(L.g, t, L.mc);
    march_direct<T, T, MTX, MTY, VX, NH, 0, MG_D, 0, INT>(L.g, s, smem, hsrc, osrc, emit, post);
  }
  sched_finish(ts);
}

// Residual and its restriction.  Children of one coarse cell: 2 planes (summed
// in registers across consecutive planes of the march), 2 rows (tile rows 2k,
// 2k+1 share a warp: lane ^ 16), 2 columns (inside the thread's vector, or
// lane ^ 1 when a thread owns one cell).
template <typename T, int VX, bool EPS>
__global__ void __launch_bounds__(MTX* MTY) k_mg_rr(MgView<T> L, MgView<T> C, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  static_assert(MTX == 16, "row pairs share a warp");
  if (S->done) return;
  constexpr int NH = EPS ? 2 : 1;          // e (, eps)
  const T* hsrc[NH];
  hsrc[0] = L.e;
  if constexpr (EPS) hsrc[1] = L.eps;
  const T* osrc[1] = {L.f};
  const T scale = T(1) / T(L.fx * L.fy * L.fz);
  TileGeo<MTX, MTY, VX> s;
  T racc[VX];
#pragma unroll
  for (int i = 0; i < VX; ++i) racc[i] = T(0);
  auto emit = [&](int xy, int, const Stencil7<Raw<T, NH>>& sr, const T (&o)[1], const bool bt) -> T {
    const bool B = bt;
    const int dlo = (B && sr.zb < 0) ? (int)L.tlo[xy] : 0;
    const int dhi = (B && sr.za < 0) ? (int)L.thi[xy] : 0;
    if constexpr (EPS) {
      return o[0] - apply_aniso_eps(pick_eps(sr, 0, 1), dlo, dhi, L.ax, L.ay, L.az, bt);
    } else {
      if (!bt) {
        const Stencil7<T> e = pick(sr, 0);
        return rn_sub(o[0], apply_int(e.c, e.xm, e.xp, e.ym, e.yp, e.zm, e.zp, L.ax, L.ay, L.az));
      }
      return o[0] - apply_aniso(pick(sr, 0), dlo, dhi, L.ax, L.ay, L.az, bt);
    }
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
  const TileSched ts{&S->sched_next, &S->sched_done, L.mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < L.mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(L.g, t, L.mc);
    march_direct<T, T, MTX, MTY, VX, NH, 1, MG_D>(L.g, s, smem, hsrc, osrc, emit, post);
  }
  sched_finish(ts);
}

// Pre-smoother, residual and restriction fused, on the interior planes of a
// split FP32 level without eps whose tiles are whole (nx a multiple of 64, ny
// of 16): one pass over f instead of f -> e, then e and f again.  The residual
// at a cell needs e at its six neighbours, and e at a cell needs f at its own
// six, so a tile stages f with a two-cell ring (periodic wrap resolved in the
// source rows and columns) and forms e on its columns and on the one-cell ring
// around them, one plane ahead of the residual.  e of the plane just below or
// above the tile is formed too (own columns), except on the planes next to a z
// face, which belong to the face slabs: there it is the face-slab
// pre-smoother's output, read back (that launch runs first; the face-slab
// residual runs after this one).  The arithmetic per cell is pre_int and
// apply_int, as in k_mg_pre and k_mg_rr, so the results are bit-identical.
// One barrier per plane: the e plane a tile writes at plane u (buffer u mod 2)
// was last read for the residual of plane u - 2, and stage u + 4 mod 5 last
// held plane u - 1; both reads end before the barrier of plane u.
constexpr int PRR_D = 2;                   // planes of cp.async look-ahead
constexpr int PRR_NS = PRR_D + 3;          // f planes w, w + 1, w + 2 in use, PRR_D in flight
constexpr int PRR_RS = 72;                 // a staged row: x0 - 4 .. x0 + 67 (x0 at 4: 16-byte aligned)
constexpr int PRR_RH = 20;                 // staged rows: y0 - 2 .. y0 + 17
constexpr int PRR_EH = 18;                 // e plane rows: y0 - 1 .. y0 + 16 (columns as staged)
constexpr int PRR_STAGE = PRR_RS * PRR_RH;
constexpr int PRR_EPLANE = PRR_RS * PRR_EH;
constexpr size_t prr_smem_bytes() { return (size_t)(PRR_NS * PRR_STAGE + 2 * PRR_EPLANE) * sizeof(float); }

__global__ void __launch_bounds__(MTX* MTY, 4) k_mg_prr(MgView<float> L, MgView<float> C, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  static_assert(MTX == 16 && MTY == 16, "tiles of 64 x 16 columns, four cells a thread");
  static_assert(PRR_RH * 16 <= 2 * MTX * MTY && PRR_RH * 4 <= MTX * MTY, "a plane's copies: two vectors and one ring cell a thread");
  if (S->done) return;
  float* const stg = reinterpret_cast<float*>(smem);
  float* const eb = stg + PRR_NS * PRR_STAGE;
  const int nx = L.g.nx, ny = L.g.ny, nz = L.g.nz;
  const long long nxy = L.g.nxy;
  const float om1 = mg_omega1<float>(), om2 = mg_omega2<float>(), inv_int = mg_inv_int(L);
  const float w1 = rn_mul(om1, inv_int), w2d = rn_mul(om2, inv_int);
  const float ax = L.ax, ay = L.ay, az = L.az;
  const float scale = 1.0f / float(L.fx * L.fy * L.fz);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * MTX;
  const int c0 = 4 + 4 * tx;               // column of the own vector in a stage or e plane
  const int so = (ty + 2) * PRR_RS + c0;   // own vector in a stage
  const int eo = (ty + 1) * PRR_RS + c0;   // own vector in an e plane
  // ring cell of this thread (threads 0 .. 159): stage row, e-plane row, column
  int rr = -1, re = -1, rc = -1;
  if (tid < 64) { rr = 1; re = 0; rc = 4 + tid; }
  else if (tid < 128) { rr = 18; re = 17; rc = 4 + tid - 64; }
  else if (tid < 144) { rr = 2 + tid - 128; re = 1 + tid - 128; rc = 3; }
  else if (tid < 160) { rr = 2 + tid - 144; re = 1 + tid - 144; rc = 68; }
  auto load4 = [](const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  };
  const TileSched ts{&S->sched_next, &S->sched_done, L.mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < L.mc.ntiles; t = sched_next(ts, &tile_slot)) {
    const TileGeo<MTX, MTY, 4> s = tile_geo<MTX, MTY, 4>(L.g, t, L.mc);
    const int x0 = s.x - 4 * tx, y0 = s.y - ty, z0 = s.z0, nt = s.z1 - s.z0;
    // A staged f plane is 20 rows of 16 vectors (320 copies) plus the ring
    // columns x0 - 2, x0 - 1, x0 + 64, x0 + 65 (80 copies): this thread's share
    // (vectors tid and tid + 256, ring cell tid), located once per tile.
    auto row_of = [&](int r) {
      int y = y0 - 2 + r;
      y += y < 0 ? ny : 0;
      y -= y >= ny ? ny : 0;
      return y * nx;
    };
    const int sv0 = (tid >> 4) * PRR_RS + 4 + 4 * (tid & 15), gv0 = row_of(tid >> 4) + x0 + 4 * (tid & 15);
    const int i1 = tid + MTX * MTY;
    const bool has1 = i1 < PRR_RH * 16;
    const int sv1 = has1 ? (i1 >> 4) * PRR_RS + 4 + 4 * (i1 & 15) : 0;
    const int gv1 = has1 ? row_of(i1 >> 4) + x0 + 4 * (i1 & 15) : 0;
    const bool hasr = tid < PRR_RH * 4;
    int svr = 0, gvr = 0;
    if (hasr) {
      const int r = tid >> 2, k = tid & 3;
      int x = k < 2 ? x0 - 2 + k : x0 + 62 + k;
      x += x < 0 ? nx : 0;
      x -= x >= nx ? nx : 0;
      svr = r * PRR_RS + (k < 2 ? 2 + k : 66 + k);
      gvr = row_of(r) + x;
    }
    // f plane w (z = z0 - 2 + w) into stage w mod PRR_NS
    auto issue = [&](int w) {
      if (w <= nt + 3) {
        float* st = stg + (w % PRR_NS) * PRR_STAGE;
        const float* src = L.f + (long long)(z0 - 2 + w) * nxy;
        cp_async<16>(st + sv0, src + gv0);
        if (has1) cp_async<16>(st + sv1, src + gv1);
        if (hasr) cp_async<4>(st + svr, src + gvr);
      }
      cp_commit();
    };
    // e at a staged cell from the f planes below, at and above it
    auto e_at = [&](const float* sm, const float* sc, const float* sp, int off) -> float {
      const float* q = sc + off;
      return pre_int(q[0], q[-1], q[1], q[-PRR_RS], q[PRR_RS], sm[off], sp[off], ax, ay, az, w1, w2d);
    };
    float em2[4], em1[4], e0[4], racc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) em2[i] = em1[i] = e0[i] = racc[i] = 0.f;
    for (int w = 0; w < PRR_D + 2; ++w) issue(w);
    for (int u = 0; u <= nt + 1; ++u) {
      cp_wait<PRR_D - 1>();                // f planes u .. u + 2 of this thread have landed
      __syncthreads();                     // ... and of every thread
      issue(u + PRR_D + 2);
      const float* sm = stg + (u % PRR_NS) * PRR_STAGE;
      const float* sc = stg + ((u + 1) % PRR_NS) * PRR_STAGE;
      const float* sp = stg + ((u + 2) % PRR_NS) * PRR_STAGE;
      float* ebu = eb + (u & 1) * PRR_EPLANE;
      const int z = z0 - 1 + u;
      // e of plane z on the own vector
      if (z == 1 || z == nz - 2) {
        load4(L.e + (long long)z * nxy + s.xy, e0);
      } else {
        float fc[4], fm[4], fp[4], fym[4], fyp[4];
        load4(sc + so, fc);
        load4(sm + so, fm);
        load4(sp + so, fp);
        load4(sc + so - PRR_RS, fym);
        load4(sc + so + PRR_RS, fyp);
        // x neighbours at the vector ends: the next lanes' vectors, or the ring at the tile edge
        float fl = __shfl_up_sync(0xffffffffu, fc[3], 1), fr = __shfl_down_sync(0xffffffffu, fc[0], 1);
        if (tx == 0) fl = sc[so - 1];
        if (tx == MTX - 1) fr = sc[so + 4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          e0[i] = pre_int(fc[i], i == 0 ? fl : fc[i - 1], i == 3 ? fr : fc[i + 1], fym[i], fyp[i], fm[i], fp[i], ax,
                          ay, az, w1, w2d);
      }
      // planes whose residual this tile forms: e on the own vector and the ring
      if (u >= 1 && u <= nt) {
        *reinterpret_cast<float4*>(ebu + eo) = make_float4(e0[0], e0[1], e0[2], e0[3]);
        if (rc >= 0) ebu[re * PRR_RS + rc] = e_at(sm, sc, sp, rr * PRR_RS + rc);
      }
      // residual of plane z - 1 (its e plane is complete since this plane's barrier)
      if (u >= 2) {
        const float* ebm = eb + ((u - 1) & 1) * PRR_EPLANE;
        float ec[4], eym[4], eyp[4], fv[4], rv[4];
        load4(ebm + eo, ec);
        load4(ebm + eo - PRR_RS, eym);
        load4(ebm + eo + PRR_RS, eyp);
        load4(sm + so, fv);                // f of plane z - 1 is f plane u
        float el = __shfl_up_sync(0xffffffffu, ec[3], 1), er = __shfl_down_sync(0xffffffffu, ec[0], 1);
        if (tx == 0) el = ebm[eo - 1];
        if (tx == MTX - 1) er = ebm[eo + 4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          rv[i] = rn_sub(fv[i], apply_int(ec[i], i == 0 ? el : ec[i - 1], i == 3 ? er : ec[i + 1], eym[i], eyp[i],
                                          em2[i], e0[i], ax, ay, az));
        const int zr = z - 1;
        *reinterpret_cast<float4*>(L.e + (long long)zr * nxy + s.xy) = make_float4(ec[0], ec[1], ec[2], ec[3]);
        // restriction: 2 planes in registers, 2 rows by lane ^ 16, 2 columns in the vector
#pragma unroll
        for (int i = 0; i < 4; ++i) racc[i] += rv[i];
        if ((zr & (L.fz - 1)) == L.fz - 1) {
          float v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            v[i] = racc[i];
            racc[i] = 0.f;
          }
          if (L.fy == 2) {
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 16);
          }
          int cnt = 4;
          if (L.fx == 2) {
#pragma unroll
            for (int j = 0; j < 2; ++j) v[j] = v[2 * j] + v[2 * j + 1];
            cnt = 2;
          }
          if (L.fy == 1 || (s.y & 1) == 0) {
            float* dst = C.f + (long long)(zr >> (L.fz - 1)) * C.g.nxy + (long long)(s.y >> (L.fy - 1)) * C.g.nx +
                         (s.x >> (L.fx - 1));
            for (int j = 0; j < cnt; ++j) dst[j] = v[j] * scale;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        em2[i] = em1[i];
        em1[i] = e0[i];
      }
    }
    cp_wait<0>();
  }
  sched_finish(ts);
}

// Prolongation sweep and second post-sweep fused, on the interior planes of the
// split finest level (FP32, eps = 1, whole tiles, every coarsening factor 2).
// Three fields are kept apart: the pre-smoothed correction L.e (read), e' in
// L.et and the result zout -- reading e with a ring while writing the result
// in place would race with the neighbouring tiles.
//   e' = u + w2 D^-1 (f - A u),  u = e + P e_c      (k_mg_post1)
//   e'' = e' + w1 D^-1 (f - A e')                   (k_mg_post2, with r.z)
// in one pass: e, e_c and f read, e'' written, instead of writing e' and
// reading it and f again.  The second sweep needs e' at six neighbours and e'
// needs u at six, so a tile stages e and f with a two-cell ring and the coarse
// parents of that box, and forms e' on its columns and the one-cell ring, one
// plane ahead of e''.  e' of the plane below or above the tile is formed too,
// except next to a face slab (planes 1 and nz - 2), where it is the face-slab
// prolongation sweep's output (that launch runs first); e' of planes 2 and
// nz - 3 is written for the face-slab second sweep (which runs after this one
// and sums the r.z tile partials of both launches: this one's first).
constexpr int PP_D = 1;                    // planes of cp.async look-ahead
constexpr int PP_NS = PP_D + 3;            // staged planes: w, w + 1, w + 2 in use, PP_D in flight
constexpr int PP_CW = 40, PP_CH = 10;      // coarse box: x0/2 - 4 .. x0/2 + 35, y0/2 - 1 .. y0/2 + 8
constexpr int PP_STAGE = 2 * PRR_STAGE + PP_CW * PP_CH;   // e, f, parents
constexpr size_t pp_smem_bytes() { return (size_t)(PP_NS * PP_STAGE + 2 * PRR_EPLANE) * sizeof(float); }

__global__ void __launch_bounds__(MTX* MTY, 3) k_mg_pp(MgView<float> L, MgView<float> C, float* zout,
                                                       double* part, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  static_assert(MTX == 16 && MTY == 16, "tiles of 64 x 16 columns, four cells a thread");
  static_assert(PP_CW * PP_CH / 4 <= MTX * MTY, "one coarse vector a thread");
  if (S->done) return;
  float* const stg = reinterpret_cast<float*>(smem);
  float* const eb = stg + PP_NS * PP_STAGE;
  const int nx = L.g.nx, ny = L.g.ny, nz = L.g.nz, cnx = C.g.nx, cny = C.g.ny;
  const long long nxy = L.g.nxy, cnxy = C.g.nxy;
  const float inv_int = mg_inv_int(L);
  const float w2d = rn_mul(mg_omega2<float>(), inv_int), w1d = rn_mul(mg_omega1<float>(), inv_int);
  const float ax = L.ax, ay = L.ay, az = L.az;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * MTX;
  const int c0 = 4 + 4 * tx;
  const int so = (ty + 2) * PRR_RS + c0;   // own vector in a staged field plane
  const int eo = (ty + 1) * PRR_RS + c0;   // own vector in an e' plane
  int rr = -1, re = -1, rc = -1;           // ring cell of threads 0 .. 159
  if (tid < 64) { rr = 1; re = 0; rc = 4 + tid; }
  else if (tid < 128) { rr = 18; re = 17; rc = 4 + tid - 64; }
  else if (tid < 144) { rr = 2 + tid - 128; re = 1 + tid - 128; rc = 3; }
  else if (tid < 160) { rr = 2 + tid - 144; re = 1 + tid - 144; rc = 68; }
  auto load4 = [](const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  };
  Acc<float> arz;
  const TileSched ts{&S->sched_next, &S->sched_done, L.mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < L.mc.ntiles; t = sched_next(ts, &tile_slot)) {
    const TileGeo<MTX, MTY, 4> s = tile_geo<MTX, MTY, 4>(L.g, t, L.mc);
    const int x0 = s.x - 4 * tx, y0 = s.y - ty, z0 = s.z0, nt = s.z1 - s.z0;
    auto row_of = [&](int r) {
      int y = y0 - 2 + r;
      y += y < 0 ? ny : 0;
      y -= y >= ny ? ny : 0;
      return y * nx;
    };
    // this thread's copies of a staged plane: e and f vectors tid, tid + 256
    // (of 320), ring cell tid (of 80), and coarse vector tid (of 100)
    const int sv0 = (tid >> 4) * PRR_RS + 4 + 4 * (tid & 15), gv0 = row_of(tid >> 4) + x0 + 4 * (tid & 15);
    const int i1 = tid + MTX * MTY;
    const bool has1 = i1 < PRR_RH * 16;
    const int sv1 = has1 ? (i1 >> 4) * PRR_RS + 4 + 4 * (i1 & 15) : 0;
    const int gv1 = has1 ? row_of(i1 >> 4) + x0 + 4 * (i1 & 15) : 0;
    const bool hasr = tid < PRR_RH * 4;
    int svr = 0, gvr = 0;
    if (hasr) {
      const int r = tid >> 2, k = tid & 3;
      int x = k < 2 ? x0 - 2 + k : x0 + 62 + k;
      x += x < 0 ? nx : 0;
      x -= x >= nx ? nx : 0;
      svr = r * PRR_RS + (k < 2 ? 2 + k : 66 + k);
      gvr = row_of(r) + x;
    }
    const bool hasc = tid < PP_CW * PP_CH / 4;
    int svc = 0, gvc = 0;
    if (hasc) {
      const int r = tid / (PP_CW / 4), v = tid % (PP_CW / 4);
      int y = y0 / 2 - 1 + r;
      y += y < 0 ? cny : 0;
      y -= y >= cny ? cny : 0;
      int x = x0 / 2 - 4 + 4 * v;          // whole 16-byte vectors: x0 / 2 is a multiple of 32
      x += x < 0 ? cnx : 0;
      x -= x >= cnx ? cnx : 0;
      svc = r * PP_CW + 4 * v;
      gvc = y * cnx + x;
    }
    // e, f and the parents of plane w (z = z0 - 2 + w) into stage w mod PP_NS
    auto issue = [&](int w) {
      if (w <= nt + 3) {
        const int z = z0 - 2 + w;
        float* st = stg + (w % PP_NS) * PP_STAGE;
        const float* se = L.e + (long long)z * nxy;
        const float* sf = L.f + (long long)z * nxy;
        cp_async<16>(st + sv0, se + gv0);
        cp_async<16>(st + PRR_STAGE + sv0, sf + gv0);
        if (has1) {
          cp_async<16>(st + sv1, se + gv1);
          cp_async<16>(st + PRR_STAGE + sv1, sf + gv1);
        }
        if (hasr) {
          cp_async<4>(st + svr, se + gvr);
          cp_async<4>(st + PRR_STAGE + svr, sf + gvr);
        }
        if (hasc) cp_async<16>(st + 2 * PRR_STAGE + svc, C.e + (long long)(z >> 1) * cnxy + gvc);
      }
      cp_commit();
    };
    // u = e + P e_c at staged cell (r, c) of a stage: the parent of column c is
    // coarse column 2 + c / 2 of the box, of row r the coarse row r / 2
    auto u_at = [&](const float* st, int r, int c) -> float {
      return st[r * PRR_RS + c] + st[2 * PRR_STAGE + (r >> 1) * PP_CW + 2 + (c >> 1)];
    };
    // e' at staged cell (r, c) from the stages of the planes below, at and above it
    auto ep_at = [&](const float* sm, const float* sc, const float* sp, int r, int c) -> float {
      const float uc = u_at(sc, r, c);
      const float Au = apply_int(uc, u_at(sc, r, c - 1), u_at(sc, r, c + 1), u_at(sc, r - 1, c), u_at(sc, r + 1, c),
                                 u_at(sm, r, c), u_at(sp, r, c), ax, ay, az);
      return rn_fma(w2d, rn_sub(sc[PRR_STAGE + r * PRR_RS + c], Au), uc);
    };
    float em2[4], e0[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) em2[i] = e0[i] = 0.f;
    float em1[4] = {0.f, 0.f, 0.f, 0.f};
    arz = Acc<float>();
    for (int w = 0; w < PP_D + 2; ++w) issue(w);
    for (int u = 0; u <= nt + 1; ++u) {
      cp_wait<PP_D - 1>();                 // planes u .. u + 2 of this thread have landed
      __syncthreads();                     // ... and of every thread
      issue(u + PP_D + 2);
      const float* sm = stg + (u % PP_NS) * PP_STAGE;
      const float* sc = stg + ((u + 1) % PP_NS) * PP_STAGE;
      const float* sp = stg + ((u + 2) % PP_NS) * PP_STAGE;
      float* ebu = eb + (u & 1) * PRR_EPLANE;
      const int z = z0 - 1 + u;
      if (z == 1 || z == nz - 2) {
        load4(L.et + (long long)z * nxy + s.xy, e0);
      } else {
        // e' on the own vector: u = e + parent on the vector, its rows above and
        // below, the planes below and above, and the two cells beside it
        const int r = ty + 2, pc = 4 + 2 * tx;          // parent columns of the vector: pc, pc + 1
        const float* pb = sc + 2 * PRR_STAGE;
        float ec[4], eym[4], eyp[4], ezm[4], ezp[4], fc[4];
        load4(sc + so, ec);
        load4(sc + so - PRR_RS, eym);
        load4(sc + so + PRR_RS, eyp);
        load4(sm + so, ezm);
        load4(sp + so, ezp);
        load4(sc + PRR_STAGE + so, fc);
        auto par2 = [](const float* q) { return *reinterpret_cast<const float2*>(q); };
        const float2 pC = par2(pb + (r >> 1) * PP_CW + pc), pYM = par2(pb + ((r - 1) >> 1) * PP_CW + pc),
                     pYP = par2(pb + ((r + 1) >> 1) * PP_CW + pc),
                     pZM = par2(sm + 2 * PRR_STAGE + (r >> 1) * PP_CW + pc),
                     pZP = par2(sp + 2 * PRR_STAGE + (r >> 1) * PP_CW + pc);
        const float uL = sc[so - 1] + pb[(r >> 1) * PP_CW + pc - 1];
        const float uR = sc[so + 4] + pb[(r >> 1) * PP_CW + pc + 2];
        float uc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) uc[i] = ec[i] + (i < 2 ? pC.x : pC.y);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float ym = eym[i] + (i < 2 ? pYM.x : pYM.y), yp = eyp[i] + (i < 2 ? pYP.x : pYP.y);
          const float zm = ezm[i] + (i < 2 ? pZM.x : pZM.y), zp = ezp[i] + (i < 2 ? pZP.x : pZP.y);
          const float Au = apply_int(uc[i], i == 0 ? uL : uc[i - 1], i == 3 ? uR : uc[i + 1], ym, yp, zm, zp, ax, ay, az);
          e0[i] = rn_fma(w2d, rn_sub(fc[i], Au), uc[i]);
        }
      }
      if (u >= 1 && u <= nt) {
        *reinterpret_cast<float4*>(ebu + eo) = make_float4(e0[0], e0[1], e0[2], e0[3]);
        if (rc >= 0) ebu[re * PRR_RS + rc] = ep_at(sm, sc, sp, rr, rc);
        if (z == 2 || z == nz - 3)         // handed to the face-slab second sweep
          *reinterpret_cast<float4*>(L.et + (long long)z * nxy + s.xy) = make_float4(e0[0], e0[1], e0[2], e0[3]);
      }
      if (u >= 2) {                        // e'' of plane z - 1
        const float* ebm = eb + ((u - 1) & 1) * PRR_EPLANE;
        float ec[4], eym[4], eyp[4], fv[4], ev[4];
        load4(ebm + eo, ec);
        load4(ebm + eo - PRR_RS, eym);
        load4(ebm + eo + PRR_RS, eyp);
        load4(sm + PRR_STAGE + so, fv);    // f of plane z - 1: stage u
        float el = __shfl_up_sync(0xffffffffu, ec[3], 1), er = __shfl_down_sync(0xffffffffu, ec[0], 1);
        if (tx == 0) el = ebm[eo - 1];
        if (tx == MTX - 1) er = ebm[eo + 4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float Ae = apply_int(ec[i], i == 0 ? el : ec[i - 1], i == 3 ? er : ec[i + 1], eym[i], eyp[i], em2[i],
                                     e0[i], ax, ay, az);
          ev[i] = rn_fma(w1d, rn_sub(fv[i], Ae), ec[i]);
          arz.add(fv[i], ev[i]);
        }
        arz.run();
        *reinterpret_cast<float4*>(zout + (long long)(z - 1) * nxy + s.xy) = make_float4(ev[0], ev[1], ev[2], ev[3]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        em2[i] = em1[i];
        em1[i] = e0[i];
      }
    }
    cp_wait<0>();
    double v[1] = {arz.value()};
    tile_partials<1, MTX * MTY>(v, part, t);
  }
  sched_finish(ts);
}

// Prolongation + correction fused into the first post-smoothing sweep: the
// stencil field is e + e_c(parent), the parents staged with the fine planes
// and combined with e at each of the seven cells.
template <typename T, int VX, bool EPS, bool INT = false>
__global__ void __launch_bounds__(MTX* MTY, (sizeof(T) == 4 && !EPS) ? 3 : 2) k_mg_post1(MgView<T> L, MgView<T> C, Scalars* S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  if (S->done) return;
  constexpr int NH = EPS ? 2 : 1;          // e (, eps); the parents come as field NH
  constexpr int NO = EPS ? 2 : 1;          // f (, 1/diag)
  const T om = mg_omega2<T>(), inv_int = mg_inv_int(L);
  const T* hsrc[NH];
  hsrc[0] = L.e;
  if constexpr (EPS) hsrc[1] = L.eps;
  const T* osrc[NO];
  osrc[0] = L.f;
  if constexpr (EPS) osrc[1] = L.invd;
  const ParentSrc<T> par{C.e, L.fx, L.fy, L.fz, C.g.nx, C.g.nxy};
  TileGeo<MTX, MTY, VX> s;
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, NH + 1>>& sr, const T (&o)[NO], const bool bt) -> T {
    Stencil7<T> st;
    st.c = sr.c.v[0] + sr.c.v[NH];
    st.xm = sr.xm.v[0] + sr.xm.v[NH];
    st.xp = sr.xp.v[0] + sr.xp.v[NH];
    st.ym = sr.ym.v[0] + sr.ym.v[NH];
    st.yp = sr.yp.v[0] + sr.yp.v[NH];
    st.zm = sr.zm.v[0] + sr.zm.v[NH];
    st.zp = sr.zp.v[0] + sr.zp.v[NH];
    st.zb = sr.zb;
    st.za = sr.za;
    const bool B = bt;
    const int dlo = (B && st.zb < 0) ? (int)L.tlo[xy] : 0;
    const int dhi = (B && st.za < 0) ? (int)L.thi[xy] : 0;
    if constexpr (EPS) {
      Stencil7<EpsVal<T>> se = pick_eps(sr, 0, 1);
      se.c.v = st.c;
      se.xm.v = st.xm;
      se.xp.v = st.xp;
      se.ym.v = st.ym;
      se.yp.v = st.yp;
      se.zm.v = st.zm;
      se.zp.v = st.zp;
      const T Ae = apply_aniso_eps(se, dlo, dhi, L.ax, L.ay, L.az, bt);
      return st.c + om * o[1] * (o[0] - Ae);
    } else {
      const T Ae = apply_aniso(st, dlo, dhi, L.ax, L.ay, L.az, bt);
      return st.c + om * mg_inv_bt(L, xy, z, inv_int, bt) * (o[0] - Ae);
    }
  };
  auto post = [&](int z, const T (&ov)[VX]) { store_n<T, VX>(L.et + (long long)z * L.g.nxy + s.xy, ov); };
  const TileSched ts{&S->sched_next, &S->sched_done, L.mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < L.mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(L.g, t, L.mc);
    march_direct<T, T, MTX, MTY, VX, NH, NO, MG_D, 1, INT>(L.g, s, smem, hsrc, osrc, emit, post, par);
  }
  sched_finish(ts);
}

// Last post-smoothing sweep.  On the finest level (LAST) it also forms
// r.z (f = r, e = z): the last block sets beta = (r.z)_new / (r.z)_old.
template <typename T, bool LAST, int VX, bool EPS, bool INT = false>
__global__ void __launch_bounds__(MTX* MTY, (sizeof(T) == 4 && !EPS) ? (INT ? 5 : (LAST ? 3 : 4)) : 2) k_mg_post2(MgView<T> L, double* part, Scalars* S,
                                                                                                long long pofs,
                                                                                                long long ptot) {
  // pofs, ptot (finest level): this launch's tile partials go to part[pofs + t]; the
  // last block sums part[0 .. ptot) (a fused interior launch wrote the first pofs)
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long tile_slot;
  if (S->done) return;
  constexpr int NH = EPS ? 2 : 1;          // et (, eps)
  constexpr int NO = EPS ? 2 : 1;          // f (, 1/diag)
  const T om = mg_omega1<T>(), inv_int = mg_inv_int(L);
  const T* hsrc[NH];
  hsrc[0] = L.et;
  if constexpr (EPS) hsrc[1] = L.eps;
  const T* osrc[NO];
  osrc[0] = L.f;
  if constexpr (EPS) osrc[1] = L.invd;
  Acc<T> arz;
  TileGeo<MTX, MTY, VX> s;
  auto emit = [&](int xy, int z, const Stencil7<Raw<T, NH>>& sr, const T (&o)[NO], const bool bt) -> T {
    const bool B = bt;
    const int dlo = (B && sr.zb < 0) ? (int)L.tlo[xy] : 0;
    const int dhi = (B && sr.za < 0) ? (int)L.thi[xy] : 0;
    T e;
    if constexpr (EPS) {
      const T Ae = apply_aniso_eps(pick_eps(sr, 0, 1), dlo, dhi, L.ax, L.ay, L.az, bt);
      e = sr.c.v[0] + om * o[1] * (o[0] - Ae);
    } else {
      const Stencil7<T> st = pick(sr, 0);
      const T Ae = apply_aniso(st, dlo, dhi, L.ax, L.ay, L.az, bt);
      e = st.c + om * mg_inv_bt(L, xy, z, inv_int, bt) * (o[0] - Ae);
    }
    if (LAST) arz.add(o[0], e);
    return e;
  };
  auto post = [&](int z, const T (&ov)[VX]) {
    if (LAST) arz.run();
    store_n<T, VX>(L.e + (long long)z * L.g.nxy + s.xy, ov);
  };
  const TileSched ts{&S->sched_next, &S->sched_done, L.mc.ntiles};
  for (long long t = sched_first(ts, &tile_slot); t < L.mc.ntiles; t = sched_next(ts, &tile_slot)) {
    s = tile_geo<MTX, MTY, VX>(L.g, t, L.mc);
    arz = Acc<T>();
    march_direct<T, T, MTX, MTY, VX, NH, NO, MG_D, 0, INT>(L.g, s, smem, hsrc, osrc, emit, post);
    if (LAST) {
      double v[1] = {arz.value()};
      tile_partials<1, MTX * MTY>(v, part + pofs, t);
    }
  }
  sched_finish(ts);
  if (!LAST) return;
  if (last_block<MTX * MTY>(&S->ticket)) {
    double out[1];
    gather_partials<1, MTX * MTY>(part, ptot, out);
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

// Sum over a warp with every lane receiving the total.  The butterfly adds
// the same two partial sums in every lane of a pair, so all lanes end with
// bitwise the same value (addition is commutative).
__device__ __forceinline__ double warp_sum_all(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Barrier of the first nw warps of the block (named barrier 1; one warp:
// a warp barrier).
__device__ __forceinline__ void warps_sync(int nw) {
  if (nw == 1) __syncwarp();
  else asm volatile("bar.sync 1, %0;\n" ::"r"(nw * 32) : "memory");
}

// Sum over the first nw warps, the same value in every thread (fixed order).
__device__ __forceinline__ double warps_sum(double v, int nw, double* red) {
  v = warp_sum_all(v);
  if (nw == 1) return v;
  warps_sync(nw);                  // red[] may still be read from the previous sum
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  warps_sync(nw);
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Jacobi-preconditioned conjugate gradients on the coarsest level, FP64, one
// cell per thread in the first ceil(n / 32) warps of the block (the other
// warps return at once; the caller's next __syncthreads joins them), to a
// relative residual of 1e-12.  The diagonal scaling matters where a
// permittivity field makes the coarse operator's diagonal vary by orders of
// magnitude.  With no electrode the level is singular: the right-hand side and
// the solution are projected to zero mean.
// A coarsest level that is one z column (1 x 1 x nz: the in-plane faces join a
// cell to itself and drop out) with non-periodic z is tridiagonal: solved
// directly by the Thomas algorithm (forward elimination, back substitution)
// in FP64 by one thread, with scratch for 2 nz values.  Jacobi-PCG on such a
// column (a film whose z axis stops coarsening, as under air layers) needed up
// to nz iterations of three block reductions each.
template <typename T>
__device__ __forceinline__ void coarse_column_solve(const MgView<T>& C, const T* cf, T* ce, double* scratch) {
  const int n = C.g.nz;
  const double az = C.az;
  double* cpr = scratch;                        // c'_z
  double* dpr = scratch + n;                    // d'_z
  auto w = [&](int z, int nb) -> double {       // face weight between cells z and nb
    if (!C.eps) return 1.0;
    const double ec = (double)C.eps[z], en = (double)C.eps[nb];
    return 2.0 * ec * en / (ec + en);
  };
  double prev_c = 0.0, prev_d = 0.0;
  for (int z = 0; z < n; ++z) {
    const double wm = z > 0 ? w(z, z - 1) : 0.0, wp = z < n - 1 ? w(z, z + 1) : 0.0;
    const double wd = C.eps ? (double)C.eps[z] : 1.0;
    double diag = az * (wm + wp);
    if (z == 0 && C.tlo[0]) diag += az * 2.0 * wd;
    if (z == n - 1 && C.thi[0]) diag += az * 2.0 * wd;
    const double lower = -az * wm, upper = -az * wp;
    const double m = diag - lower * prev_c;
    prev_c = upper / m;
    prev_d = ((double)cf[z] - lower * prev_d) / m;
    cpr[z] = prev_c;
    dpr[z] = prev_d;
  }
  double x = 0.0;
  for (int z = n - 1; z >= 0; --z) {
    x = dpr[z] - cpr[z] * x;
    ce[z] = (T)x;
  }
}

template <typename T>
__device__ __forceinline__ void mg_coarse_solve(const MgView<T>& C, const T* cf, T* ce, int singular, double* ps,
                                                double* red) {
  if (C.g.nx == 1 && C.g.ny == 1 && !C.g.periodic_z && !singular && 2 * C.g.nz <= MG_MAX_COARSE &&
      (C.tlo[0] || C.thi[0])) {
    if (threadIdx.x == 0) coarse_column_solve(C, cf, ce, ps);
    return;
  }
  const int n = (int)C.g.n, tid = threadIdx.x;
  const int nw = (n + 31) >> 5;
  if (tid >= nw * 32) return;
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
  // face weights: 1, or the harmonic mean of the cells' eps (electrode: 2 eps_c)
  double wxm = 1.0, wxp = 1.0, wym = 1.0, wyp = 1.0, wzm = 1.0, wzp = 1.0, wd = 1.0;
  if (C.eps && on) {
    const double ec = (double)C.eps[tid];
    auto hm = [&](int nb) { const double en = (double)C.eps[nb]; return 2.0 * ec * en / (ec + en); };
    wxm = hm(xm);
    wxp = hm(xp);
    wym = hm(ym);
    wyp = hm(yp);
    wzm = zm >= 0 ? hm(zm) : 0.0;
    wzp = zp >= 0 ? hm(zp) : 0.0;
    wd = ec;
  }
  auto apply = [&](const double* v) -> double {
    const double c = v[tid];
    double sz = 0.0;
    if (zm >= 0) sz += wzm * (c - v[zm]);
    else if (dlo) sz += 2.0 * wd * c;
    if (zp >= 0) sz += wzp * (c - v[zp]);
    else if (dhi) sz += 2.0 * wd * c;
    return ax * (wxm * (c - v[xm]) + wxp * (c - v[xp])) + ay * (wym * (c - v[ym]) + wyp * (c - v[yp])) + az * sz;
  };
  double dg = ax * (wxm + wxp) + ay * (wym + wyp);
  dg += az * ((zm >= 0 ? wzm : (dlo ? 2.0 * wd : 0.0)) + (zp >= 0 ? wzp : (dhi ? 2.0 * wd : 0.0)));
  const double dinv = (on && dg > 0.0) ? 1.0 / dg : 0.0;
  double b = on ? (double)cf[tid] : 0.0;
  if (singular) b -= warps_sum(b, nw, red) / n;
  double xv = 0.0, r = b;
  const double bb = warps_sum(r * r, nw, red);
  if (bb > 0.0) {
    double zv = r * dinv;
    double p = zv;
    double rz = warps_sum(r * zv, nw, red);
    for (int it = 0; it < 4 * n + 20; ++it) {
      warps_sync(nw);              // ps[] may still be read from the previous iteration
      if (on) ps[tid] = p;
      warps_sync(nw);
      const double q = on ? apply(ps) : 0.0;
      const double pq = warps_sum(p * q, nw, red);
      if (!(pq > 0.0)) break;
      const double a = rz / pq;
      xv += a * p;
      r -= a * q;
      const double rrn = warps_sum(r * r, nw, red);
      if (rrn <= 1e-24 * bb) break;
      zv = r * dinv;
      const double rzn = warps_sum(r * zv, nw, red);
      p = zv + (rzn / rz) * p;
      rz = rzn;
    }
  }
  if (singular) xv -= warps_sum(on ? xv : 0.0, nw, red) / n;
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

// Column walk of a small level: thread t of the block takes the columns t,
// t + blockDim.x, ... of the nx x ny plane and walks them along z, so the
// in-plane neighbour offsets, the face masks and the boundary diagonals are
// formed once per column instead of from the linear index at every cell.
// When the level has fewer columns than the block has threads (a deep, narrow
// level such as 8 x 8 x 37), each column is cut into z chunks walked by
// different threads.  body(o, x, y, z0, z1) walks planes [z0, z1).
struct TailCol {
  int xy;                   // the column (y nx + x)
  int dxm, dxp, dym, dyp;   // offsets of the in-plane neighbours (periodic wrap)
  int dlo, dhi;             // electrode masks of the column's z faces
};

// Quotient of small non-negative ints (a < 2^22) by d >= 1 through a float
// reciprocal formed once per level: the rounded product is at most one off,
// and one compare on each side corrects it.  The column walks divide by the
// level's sizes at every item of every phase; an integer division there cost
// more than the arithmetic of the cell it located.
struct SmallDiv {
  int d;
  float r;
  __device__ __forceinline__ explicit SmallDiv(int d_) : d(d_), r(1.0f / (float)d_) {}
  __device__ __forceinline__ int operator()(int a) const {
    int q = (int)((float)a * r);
    if (q * d > a) --q;
    else if ((q + 1) * d <= a) ++q;
    return q;
  }
};

template <typename T, class Body>
__device__ __forceinline__ void tail_cols(const MgView<T>& L, Body body) {
  const int nx = L.g.nx, ny = L.g.ny, nxy = (int)L.g.nxy, nz = L.g.nz;
  const int nch = nxy >= (int)blockDim.x ? 1 : min(nz, (int)blockDim.x / nxy);   // z chunks per column
  const SmallDiv by_nxy(nxy), by_nch(nch), by_nx(nx);
  for (int item = threadIdx.x; item < nxy * nch; item += blockDim.x) {
    const int ch = nch > 1 ? by_nxy(item) : 0, col = item - ch * nxy;
    const int z0 = nch > 1 ? by_nch(ch * nz) : 0, z1 = nch > 1 ? by_nch((ch + 1) * nz) : nz;
    const int y = by_nx(col), x = col - y * nx;
    TailCol o;
    o.xy = col;
    o.dxm = x == 0 ? nx - 1 : -1;
    o.dxp = x == nx - 1 ? -(nx - 1) : 1;
    o.dym = y == 0 ? (ny - 1) * nx : -nx;
    o.dyp = y == ny - 1 ? -(ny - 1) * nx : nx;
    o.dlo = L.g.periodic_z ? 0 : (int)L.tlo[col];
    o.dhi = L.g.periodic_z ? 0 : (int)L.thi[col];
    body(o, x, y, z0, z1);
  }
}

// 1/diag at plane z of a column (eps = 1); iint: the interior value.
template <typename T>
__device__ __forceinline__ T col_inv(const MgView<T>& L, const TailCol& o, int z, T iint) {
  const int nz = L.g.nz;
  if (L.g.periodic_z || (z > 0 && z < nz - 1)) return iint;
  int cz = 2;
  if (z == 0) cz += 2 * o.dlo - 1;
  if (z == nz - 1) cz += 2 * o.dhi - 1;
  return T(1) / (T(2) * L.ax + T(2) * L.ay + T(cz) * L.az);
}

// (A v) at plane z of a column and 1/diag there: the same operator, face
// order and diagonal as the sweep kernels (per-direction 1/h^2; with eps the
// harmonic-mean face weights and the precomputed 1/diag; iint: the interior
// 1/diag with eps = 1, so only the face planes divide).
template <typename T>
__device__ __forceinline__ T col_apply(const MgView<T>& L, const T* v, const TailCol& o, int z, T& inv, T iint) {
  const int nz = L.g.nz, nxy = (int)L.g.nxy;
  const int c = z * nxy + o.xy;
  const T vc = v[c];
  const int zm = z > 0 ? c - nxy : (L.g.periodic_z ? c + (nz - 1) * nxy : -1);
  const int zp = z < nz - 1 ? c + nxy : (L.g.periodic_z ? c - (nz - 1) * nxy : -1);
  if (L.eps) {
    const T ec = L.eps[c];
    auto face = [&](int nb) { return hmean2(ec, L.eps[nb]) * (vc - v[nb]); };
    const T sx = face(c + o.dxm) + face(c + o.dxp);
    const T sy = face(c + o.dym) + face(c + o.dyp);
    T sz = T(0);
    if (zm >= 0) sz += face(zm);
    else if (o.dlo) sz += T(2) * ec * vc;
    if (zp >= 0) sz += face(zp);
    else if (o.dhi) sz += T(2) * ec * vc;
    inv = L.invd[c];
    return L.ax * sx + L.ay * sy + L.az * sz;
  }
  const T sx = (vc - v[c + o.dxm]) + (vc - v[c + o.dxp]);
  const T sy = (vc - v[c + o.dym]) + (vc - v[c + o.dyp]);
  T sz = T(0);
  if (zm >= 0) sz += vc - v[zm];
  else if (o.dlo) sz += T(2) * vc;
  if (zp >= 0) sz += vc - v[zp];
  else if (o.dhi) sz += T(2) * vc;
  inv = col_inv(L, o, z, iint);
  return L.ax * sx + L.ay * sy + L.az * sz;
}

// The V-cycle below level k0 (all levels small) in one block: per level two
// pre-smoothing sweeps from zero, the residual, its restriction, the coarsest
// solve, then prolongation and two post-smoothing sweeps, each phase a walk
// over the level's columns followed by a block barrier.  Same operators,
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
    const int nxy = (int)L.g.nxy, nz = L.g.nz;
    const T iint = mg_inv_int(L);
    tail_cols(L, [&](const TailCol& o, int, int, int z0, int z1) {
      for (int z = z0; z < z1; ++z) {
        const int c = z * nxy + o.xy;
        const T inv = L.eps ? L.invd[c] : col_inv(L, o, z, iint);
        et[c] = om1 * inv * f[c];
      }
    });
    __syncthreads();
    tail_cols(L, [&](const TailCol& o, int, int, int z0, int z1) {
      for (int z = z0; z < z1; ++z) {
        T inv;
        const T Ae = col_apply(L, et, o, z, inv, iint);
        const int c = z * nxy + o.xy;
        e[c] = et[c] + om2 * inv * (f[c] - Ae);
      }
    });
    __syncthreads();
    // the residual (into e_tmp, free again), then the sum of each coarse
    // cell's children in the order dz, dy, dx
    tail_cols(L, [&](const TailCol& o, int, int, int z0, int z1) {
      for (int z = z0; z < z1; ++z) {
        T inv;
        const T Ae = col_apply(L, e, o, z, inv, iint);
        const int c = z * nxy + o.xy;
        et[c] = f[c] - Ae;
      }
    });
    __syncthreads();
    const T scale = T(1) / T(L.fx * L.fy * L.fz);
    T* fc = F(k + 1);
    const int ncxy = (int)C.g.nxy;
    tail_cols(C, [&](const TailCol& o, int X, int Y, int z0, int z1) {
      for (int Z = z0; Z < z1; ++Z) {
        T acc = T(0);
        for (int dz = 0; dz < L.fz; ++dz)
          for (int dy = 0; dy < L.fy; ++dy)
            for (int dx = 0; dx < L.fx; ++dx)
              acc += et[((Z * L.fz + dz) * L.g.ny + Y * L.fy + dy) * L.g.nx + X * L.fx + dx];
        fc[Z * ncxy + o.xy] = acc * scale;
      }
    });
    __syncthreads();
  }
  mg_coarse_solve(t.lv[t.nl - 1], F(t.nl - 1), E(t.nl - 1), singular, ps, red);
  __syncthreads();
  for (int k = t.nl - 2; k >= 0; --k) {
    const MgView<T>& L = t.lv[k];
    const MgView<T>& C = t.lv[k + 1];
    T *f = F(k), *e = E(k), *et = ET(k);
    const T* ec = E(k + 1);
    const int nxy = (int)L.g.nxy, nz = L.g.nz;
    const T iint = mg_inv_int(L);
    tail_cols(L, [&](const TailCol& o, int x, int y, int z0, int z1) {
      const int pxy = (y >> (L.fy - 1)) * C.g.nx + (x >> (L.fx - 1));
      for (int z = z0; z < z1; ++z) e[z * nxy + o.xy] += ec[(z >> (L.fz - 1)) * (int)C.g.nxy + pxy];
    });
    __syncthreads();
    tail_cols(L, [&](const TailCol& o, int, int, int z0, int z1) {
      for (int z = z0; z < z1; ++z) {
        T inv;
        const T Ae = col_apply(L, e, o, z, inv, iint);
        const int c = z * nxy + o.xy;
        et[c] = e[c] + om2 * inv * (f[c] - Ae);
      }
    });
    __syncthreads();
    T* eo = k == 0 ? t.lv[0].e : e;                    // the first level's result goes to global memory
    tail_cols(L, [&](const TailCol& o, int, int, int z0, int z1) {
      for (int z = z0; z < z1; ++z) {
        T inv;
        const T Ae = col_apply(L, et, o, z, inv, iint);
        const int c = z * nxy + o.xy;
        eo[c] = et[c] + om1 * inv * (f[c] - Ae);
      }
    });
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

// A level split by mg_split_level: the view of its interior planes (tiles of
// the level's depth over [b, nz - b)) and of its two face slabs of b planes.
template <typename T>
static bool split_views(const MgView<T>& lv, MgView<T>& vi, MgView<T>& vb) {
  if (!lv.split) return false;
  constexpr int b = MG_SPLIT_B;
  const long long cols = (long long)lv.mc.tiles_x * lv.mc.tiles_y;
  vi = lv;
  vi.mc.zlo = b;
  vi.mc.zcut = b;
  vi.mc.zskip = 0;
  vi.mc.ntiles = cols * ((lv.g.nz - 2 * b + lv.mc.tz - 1) / lv.mc.tz);
  vb = lv;
  vb.mc.tz = b;
  vb.mc.zlo = 0;
  vb.mc.zcut = 0;
  vb.mc.zskip = lv.g.nz - 2 * b;
  vb.mc.ntiles = cols * 2;
  return true;
}

template <typename T, int VX, bool E, bool I>
static void pre_l(const LaunchCfg& L, const MgView<T>& lv, Scalars* S) {
  static bool f = false;
  static int res = 0;
  const size_t bytes = MgPipeD0<T, VX, E>::bytes();
  smem_once(k_mg_pre<T, VX, E, I>, bytes, f);
  const int grid = mg_grid(k_mg_pre<T, VX, E, I>, bytes, lv.mc.ntiles, res);
  k_mg_pre<T, VX, E, I><<<grid, dim3(MTX, MTY), bytes, L.stream>>>(lv, S);
}
template <typename T, int VX, bool E>
static int pre_v(const LaunchCfg& L, const MgView<T>& lv, Scalars* S) {
  MgView<T> vi, vb;
  if (!split_views(lv, vi, vb)) {
    pre_l<T, VX, E, false>(L, lv, S);
    return 1;
  }
  pre_l<T, VX, E, true>(L, vi, S);
  pre_l<T, VX, E, false>(L, vb, S);
  return 2;
}
// (the residual's face code costs it no registers: never split)
template <typename T, int VX, bool E>
static int rr_v(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  static bool f = false;
  static int res = 0;
  const size_t bytes = MgPipeR<T, VX, E>::bytes();
  smem_once(k_mg_rr<T, VX, E>, bytes, f);
  const int grid = mg_grid(k_mg_rr<T, VX, E>, bytes, lv.mc.ntiles, res);
  k_mg_rr<T, VX, E><<<grid, dim3(MTX, MTY), bytes, L.stream>>>(lv, cv, S);
  return 1;
}
// The fused pre-smoother + residual on a split FP32 level without eps and with
// whole tiles: face-slab pre-smoother, fused interior, face-slab residual
// (3 launches, as the split pre-smoother plus the residual).  0: not eligible.
template <typename T>
static int prr_v(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S,
                 const std::function<void(int)>& mark) {
  if constexpr (sizeof(T) != 4) {
    return 0;
  } else {
    MgView<T> vi, vb;
    if (lv.eps || lv.mc.vx != 4 || lv.g.nx % (MTX * 4) != 0 || lv.g.ny % MTY != 0 || !split_views(lv, vi, vb))
      return 0;
    static bool f = false;
    static int res = 0;
    const size_t bytes = prr_smem_bytes();
    smem_once(k_mg_prr, bytes, f);
    pre_l<T, 4, false, false>(L, vb, S);
    mark(0);
    const int grid = mg_grid(k_mg_prr, bytes, vi.mc.ntiles, res);
    k_mg_prr<<<grid, dim3(MTX, MTY), bytes, L.stream>>>(vi, cv, S);
    mark(1);
    rr_v<T, 4, false>(L, vb, cv, S);
    mark(2);
    return 3;
  }
}

// The finest level's prolongation sweep and second post-sweep as face-slab
// prolongation sweep, fused interior, face-slab second sweep (3 launches, as
// the split prolongation sweep plus the unsplit second sweep); lv.e holds the
// pre-smoothed correction, ep receives e', z the result.  0: not eligible.
template <typename T>
static bool pp_ok(const MgView<T>& lv) {
  return sizeof(T) == 4 && lv.split && !lv.eps && lv.mc.vx == 4 && lv.g.nx % (MTX * 4) == 0 && lv.g.ny % MTY == 0 &&
         lv.fx == 2 && lv.fy == 2 && lv.fz == 2;
}

template <typename T, int VX, bool E, bool I>
static void post1_l(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  static bool f = false;
  static int res = 0;
  const size_t bytes = MgPipeP<T, VX, E>::bytes();
  smem_once(k_mg_post1<T, VX, E, I>, bytes, f);
  const int grid = mg_grid(k_mg_post1<T, VX, E, I>, bytes, lv.mc.ntiles, res);
  k_mg_post1<T, VX, E, I><<<grid, dim3(MTX, MTY), bytes, L.stream>>>(lv, cv, S);
}
template <typename T, int VX, bool E>
static int post1_v(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  MgView<T> vi, vb;
  if (!split_views(lv, vi, vb)) {
    post1_l<T, VX, E, false>(L, lv, cv, S);
    return 1;
  }
  post1_l<T, VX, E, true>(L, vi, cv, S);
  post1_l<T, VX, E, false>(L, vb, cv, S);
  return 2;
}
template <typename T, bool LAST, int VX, bool E, bool I>
static void post2_l(const LaunchCfg& L, const MgView<T>& lv, double* part, Scalars* S, long long pofs = 0,
                    long long ptot = -1) {
  static bool f = false;
  static int res = 0;
  const size_t bytes = MgPipeD<T, VX, E>::bytes();
  smem_once(k_mg_post2<T, LAST, VX, E, I>, bytes, f);
  const int grid = mg_grid(k_mg_post2<T, LAST, VX, E, I>, bytes, lv.mc.ntiles, res);
  k_mg_post2<T, LAST, VX, E, I><<<grid, dim3(MTX, MTY), bytes, L.stream>>>(lv, part, S, pofs,
                                                                          ptot < 0 ? lv.mc.ntiles : ptot);
}
// The finest level's second post-sweep also reduces r.z over all its tiles,
// so it is never split.
template <typename T, bool LAST, int VX, bool E>
static int post2_v(const LaunchCfg& L, const MgView<T>& lv, double* part, Scalars* S) {
  MgView<T> vi, vb;
  if (LAST || !split_views(lv, vi, vb)) {
    post2_l<T, LAST, VX, E, false>(L, lv, part, S);
    return 1;
  }
  post2_l<T, LAST, VX, E, true>(L, vi, part, S);
  post2_l<T, LAST, VX, E, false>(L, vb, part, S);
  return 2;
}

constexpr int vec_of(size_t bytes) { return (int)(16 / bytes); }

template <typename T>
int launch_mg_pre(const LaunchCfg& L, const MgView<T>& lv, Scalars* S) {
  constexpr int V = vec_of(sizeof(T));
  if (lv.eps) {
    return lv.mc.vx > 1 ? pre_v<T, V, true>(L, lv, S)
                        : pre_v<T, 1, true>(L, lv, S);
  } else {
    return lv.mc.vx > 1 ? pre_v<T, V, false>(L, lv, S)
                        : pre_v<T, 1, false>(L, lv, S);
  }
}

template <typename T>
int launch_mg_prr(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S,
                  const std::function<void(int)>& mark) {
  return prr_v<T>(L, lv, cv, S, mark);
}

template <typename T>
int launch_mg_rr(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  constexpr int V = vec_of(sizeof(T));
  if (lv.eps) {
    return lv.mc.vx > 1 ? rr_v<T, V, true>(L, lv, cv, S)
                        : rr_v<T, 1, true>(L, lv, cv, S);
  } else {
    return lv.mc.vx > 1 ? rr_v<T, V, false>(L, lv, cv, S)
                        : rr_v<T, 1, false>(L, lv, cv, S);
  }
}

template <typename T>
void launch_mg_coarse(const LaunchCfg& L, const MgView<T>& cv, int singular, Scalars* S) {
  const int threads = ((int)cv.g.n + 31) / 32 * 32;
  k_mg_coarse<T><<<1, threads, 0, L.stream>>>(cv, singular, S);
}

template <typename T>
int launch_mg_post1(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, Scalars* S) {
  constexpr int V = vec_of(sizeof(T));
  if (lv.eps) {
    return lv.mc.vx > 1 ? post1_v<T, V, true>(L, lv, cv, S)
                        : post1_v<T, 1, true>(L, lv, cv, S);
  } else {
    return lv.mc.vx > 1 ? post1_v<T, V, false>(L, lv, cv, S)
                        : post1_v<T, 1, false>(L, lv, cv, S);
  }
}

template <typename T, bool E>
static int post2_e(const LaunchCfg& L, const MgView<T>& lv, int last, double* part, Scalars* S) {
  constexpr int V = vec_of(sizeof(T));
  if (last) {
    return lv.mc.vx > 1 ? post2_v<T, true, V, E>(L, lv, part, S)
                        : post2_v<T, true, 1, E>(L, lv, part, S);
  } else {
    return lv.mc.vx > 1 ? post2_v<T, false, V, E>(L, lv, part, S)
                        : post2_v<T, false, 1, E>(L, lv, part, S);
  }
}

template <typename T>
bool mg_fused_post(const MgView<T>& lv) {
  return pp_ok(lv);
}

template <typename T>
int launch_mg_pp(const LaunchCfg& L, const MgView<T>& lv, const MgView<T>& cv, T* ep, T* z, double* part,
                 Scalars* S, const std::function<void(int)>& mark) {
  if constexpr (sizeof(T) != 4) {
    return 0;
  } else {
    MgView<T> vi, vb;
    if (!pp_ok(lv) || !split_views(lv, vi, vb)) return 0;
    MgView<T> v1 = vb;                     // face slabs: e -> e'
    v1.et = ep;
    post1_l<T, 4, false, false>(L, v1, cv, S);
    mark(0);
    static bool f = false;
    static int res = 0;
    const size_t bytes = pp_smem_bytes();
    smem_once(k_mg_pp, bytes, f);
    MgView<T> vp = vi;                     // interior: e (and e' of the face-adjacent planes) -> z
    vp.et = ep;
    const int grid = mg_grid(k_mg_pp, bytes, vi.mc.ntiles, res);
    k_mg_pp<<<grid, dim3(MTX, MTY), bytes, L.stream>>>(vp, cv, z, part, S);
    mark(1);
    MgView<T> v2 = vb;                     // face slabs: e' -> z, then r.z over both launches' tiles
    v2.et = ep;
    v2.e = z;
    post2_l<T, true, 4, false, false>(L, v2, part, S, vi.mc.ntiles, vi.mc.ntiles + vb.mc.ntiles);
    mark(2);
    return 3;
  }
}

template <typename T>
int launch_mg_post2(const LaunchCfg& L, const MgView<T>& lv, int last, double* part, Scalars* S) {
  return lv.eps ? post2_e<T, true>(L, lv, last, part, S) : post2_e<T, false>(L, lv, last, part, S);
}

// ------------------------------------------------ permittivity of the levels

// Coarse cell permittivity: the mean of its children's.
template <typename T>
__global__ void __launch_bounds__(256) k_mg_eps_restrict(MgView<T> F, MgView<T> C, T* __restrict__ ceps) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const T scale = T(1) / T(F.fx * F.fy * F.fz);
  for (long long cc = blockIdx.x * (long long)blockDim.x + threadIdx.x; cc < C.g.n; cc += stride) {
    const int X = (int)(cc % C.g.nx), Y = (int)((cc / C.g.nx) % C.g.ny), Z = (int)(cc / C.g.nxy);
    T acc = T(0);
    for (int dz = 0; dz < F.fz; ++dz)
      for (int dy = 0; dy < F.fy; ++dy)
        for (int dx = 0; dx < F.fx; ++dx)
          acc += F.eps[((long long)(Z * F.fz + dz) * F.g.ny + Y * F.fy + dy) * F.g.nx + X * F.fx + dx];
    ceps[cc] = acc * scale;
  }
}

// 1/diag of a level's operator with cell permittivities: the face weights
// (harmonic means; an electrode face 2 eps_c) times 1/h^2 per direction.
template <typename T>
__global__ void __launch_bounds__(256) k_mg_invdiag(MgView<T> L, T* __restrict__ invd) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int nx = L.g.nx, ny = L.g.ny, nz = L.g.nz;
  const long long nxy = L.g.nxy;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < L.g.n; c += stride) {
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / nxy);
    const long long r0 = c - x, p0 = c - (long long)y * nx - x;
    const T ec = L.eps[c];
    const T sx = hmean2(ec, L.eps[r0 + (x == 0 ? nx - 1 : x - 1)]) + hmean2(ec, L.eps[r0 + (x == nx - 1 ? 0 : x + 1)]);
    const T sy = hmean2(ec, L.eps[p0 + (long long)(y == 0 ? ny - 1 : y - 1) * nx + x]) +
                 hmean2(ec, L.eps[p0 + (long long)(y == ny - 1 ? 0 : y + 1) * nx + x]);
    const long long xy = (long long)y * nx + x;
    T sz = T(0);
    if (z > 0) sz += hmean2(ec, L.eps[c - nxy]);
    else if (L.g.periodic_z) sz += hmean2(ec, L.eps[c + (nz - 1) * nxy]);
    else if (L.tlo[xy]) sz += T(2) * ec;
    if (z < nz - 1) sz += hmean2(ec, L.eps[c + nxy]);
    else if (L.g.periodic_z) sz += hmean2(ec, L.eps[c - (nz - 1) * nxy]);
    else if (L.thi[xy]) sz += T(2) * ec;
    invd[c] = T(1) / (L.ax * sx + L.ay * sy + L.az * sz);
  }
}

template <typename T>
void launch_mg_eps_level(const LaunchCfg& L, const MgView<T>& fine, const MgView<T>& coarse, T* ceps, T* cinvd) {
  const int g1 = (int)std::max<long long>(1, std::min<long long>((coarse.g.n + 255) / 256, 4096));
  k_mg_eps_restrict<T><<<g1, 256, 0, L.stream>>>(fine, coarse, ceps);
  MgView<T> c = coarse;
  c.eps = ceps;
  k_mg_invdiag<T><<<g1, 256, 0, L.stream>>>(c, cinvd);
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
  allow_smem(k_mg_post1<T, V, false>, MgPipeP<T, V>::bytes());
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mg_post1<T, V, false>, MTX * MTY,
                                                    MgPipeP<T, V>::bytes()) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

#define PF_MG_INSTANTIATE(T)                                                           \
  template int launch_mg_pre<T>(const LaunchCfg&, const MgView<T>&, Scalars*);                   \
  template int launch_mg_rr<T>(const LaunchCfg&, const MgView<T>&, const MgView<T>&, Scalars*);  \
  template int launch_mg_prr<T>(const LaunchCfg&, const MgView<T>&, const MgView<T>&, Scalars*,   \
                                 const std::function<void(int)>&);                               \
  template bool mg_fused_post<T>(const MgView<T>&);                                              \
  template int launch_mg_pp<T>(const LaunchCfg&, const MgView<T>&, const MgView<T>&, T*, T*, double*, Scalars*, \
                                const std::function<void(int)>&);                                             \
  template void launch_mg_coarse<T>(const LaunchCfg&, const MgView<T>&, int, Scalars*);          \
  template void launch_mg_tail<T>(const LaunchCfg&, const MgTail<T>&, int, Scalars*);            \
  template int launch_mg_post1<T>(const LaunchCfg&, const MgView<T>&, const MgView<T>&, Scalars*); \
  template int launch_mg_post2<T>(const LaunchCfg&, const MgView<T>&, int, double*, Scalars*);         \
  template void launch_mg_eps_level<T>(const LaunchCfg&, const MgView<T>&, const MgView<T>&, T*, T*);  \
  template int mg_blocks_per_sm<T>();

PF_MG_INSTANTIATE(float)
PF_MG_INSTANTIATE(double)

}  // namespace pf
