// Pipelined 2.5-D plane march for 7-point stencils (vectorised cp.async staging).
//
// A thread block of TXT x TYT threads owns a BX x BY tile of (x, y) columns,
// BX = TXT * VX: each thread owns VX consecutive cells of a row (one 16-byte
// vector: 4 floats or 2 doubles; VX = 1 when nx is not a multiple of that).
// Tiles are handed out dynamically (an atomic counter), so blocks that finish
// early take more work.  Along its z range the block streams the raw inputs
// of the stencil (NH arrays) with a one-cell halo ring, and the own-cell-only
// inputs (NO arrays), copied global -> shared with cp.async D planes ahead
// into a ring of D + 2 stages (16-byte copies for the vectors, 4/8-byte
// copies for the x halo).  Two walks use them:
//   - march: the stencil field (the caller's val functor applied to the raw
//     values, e.g. p = r/diag + beta p_old) is formed once per cell into a
//     shared buffer of plane z (ring of three planes), read by the in-plane
//     neighbours after the plane's barrier;
//   - march_direct: the stencil is the raw input itself, read straight from
//     the stage of plane z.
// In both, each thread keeps its own column's values of planes z-1, z, z+1
// in registers, so only in-plane neighbours cross threads, all within the
// current plane: one __syncthreads per plane orders every shared access.
// x neighbours inside a vector come from registers, across vectors of one
// warp row from shuffles, across the tile edge from the halo.  Periodic x/y
// wrap is resolved in the halo source addresses; ragged tiles put their
// right/bottom halo right after the last valid column/row.  Planes below
// z = 0 / above nz - 1 exist only for periodic z.
#pragma once

#include "pf_common.cuh"

namespace pf {

template <int TXT, int TYT, int VX>
struct TileGeo {
  int z0, z1;            // z range [z0, z1)
  int w, h;              // valid width (cells) / height of the tile
  int tx, ty;
  int x, y;              // first own cell
  bool act;              // own vector inside the grid
  int xy;                // y*nx + x of the first own cell
  int xl, xr, yt, yb;    // wrapped coordinates of the halo column/rows
  int xy_l, xy_r;        // x-halo cells this thread fills (-1: none)
  int xy_t, xy_b;        // first cell of the y-halo vector this thread fills (-1: none)
};

template <int TXT, int TYT, int VX>
__device__ __forceinline__ TileGeo<TXT, TYT, VX> tile_geo(const Geo& g, long long t, const MarchCfg& mc) {
  constexpr int BX = TXT * VX;
  TileGeo<TXT, TYT, VX> s;
  const int tt = (int)t;                 // tile counts stay far below 2^31
  const int ix = tt % mc.tiles_x;
  const int r = tt / mc.tiles_x;
  const int iy = r % mc.tiles_y;
  const int iz = r / mc.tiles_y;
  const int x0 = ix * BX, y0 = iy * TYT;
  s.z0 = mc.zlo + iz * (mc.tz + mc.zskip);
  s.z1 = min(s.z0 + mc.tz, g.nz - mc.zcut);
  s.w = min(BX, g.nx - x0);
  s.h = min(TYT, g.ny - y0);
  s.tx = threadIdx.x;
  s.ty = threadIdx.y;
  s.x = x0 + s.tx * VX;
  s.y = y0 + s.ty;
  s.act = s.tx * VX < s.w && s.ty < s.h;
  s.xy = s.y * g.nx + s.x;
  s.xl = x0 == 0 ? g.nx - 1 : x0 - 1;
  s.xr = x0 + s.w == g.nx ? 0 : x0 + s.w;
  s.yt = y0 == 0 ? g.ny - 1 : y0 - 1;
  s.yb = y0 + s.h == g.ny ? 0 : y0 + s.h;
  s.xy_l = s.xy_r = s.xy_t = s.xy_b = -1;
  if (s.act) {
    if (s.tx == 0) s.xy_l = s.y * g.nx + s.xl;
    if (s.tx == s.w / VX - 1) s.xy_r = s.y * g.nx + s.xr;
    if (s.ty == 0) s.xy_t = s.yt * g.nx + s.x;
    if (s.ty == s.h - 1) s.xy_b = s.yb * g.nx + s.x;
  }
  return s;
}

// z plane below/above z, or -1 at a non-periodic boundary.
__device__ __forceinline__ int z_below(const Geo& g, int z) {
  return z > 0 ? z - 1 : (g.periodic_z ? g.nz - 1 : -1);
}
__device__ __forceinline__ int z_above(const Geo& g, int z) {
  return z < g.nz - 1 ? z + 1 : (g.periodic_z ? 0 : -1);
}

// Neighbour values of one cell handed to the emit functor.
template <typename F>
struct Stencil7 {
  F c, xm, xp, ym, yp, zm, zp;
  int zb, za;        // plane below / above (-1: boundary face)
};

// ------------------------------------------------------------- cp.async

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// VX consecutive values through one 16-byte access when they fill it.
template <typename V, int VX>
__device__ __forceinline__ void load_n(const V* p, V (&o)[VX]) {
  if constexpr (VX == 2 && sizeof(V) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    reinterpret_cast<float*>(o)[0] = t.x;
    reinterpret_cast<float*>(o)[1] = t.y;
  } else if constexpr (VX == 4 && sizeof(V) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    const float* f = reinterpret_cast<const float*>(&t);
#pragma unroll
    for (int i = 0; i < 4; ++i) reinterpret_cast<float*>(o)[i] = f[i];
  } else if constexpr (VX == 2 && sizeof(V) == 8) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    reinterpret_cast<double*>(o)[0] = t.x;
    reinterpret_cast<double*>(o)[1] = t.y;
  } else {
#pragma unroll
    for (int i = 0; i < VX; ++i) o[i] = p[i];
  }
}
template <typename V, int VX>
__device__ __forceinline__ void store_n(V* p, const V (&v)[VX]) {
  if constexpr (VX == 4 && sizeof(V) == 4) {
    const float* f = reinterpret_cast<const float*>(v);
    *reinterpret_cast<float4*>(p) = make_float4(f[0], f[1], f[2], f[3]);
  } else if constexpr (VX == 2 && sizeof(V) == 8) {
    const double* d = reinterpret_cast<const double*>(v);
    *reinterpret_cast<double2*>(p) = make_double2(d[0], d[1]);
  } else {
#pragma unroll
    for (int i = 0; i < VX; ++i) p[i] = v[i];
  }
}

// Stencil field with the cell permittivity carried along (eps bound); the
// face permittivity is the harmonic mean of the two cells.
template <typename T>
struct EpsVal {
  T v, e;
};

// Warp shuffles of a field value (scalar or EpsVal).
template <typename T>
__device__ __forceinline__ T shfl_up1(T v) {
  return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ EpsVal<T> shfl_up1(EpsVal<T> v) {
  return EpsVal<T>{__shfl_up_sync(0xffffffffu, v.v, 1), __shfl_up_sync(0xffffffffu, v.e, 1)};
}
template <typename T>
__device__ __forceinline__ T shfl_down1(T v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ EpsVal<T> shfl_down1(EpsVal<T> v) {
  return EpsVal<T>{__shfl_down_sync(0xffffffffu, v.v, 1), __shfl_down_sync(0xffffffffu, v.e, 1)};
}

// ------------------------------------------------------------ the march

template <typename T, typename F, int TXT, int TYT, int VX, int NH, int NO, int D, int NP = 0>
struct Pipe {
  static constexpr int BX = TXT * VX, BY = TYT;
  static constexpr int OFF = VX;                     // interior starts 16-byte aligned
  static constexpr int RS = BX + 2 * OFF, HH = BY + 2;
  static constexpr int NS = D + 2;
  // NP = 1: one more halo-shaped plane holding each cell's coarse-grid parent
  static constexpr int STAGE = (NH + NP) * HH * RS + NO * BY * BX;   // elements of T per stage
  // F = void: the stencil is read straight from the staged raw planes
  static constexpr size_t field_bytes() {
    if constexpr (std::is_same<F, void>::value) return 0;
    else return 3 * (size_t)HH * RS * sizeof(F);
  }
  static constexpr size_t bytes() { return (size_t)NS * STAGE * sizeof(T) + field_bytes(); }
};

// Tile scheduler.  A grid with a block per tile (the small multigrid levels)
// takes tile blockIdx.x and touches no counter.  Otherwise tiles are handed
// out dynamically: thread 0 takes the next tile from an atomic counter, and
// the last block to run out resets the counter for the next launch.
struct TileSched {
  unsigned long long* next;
  unsigned* done;
  bool fixed;                      // a block per tile: tile blockIdx.x, no counter
  __device__ __forceinline__ TileSched(unsigned long long* n, unsigned* d, long long ntiles)
      : next(n), done(d), fixed((long long)gridDim.x >= ntiles) {}
};

__device__ __forceinline__ long long sched_take(const TileSched& ts, long long* slot) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) *slot = (long long)atomicAdd(ts.next, 1ull);
  __syncthreads();
  return *slot;
}

__device__ __forceinline__ long long sched_first(const TileSched& ts, long long* slot) {
  return ts.fixed ? (long long)blockIdx.x : sched_take(ts, slot);
}

// the next tile; past every tile (so the caller's loop ends) in the fixed form
__device__ __forceinline__ long long sched_next(const TileSched& ts, long long* slot) {
  return ts.fixed ? (1LL << 62) : sched_take(ts, slot);
}

__device__ __forceinline__ void sched_finish(const TileSched& ts) {
  if (ts.fixed) return;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    if (atomicAdd(ts.done, 1u) == gridDim.x - 1) {
      *ts.next = 0ull;
      *ts.done = 0u;
      __threadfence();
    }
  }
}

// Coarse-grid parent of every fine cell (multigrid prolongation): the value
// of field ec at (z/fz, y/fy, x/fx) of a grid with row nxc and plane nxyc.
// The factors are 1 or 2, so the divisions are shifts by f - 1.
template <typename T>
struct ParentSrc {
  const T* ec;
  int fx, fy, fz, nxc;
  long long nxyc;
  __device__ __forceinline__ long long at(int x, int y, int z) const {
    return (long long)(z >> (fz - 1)) * nxyc + (long long)(y >> (fy - 1)) * nxc + (x >> (fx - 1));
  }
};

// The staging ring of one tile: virtual plane v = 0 .. nt+1 is z0-1 .. z1
// (v = 0 and nt+1 feed only the own column's z neighbours).  With NP = 1 the
// parents of the staged cells are staged too: a vector of VX fine cells has
// VX/fx parents, stored from its first slot on.
template <typename T, int TXT, int TYT, int VX, int NH, int NO, int D, int NP = 0>
struct Stager {
  using P = Pipe<T, void, TXT, TYT, VX, NH, NO, D, NP>;
  static constexpr int OFF = P::OFF, RS = P::RS, HH = P::HH, BX = P::BX, NS = P::NS, STAGE = P::STAGE;
  const Geo& g;
  const TileGeo<TXT, TYT, VX>& s;
  T* stages;
  const T* const* hsrc;
  const T* const* osrc;
  ParentSrc<T> par;
  int nt, zlo, zhi, row, col;

  __device__ __forceinline__ Stager(const Geo& g_, const TileGeo<TXT, TYT, VX>& s_, T* st, const T* const* h,
                                    const T* const* o, ParentSrc<T> pr = ParentSrc<T>{})
      : g(g_), s(s_), stages(st), hsrc(h), osrc(o), par(pr) {
    nt = s.z1 - s.z0;
    zlo = z_below(g, s.z0);
    zhi = z_above(g, s.z1 - 1);
    row = s.ty + 1;
    col = OFF + s.tx * VX;
  }
  // parent plane of stage st (same shape as a halo plane)
  __device__ __forceinline__ T* PA(int st, int rw, int cl) const {
    return stages + (size_t)st * STAGE + (NH * HH + rw) * RS + cl;
  }
  // parent slot of vector element i (own vector or a y-halo vector)
  __device__ __forceinline__ int pslot(int i) const { return col + (i >> (par.fx - 1)); }
  // copy the parents of a vector starting at fine (x, y) of plane z into slot (rw, col)
  __device__ __forceinline__ void issue_parent_vec(int st, int rw, int x, int y, int z) const {
    const T* src = par.ec + par.at(x, y, z);
    if (par.fx == 2) {
      if constexpr (VX >= 2) cp_async<(VX / 2) * sizeof(T)>(PA(st, rw, col), src);
      else cp_async<sizeof(T)>(PA(st, rw, col), src);
    } else {
      cp_async<VX * sizeof(T)>(PA(st, rw, col), src);
    }
  }
  __device__ __forceinline__ void issue_parent_one(int st, int rw, int cl, int x, int y, int z) const {
    cp_async<sizeof(T)>(PA(st, rw, cl), par.ec + par.at(x, y, z));
  }
  __device__ __forceinline__ int plane(int v) const { return v == 0 ? zlo : (v == nt + 1 ? zhi : s.z0 + v - 1); }
  __device__ __forceinline__ T* H(int st, int k, int rw, int cl) const {
    return stages + (size_t)st * STAGE + (k * HH + rw) * RS + cl;
  }
  // own-cell plane k of stage st (after the NH halo planes and the parent plane)
  __device__ __forceinline__ T* O(int st, int k) const {
    return stages + (size_t)st * STAGE + (NH + NP) * HH * RS + (k * TYT + s.ty) * BX + s.tx * VX;
  }
  // Copy plane v (own cells; halo cells too for in-tile planes) into its stage.
  __device__ __forceinline__ void issue(int v) const {
    if (v <= nt + 1 && s.act) {
      const int z = plane(v);
      if (z >= 0) {
        const long long zo = (long long)z * g.nxy;
        const int st = v % NS;
        const bool halo = v >= 1 && v <= nt;
#pragma unroll
        for (int k = 0; k < NH; ++k) {
          const T* src = hsrc[k] + zo;
          cp_async<VX * sizeof(T)>(H(st, k, row, col), src + s.xy);
          if (halo) {
            if (s.xy_l >= 0) cp_async<sizeof(T)>(H(st, k, row, OFF - 1), src + s.xy_l);
            if (s.xy_r >= 0) cp_async<sizeof(T)>(H(st, k, row, OFF + s.w), src + s.xy_r);
            if (s.xy_t >= 0) cp_async<VX * sizeof(T)>(H(st, k, 0, col), src + s.xy_t);
            if (s.xy_b >= 0) cp_async<VX * sizeof(T)>(H(st, k, s.h + 1, col), src + s.xy_b);
          }
        }
#pragma unroll
        for (int k = 0; k < NO; ++k) cp_async<VX * sizeof(T)>(O(st, k), osrc[k] + zo + s.xy);
        if constexpr (NP > 0) {
          issue_parent_vec(st, row, s.x, s.y, z);
          if (halo) {
            if (s.xy_l >= 0) issue_parent_one(st, row, OFF - 1, s.xl, s.y, z);
            if (s.xy_r >= 0) issue_parent_one(st, row, OFF + s.w, s.xr, s.y, z);
            if (s.xy_t >= 0) issue_parent_vec(st, 0, s.x, s.yt, z);
            if (s.xy_b >= 0) issue_parent_vec(st, s.h + 1, s.x, s.yb, z);
          }
        }
      }
    }
    cp_commit();          // one group per virtual plane, empty or not
  }
};

// Raw values of NH fields at one cell (the stencil type of march_direct).
template <typename T, int NH>
struct Raw {
  T v[NH];
};

// Walk one tile, stencil field formed by val.
//   hsrc[k]  NH raw arrays needed with halo;  osrc[k]  NO raw arrays needed at
//            the own cells only (linear cell index).
//   val(const T (&h)[NH], xy, z, col, i, [parent,] bt) -> F   stencil field at one
//            cell from its raw values; col: 0 own vector, 1..4 left/right/top/
//            bottom halo; i: index inside the vector (0 for the x halo); parent:
//            the staged coarse parent (NP = 1 only).
//   emit(xy, z, const Stencil7<F>&, const T (&h)[NH], const T (&o)[NO], bt) -> Out
//            consumes one own cell and returns its outputs.
//   bt is true on the planes next to a non-periodic z face and false
//   elsewhere (always a constant after inlining): the functors keep their
//   boundary handling behind it (there zb/za of the stencil say which face
//   is open); on other planes zb = za = 0.
//   post(z, const Out (&out)[VX])  receives the outputs of the own vector
//            (and stores them: 16-byte stores of whole vectors).
// smem: Pipe<...>::bytes() bytes, 16-byte aligned.  Every thread of the block
// must call this (it synchronises).
template <typename T, typename F, typename Out, int TXT, int TYT, int VX, int NH, int NO, int D, int NP = 0,
          bool INTR = false, class Val, class Emit, class Post>
__device__ __forceinline__ void march(const Geo& g, const TileGeo<TXT, TYT, VX>& s, unsigned char* smem,
                                      const T* const (&hsrc)[NH], const T* const (&osrc)[NO > 0 ? NO : 1],
                                      Val val, Emit emit, Post post, ParentSrc<T> par = ParentSrc<T>{}) {
  using P = Pipe<T, F, TXT, TYT, VX, NH, NO, D, NP>;
  using SG = Stager<T, TXT, TYT, VX, NH, NO, D, NP>;
  constexpr int OFF = P::OFF, RS = P::RS, HH = P::HH, NS = P::NS;
  static_assert(TXT == 16 || TXT == 32, "a warp holds one or two tile rows");
  const SG sg(g, s, reinterpret_cast<T*>(smem), hsrc, osrc, par);
  // the stencil field at one cell; with staged parents val also gets the parent.
  // bt is true on the planes next to a non-periodic z face, where boundary
  // data matter; the march calls its (inlined) loops with the constants true
  // and false, so each copy compiles only the code it needs.
  auto val_at = [&](const T (&h1)[NH], int xy, int z, int colid, int i, int st, int rw, int pcl, const bool bt) -> F {
    if constexpr (NP > 0) return val(h1, xy, z, colid, i, *sg.PA(st, rw, pcl), bt);
    else return val(h1, xy, z, colid, i, bt);
  };
  F* pn = reinterpret_cast<F*>(smem + (size_t)NS * P::STAGE * sizeof(T));
  auto PN = [&](int b, int rw, int cl) -> F* { return pn + (b * HH + rw) * RS + cl; };
  const int nt = sg.nt, row = sg.row, col = sg.col;
  const bool left_in_warp = s.tx > 0;
  const bool right_in_warp = s.tx < TXT - 1 && (s.tx + 1) * VX < s.w;

  auto form_vec = [&](int st, int rw, int cl, int xy, int z, int colid, F (&fv)[VX], const bool bt) {
    T hv[NH][VX];
#pragma unroll
    for (int k = 0; k < NH; ++k) load_n<T, VX>(sg.H(st, k, rw, cl), hv[k]);
#pragma unroll
    for (int i = 0; i < VX; ++i) {
      T h1[NH];
#pragma unroll
      for (int k = 0; k < NH; ++k) h1[k] = hv[k][i];
      fv[i] = val_at(h1, xy + i, z, colid, i, st, rw, NP > 0 ? sg.pslot(i) : 0, bt);
    }
  };
  // Stencil field of plane v (into field buffer b = v mod 3): own vector,
  // plus the halo cells for in-tile planes.
  auto form_t = [&](int v, int b, int z, F (&fv)[VX], const bool bt) {
    const int st = v % NS;
    form_vec(st, row, col, s.xy, z, 0, fv, bt);
    store_n<F, VX>(PN(b, row, col), fv);
    if (v < 1 || v > nt) return;
    T h1[NH];
    if (s.xy_l >= 0) {
#pragma unroll
      for (int k = 0; k < NH; ++k) h1[k] = *sg.H(st, k, row, OFF - 1);
      *PN(b, row, OFF - 1) = val_at(h1, s.xy_l, z, 1, 0, st, row, OFF - 1, bt);
    }
    if (s.xy_r >= 0) {
#pragma unroll
      for (int k = 0; k < NH; ++k) h1[k] = *sg.H(st, k, row, OFF + s.w);
      *PN(b, row, OFF + s.w) = val_at(h1, s.xy_r, z, 2, 0, st, row, OFF + s.w, bt);
    }
    if (s.xy_t >= 0) {
      F hv[VX];
      form_vec(st, 0, col, s.xy_t, z, 3, hv, bt);
      store_n<F, VX>(PN(b, 0, col), hv);
    }
    if (s.xy_b >= 0) {
      F hv[VX];
      form_vec(st, s.h + 1, col, s.xy_b, z, 4, hv, bt);
      store_n<F, VX>(PN(b, s.h + 1, col), hv);
    }
  };
  // Form plane v into field buffer b; own receives the thread's own vector.
  auto form = [&](int v, int b, F (&own)[VX]) {
    const int z = sg.plane(v);
    if (!s.act || z < 0) return;
    if (z_below(g, z) < 0 || z_above(g, z) < 0) form_t(v, b, z, own, true);
    else form_t(v, b, z, own, false);
  };

  // The own column's field values of planes v - 1, v, v + 1 stay in
  // registers; only the in-plane neighbours are read from the shared buffer
  // of plane v.  The buffer written at iteration v (plane v + 1) is then
  // never one that a thread still in iteration v - 1 reads (plane v - 1), so
  // one barrier per plane orders every shared access.
  F zmr[VX], cvr[VX], zpr[VX];
#pragma unroll
  for (int i = 0; i < VX; ++i) zmr[i] = cvr[i] = zpr[i] = F{};
  for (int v = 0; v <= D; ++v) sg.issue(v);
  cp_wait<D - 1>();                 // planes 0 and 1 have landed
  form(0, 0, zmr);
  form(1, 1, cvr);
  int bp = 0, b = 1, bn = 2;        // field buffers of planes v - 1, v, v + 1 (v mod 3)
  for (int v = 1; v <= nt; ++v) {
    sg.issue(v + D);
    cp_wait<D - 1>();               // plane v + 1 has landed
    form(v + 1, bn, zpr);
    __syncthreads();
    const int zb = sg.plane(v - 1), za = sg.plane(v + 1);
    F cv[VX], ym[VX], yp[VX];
    if (s.act) {
#pragma unroll
      for (int i = 0; i < VX; ++i) cv[i] = cvr[i];
      load_n<F, VX>(PN(b, row - 1, col), ym);
      load_n<F, VX>(PN(b, row + 1, col), yp);
    } else {
#pragma unroll
      for (int i = 0; i < VX; ++i) cv[i] = F{};
    }
    // x neighbours at the vector ends: the neighbouring lane's vector, or
    // shared memory (halo) at the tile-row ends
    F lft = shfl_up1(cv[VX - 1]);
    F rgt = shfl_down1(cv[0]);
    if (s.act) {
      if (!left_in_warp) lft = *PN(b, row, col - 1);
      if (!right_in_warp) rgt = *PN(b, row, col + VX);
      const int z = s.z0 + v - 1;
      const int st = v % NS;
      T hv[NH][VX], ov[NO > 0 ? NO : 1][VX];
#pragma unroll
      for (int k = 0; k < NH; ++k) load_n<T, VX>(sg.H(st, k, row, col), hv[k]);
#pragma unroll
      for (int k = 0; k < NO; ++k) load_n<T, VX>(sg.O(st, k), ov[k]);
      auto emit_all = [&](const bool B) {
        Out outv[VX];
#pragma unroll
        for (int i = 0; i < VX; ++i) {
          Stencil7<F> sc;
          sc.c = cv[i];
          sc.xm = i == 0 ? lft : cv[i - 1];
          sc.xp = i == VX - 1 ? rgt : cv[i + 1];
          sc.ym = ym[i];
          sc.yp = yp[i];
          sc.zm = (!B || zb >= 0) ? zmr[i] : F{};
          sc.zp = (!B || za >= 0) ? zpr[i] : F{};
          sc.zb = B ? zb : 0;
          sc.za = B ? za : 0;
          T h1[NH], o1[NO > 0 ? NO : 1];
#pragma unroll
          for (int k = 0; k < NH; ++k) h1[k] = hv[k][i];
#pragma unroll
          for (int k = 0; k < NO; ++k) o1[k] = ov[k][i];
          outv[i] = emit(s.xy + i, z, sc, h1, o1, B);
        }
        post(z, outv);
      };
      if (!INTR && (zb < 0 || za < 0)) emit_all(true);
      else emit_all(false);
    }
#pragma unroll
    for (int i = 0; i < VX; ++i) {
      zmr[i] = cvr[i];
      cvr[i] = zpr[i];
    }
    const int t3 = bp;
    bp = b;
    b = bn;
    bn = t3;
  }
  cp_wait<0>();
}

// Walk one tile whose stencil is the raw input itself: the neighbours are read
// straight from the staged planes (after the plane's barrier), with no field
// buffer.  emit(xy, z, const Stencil7<Raw<T,NH+NP>>&, const T (&o)[NO], bt) -> Out;
// post and bt as in march.  With NP = 1 the staged coarse-grid parents come as
// field NH of the stencil (the parent of each of the seven cells); a vector's
// parents are stored compactly (VX / fx values), read with one access and
// expanded in registers.  INTR (both walks): the launch covers interior planes
// only (every plane has both z neighbours), so only the bt = false form of the
// functors is compiled -- the boundary code then costs no registers.
template <typename T, typename Out, int TXT, int TYT, int VX, int NH, int NO, int D, int NP = 0, bool INTR = false,
          class Emit, class Post>
__device__ __forceinline__ void march_direct(const Geo& g, const TileGeo<TXT, TYT, VX>& s, unsigned char* smem,
                                             const T* const (&hsrc)[NH], const T* const (&osrc)[NO > 0 ? NO : 1],
                                             Emit emit, Post post, ParentSrc<T> par = ParentSrc<T>{}) {
  using SG = Stager<T, TXT, TYT, VX, NH, NO, D, NP>;
  using R = Raw<T, NH + NP>;
  constexpr int NS = SG::NS, OFF = SG::OFF;
  static_assert(TXT == 16 || TXT == 32, "a warp holds one or two tile rows");
  const SG sg(g, s, reinterpret_cast<T*>(smem), hsrc, osrc, par);
  const int nt = sg.nt, row = sg.row, col = sg.col;
  const bool left_in_warp = s.tx > 0;
  const bool right_in_warp = s.tx < TXT - 1 && (s.tx + 1) * VX < s.w;

  // The own column's raw values of planes v - 1, v, v + 1 stay in registers
  // (each thread reads back only its own cells of planes v - 1 and v + 1);
  // other threads' cells are read from the stage of plane v alone, so the
  // stage a thread refills at iteration v (plane v + D, D >= 2) is never one
  // that a thread still in iteration v - 1 reads, and one barrier per plane
  // orders every shared access.
  static_assert(D >= 2 && NS >= D + 2, "stage ring too short for one barrier per plane");
  constexpr int NF = NH + NP;
  T zmr[NF][VX], cr[NF][VX], zpr[NF][VX];
#pragma unroll
  for (int k = 0; k < NF; ++k)
#pragma unroll
    for (int i = 0; i < VX; ++i) zmr[k][i] = cr[k][i] = zpr[k][i] = T(0);
  // field k of the vector row rw in stage st (parents: compact, expanded)
  auto load_vec = [&](int st, int k, int rw, T (&o)[VX]) {
    if (k < NH) {
      load_n<T, VX>(sg.H(st, k, rw, col), o);
    } else if constexpr (VX >= 2) {
      if (par.fx == 2) {
        T h[VX / 2];
        load_n<T, VX / 2>(sg.PA(st, rw, col), h);
#pragma unroll
        for (int i = 0; i < VX; ++i) o[i] = h[i >> 1];
      } else {
        load_n<T, VX>(sg.PA(st, rw, col), o);
      }
    } else {
      o[0] = *sg.PA(st, rw, col);
    }
  };
  for (int v = 0; v <= D; ++v) sg.issue(v);
  for (int v = 1; v <= nt; ++v) {
    sg.issue(v + D);
    cp_wait<D - 1>();               // planes <= v + 1 of this thread have landed
    __syncthreads();                // ... and of every thread
    const int st = v % NS, sa = (v + 1) % NS;
    const int zb = sg.plane(v - 1), za = sg.plane(v + 1);
    if (v == 1 && s.act) {
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        if (zb >= 0) load_vec(0, k, row, zmr[k]);
        load_vec(st, k, row, cr[k]);
      }
    }
    T ym[NF][VX], yp[NF][VX], lft[NF], rgt[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      if (s.act) {
        load_vec(st, k, row - 1, ym[k]);
        load_vec(st, k, row + 1, yp[k]);
        if (za >= 0) load_vec(sa, k, row, zpr[k]);
      }
      lft[k] = shfl_up1(s.act ? cr[k][VX - 1] : T(0));
      rgt[k] = shfl_down1(s.act ? cr[k][0] : T(0));
      if (s.act) {
        if (k < NH) {
          if (!left_in_warp) lft[k] = *sg.H(st, k, row, col - 1);
          if (!right_in_warp) rgt[k] = *sg.H(st, k, row, col + VX);
        } else {
          if (!left_in_warp) lft[k] = *sg.PA(st, row, OFF - 1);
          if (!right_in_warp) rgt[k] = *sg.PA(st, row, OFF + s.w);
        }
      }
    }
    if (s.act) {
      const int z = s.z0 + v - 1;
      T ov[NO > 0 ? NO : 1][VX];
#pragma unroll
      for (int k = 0; k < NO; ++k) load_n<T, VX>(sg.O(st, k), ov[k]);
      auto emit_all = [&](const bool B) {
        Out outv[VX];
#pragma unroll
        for (int i = 0; i < VX; ++i) {
          Stencil7<R> sc;
#pragma unroll
          for (int k = 0; k < NF; ++k) {
            sc.c.v[k] = cr[k][i];
            sc.xm.v[k] = i == 0 ? lft[k] : cr[k][i - 1];
            sc.xp.v[k] = i == VX - 1 ? rgt[k] : cr[k][i + 1];
            sc.ym.v[k] = ym[k][i];
            sc.yp.v[k] = yp[k][i];
            sc.zm.v[k] = (!B || zb >= 0) ? zmr[k][i] : T(0);
            sc.zp.v[k] = (!B || za >= 0) ? zpr[k][i] : T(0);
          }
          sc.zb = B ? zb : 0;
          sc.za = B ? za : 0;
          T o1[NO > 0 ? NO : 1];
#pragma unroll
          for (int k = 0; k < NO; ++k) o1[k] = ov[k][i];
          outv[i] = emit(s.xy + i, z, sc, o1, B);
        }
        post(z, outv);
      };
      if (!INTR && (zb < 0 || za < 0)) emit_all(true);
      else emit_all(false);
    }
#pragma unroll
    for (int k = 0; k < NF; ++k)
#pragma unroll
      for (int i = 0; i < VX; ++i) {
        zmr[k][i] = cr[k][i];
        cr[k][i] = zpr[k][i];
      }
  }
  cp_wait<0>();
}

// The k-th field of a Raw stencil as a scalar stencil.
template <typename T, int NH>
__device__ __forceinline__ Stencil7<T> pick(const Stencil7<Raw<T, NH>>& s, int k) {
  Stencil7<T> o;
  o.c = s.c.v[k];
  o.xm = s.xm.v[k];
  o.xp = s.xp.v[k];
  o.ym = s.ym.v[k];
  o.yp = s.yp.v[k];
  o.zm = s.zm.v[k];
  o.zp = s.zp.v[k];
  o.zb = s.zb;
  o.za = s.za;
  return o;
}

// --------------------------------------------------------- stencil fields

// (A v)_c for eps = 1 with homogeneous boundary data: faces summed in the
// order x-, x+, y-, y+, z-, z+; a boundary face adds 2 v_c at an electrode
// and nothing at an open surface.
template <typename T>
__device__ __forceinline__ T apply_field(const Stencil7<T>& s, int dlo, int dhi, T ih2) {
  T acc = T(0);
  acc += s.c - s.xm;
  acc += s.c - s.xp;
  acc += s.c - s.ym;
  acc += s.c - s.yp;
  if (s.zb >= 0) acc += s.c - s.zm;
  else if (dlo) acc += T(2) * s.c;
  if (s.za >= 0) acc += s.c - s.zp;
  else if (dhi) acc += T(2) * s.c;
  return acc * ih2;
}


template <typename T, bool EPS>
struct FieldOf {
  using type = T;
};
template <typename T>
struct FieldOf<T, true> {
  using type = EpsVal<T>;
};

template <typename T>
__device__ __forceinline__ T field_value(T f) { return f; }
template <typename T>
__device__ __forceinline__ T field_value(const EpsVal<T>& f) { return f.v; }

template <typename T>
__device__ __forceinline__ T hmean2(T a, T b) {
  return T(2) * a * b / (a + b);
}

template <typename T>
__device__ __forceinline__ T apply_field(const Stencil7<EpsVal<T>>& s, int dlo, int dhi, T ih2) {
  const T ec = s.c.e, vc = s.c.v;
  T acc = T(0);
  acc += hmean2(ec, s.xm.e) * (vc - s.xm.v);
  acc += hmean2(ec, s.xp.e) * (vc - s.xp.v);
  acc += hmean2(ec, s.ym.e) * (vc - s.ym.v);
  acc += hmean2(ec, s.yp.e) * (vc - s.yp.v);
  if (s.zb >= 0) acc += hmean2(ec, s.zm.e) * (vc - s.zm.v);
  else if (dlo) acc += T(2) * ec * vc;
  if (s.za >= 0) acc += hmean2(ec, s.zp.e) * (vc - s.zp.v);
  else if (dhi) acc += T(2) * ec * vc;
  return acc * ih2;
}

// Boundary-aware on the planes next to a z face (bt), plain 7-point stencil
// elsewhere.  Same face order, so both give identical sums.
template <typename T>
__device__ __forceinline__ T apply_bt(const Stencil7<T>& s, int dlo, int dhi, T ih2, const bool bt) {
  if (bt) return apply_field(s, dlo, dhi, ih2);
  Stencil7<T> t = s;
  t.zb = 0;
  t.za = 0;
  return apply_field(t, 0, 0, ih2);
}
template <typename T>
__device__ __forceinline__ T apply_bt(const Stencil7<EpsVal<T>>& s, int dlo, int dhi, T ih2, const bool bt) {
  if (bt) return apply_field(s, dlo, dhi, ih2);
  Stencil7<EpsVal<T>> t = s;
  t.zb = 0;
  t.za = 0;
  return apply_field(t, 0, 0, ih2);
}

// Set the dynamic shared-memory limit of a kernel.
template <typename K>
inline void allow_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace pf
