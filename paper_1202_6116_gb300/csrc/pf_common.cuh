// Internal device helpers of the GPU library: grid geometry, boundary masks,
// FP64-accurate reductions and the solver scalar block.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

// Tile of one thread block in the simple per-cell kernels: TX x TY columns of
// tz cells (x fastest).
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NTHREADS = TX * TY;
// Threads of a plane-march block (MTX x MTY, each owning one 16-byte vector
// of cells in x) and block size of the flat kernels.
constexpr int MTX = 16;
constexpr int MTY = 16;
constexpr int FLAT_THREADS = 256;

// Tiling of a plane-march launch: tiles of (MTX * vx) x MTY columns times tz
// planes; vx = cells per thread (16 bytes, or 1 when nx is not a multiple).
// Tile z-index iz covers planes [zlo + iz (tz + zskip), that + tz), clipped
// at nz - zcut; all three are 0 for a launch over the whole z range (a launch
// over the interior planes sets zlo = zcut = b; one over the two face slabs
// of b planes sets tz = b, zskip = nz - 2 b).
struct MarchCfg {
  int tiles_x, tiles_y, tz;
  long long ntiles;
  int grid;
  int vx;
  int zlo, zcut, zskip;
  int bps;           // resident blocks per SM asked for (0: as many as fit; kernels
                     // with their own occupancy size their grid by it)
};

struct Geo {
  int nx, ny, nz;
  int periodic_z;
  int zair;                // first air plane (nz: no air layers); P = 0 from there up
  long long nxy, n;
  double ih, ih2;          // 1/dx, 1/dx^2
  int tz;                  // cells per column in one tile
  int tiles_x, tiles_y, tiles_z;
  long long ntiles;
};

// Electrical z-face masks (per (x,y) cell of the face).
template <typename T>
struct Bc {
  const int8_t* tlo;
  const int8_t* thi;
  const T* vlo;
  const T* vhi;
};

// 16-byte vector type of a field element type.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

// 1/diag(A) at column xy of plane z when eps = 1.  The diagonal is
// (interior faces + 2 x electrode faces)/dx^2: 6/dx^2 away from the z faces.
// Every kernel forms it through this one expression, so z = r/diag agrees
// bit for bit between kernels.
template <typename T>
__device__ __forceinline__ T inv_diag_unit(const Geo& g, const Bc<T>& bc, long long xy, int z, T inv6) {
  if (g.periodic_z || (z > 0 && z < g.nz - 1)) return inv6;
  const int k = 4 + (z > 0 ? 1 : 2 * (int)bc.tlo[xy]) + (z < g.nz - 1 ? 1 : 2 * (int)bc.thi[xy]);
  return T(1) / (T(k) * T(g.ih2));
}

// Same, addressed by the linear cell index e.
template <typename T>
__device__ __forceinline__ T inv_flat(const Geo& g, const Bc<T>& bc, long long e, T inv6) {
  if (g.periodic_z || (e >= g.nxy && e < g.n - g.nxy)) return inv6;
  const int z = e < g.nxy ? 0 : g.nz - 1;
  return inv_diag_unit(g, bc, e - (long long)z * g.nxy, z, inv6);
}

// Solver state in device memory (inside the caller's workspace).
struct Scalars {
  double bb;        // ||b||^2
  double rz;        // r.z of the current residual
  double rr;        // ||r||^2
  double alpha;
  double beta;
  double pq;
  double mean_b;    // zero-mean projection of b (singular problems)
  double mean_x;    // mean of the solution (singular problems)
  double rtol;
  double last_rel;  // ||r||/||b|| at the end of the last solve
  long long total_iters;
  int maxit;
  int iter;
  int done;         // 1: the current solve has finished
  int first;        // 1: next p-update is p = z
  int pending;      // 1: x += alpha p still owed
  int zero_x;       // 1: b == 0, the solution is 0
  int status;       // 0 ok, 3 not converged (current solve)
  int pbuf;         // which of the two p buffers holds the latest p
  int nonconv;      // solves that did not converge (per pf_step call)
  int last_iters;
  unsigned ticket;  // last-block counter of the reduction kernels
  int nonfinite;
  unsigned long long sched_next;   // dynamic tile scheduler: next tile
  unsigned sched_done;             // blocks that ran out of tiles
  int zero_solves;                 // solves that ended with no iteration (per pf_step call)
  int max_iters;                   // most iterations of one solve (per pf_step call)
  int solves;                      // solves finished (per pf_step call)
  int short_solves;                // solves that ended after at most one iteration (per pf_step call)
  int xzero;                       // 1: the Krylov iterate is the correction of a compensated
                                   // start and is still 0 (its buffer holds stale values)
};

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Dot-product accumulators.  FP64 fields: plain FMA accumulation.  FP32
// fields: a short run of products (the cells of one vector, closed by run())
// is summed by plain FMAs; the run totals are summed with TwoSum (Knuth), the
// error terms collected in a second float ("cascaded" summation: the
// compensated sum of Ogita, Rump & Oishi, SIAM J. Sci. Comput. 26, 2005,
// applied to runs instead of single products); flush() moves the pair into an
// FP64 total, so the FP64 unit sees a handful of adds per tile.  A run of k
// products carries a relative error of about k u (u = 2^-24) of its absolute
// sum, so with k = 4 the dot keeps close to FP32 working accuracy of the
// absolute sum instead of the growth with the length of a plain FP32 sum.
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void run() {}
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Acc<float> {
  float part = 0.f;               // the current run
  float hi = 0.f, lo = 0.f;       // compensated sum of the closed runs
  double tot = 0.0;
  __device__ __forceinline__ void add(float a, float b) { part = fmaf(a, b, part); }
  __device__ __forceinline__ void run() {
    const float s = __fadd_rn(hi, part);
    const float z = __fsub_rn(s, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(part, z));  // hi + part = s + se
    hi = s;
    lo = __fadd_rn(lo, se);
    part = 0.f;
  }
  __device__ __forceinline__ void flush() {
    run();
    tot += (double)hi + (double)lo;
    hi = 0.f;
    lo = 0.f;
  }
  __device__ __forceinline__ double value() const { return tot + (double)hi + (double)lo + (double)part; }
};

// Block-reduce NV values, publish the block's partials, and tell whether this
// block is the last one of the grid to finish (the classic threadfence
// reduction: no block ever waits for another).  Must be called by every
// thread of the block.
template <int NV, int NT = NTHREADS>
__device__ __forceinline__ bool publish_partials(double (&v)[NV], double* part, unsigned* ticket) {
  __shared__ double sm[NV][NT / 32];
  __shared__ bool last;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k][wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = (lane < NT / 32) ? sm[k][lane] : 0.0;
      v[k] = warp_sum(x);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) part[(long long)blockIdx.x * NV + k] = v[k];
      __threadfence();
      unsigned t = atomicAdd(ticket, 1u);
      last = (t == gridDim.x - 1);
    }
  }
  __syncthreads();
  return last;
}

// Block-reduce NV values of one work tile and store them at part[t*NV + k]
// (thread 0).  Kernels that hand out tiles dynamically reduce per tile, so the
// final sum (over tiles, in tile order) does not depend on which block ran
// which tile.  Must be called by every thread of the block.
template <int NV, int NT>
__device__ __forceinline__ void tile_partials(double (&v)[NV], double* part, long long t) {
  __shared__ double sm[NV][NT / 32];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();                 // sm[] may still be read from the previous tile
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k][wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = (lane < NT / 32) ? sm[k][lane] : 0.0;
      x = warp_sum(x);
      if (lane == 0) part[t * NV + k] = x;
    }
  }
}

// After every block stored its tile partials: is this the last block to finish?
template <int NT>
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// In the last block: sum the published partials in a fixed order (so results
// are reproducible run to run).  Result valid in thread 0.
template <int NV, int NT = NTHREADS>
__device__ __forceinline__ void gather_partials(const double* part, long long nblocks, double (&out)[NV]) {
  __shared__ double sm[NV][NT / 32];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (long long i = tid; i < nblocks; i += NT) {
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(part + (long long)i * NV + k);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = warp_sum(acc[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k][wid] = acc[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = (lane < NT / 32) ? sm[k][lane] : 0.0;
      out[k] = warp_sum(x);
    }
  }
}

// ------------------------------------------------------------- tile decoding

struct TileCoord {
  int x, y, z0, z1;
  bool active;
};

__device__ __forceinline__ TileCoord tile_coord(const Geo& g, long long t) {
  TileCoord c;
  int ix = (int)(t % g.tiles_x);
  long long r = t / g.tiles_x;
  int iy = (int)(r % g.tiles_y);
  int iz = (int)(r / g.tiles_y);
  c.x = ix * TX + threadIdx.x;
  c.y = iy * TY + threadIdx.y;
  c.z0 = iz * g.tz;
  c.z1 = min(c.z0 + g.tz, g.nz);
  c.active = (c.x < g.nx) && (c.y < g.ny);
  return c;
}

}  // namespace pf
