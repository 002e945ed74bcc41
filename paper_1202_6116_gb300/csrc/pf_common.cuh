// Internal device helpers of the GPU library: grid geometry, boundary masks,
// FP64-accurate reductions and the solver scalar block.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

// Tile of one thread block: TX x TY columns of TZ cells (x fastest).
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NTHREADS = TX * TY;

struct Geo {
  int nx, ny, nz;
  int periodic_z;
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

// Inverse Jacobi diagonal when eps = 1: the diagonal is (number of interior
// faces + 2 * number of Dirichlet faces) / dx^2, an integer 3..8 times ih2.
template <typename T>
struct InvDiagTable {
  T v[9];
};

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
  int pad[4];
};

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Dot-product accumulators.  FP64 fields: plain FMA accumulation.  FP32
// fields: the compensated dot product "Dot2" of Ogita, Rump & Oishi (SIAM J.
// Sci. Comput. 26, 2005) -- the exact product by TwoProduct (one FMA) and a
// TwoSum of the running sum, with the error terms collected in a second
// float -- flushed into an FP64 total after every short run of cells, so the
// FP64 unit sees a handful of adds per column instead of one per cell.
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  double tot = 0.0;
  __device__ __forceinline__ void add(float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);            // a*b = p + pe exactly
    float s = __fadd_rn(hi, p);
    float z = __fsub_rn(s, hi);
    float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(p, z));  // hi + p = s + se
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(pe, se));
  }
  __device__ __forceinline__ void flush() {
    tot += (double)hi + (double)lo;
    hi = 0.f;
    lo = 0.f;
  }
  __device__ __forceinline__ double value() const { return tot + (double)hi + (double)lo; }
};

// Block-reduce NV values, publish the block's partials, and tell whether this
// block is the last one of the grid to finish (the classic threadfence
// reduction: no block ever waits for another).  Must be called by every
// thread of the block.
template <int NV>
__device__ __forceinline__ bool publish_partials(double (&v)[NV], double* part, unsigned* ticket) {
  __shared__ double sm[NV][NTHREADS / 32];
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
      double x = (lane < NTHREADS / 32) ? sm[k][lane] : 0.0;
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

// In the last block: sum the published partials in a fixed order (so results
// are reproducible run to run).  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void gather_partials(const double* part, int nblocks, double (&out)[NV]) {
  __shared__ double sm[NV][NTHREADS / 32];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int i = tid; i < nblocks; i += NTHREADS) {
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
      double x = (lane < NTHREADS / 32) ? sm[k][lane] : 0.0;
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
