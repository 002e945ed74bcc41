// Device side of the film batch (pf_batch_*): the per-step voltage ramps of
// the electrodes and the polarization-voltage loop record.
//
//   k_batch_ramp    every cell of a ramped z face of every film gets the
//                   common electrode voltage V = amp tri(s / period) of batch
//                   step s (tri: the unit triangle wave, 0 at 0, 1 at 1/4,
//                   -1 at 3/4); Neumann cells ignore their voltage.
//   k_batch_record  after the step: on every record_every-th batch step the
//                   mean P of every film (FP64 sums in a fixed order) is
//                   stored with the voltage it was driven by; the last block
//                   to finish advances the batch step counter.
// The paper drives switching by electrode voltages (Section Results); the
// loops are the observable of the hysteresis sweeps.
#include "pf_internal.h"

namespace pf {

__device__ __forceinline__ double tri_wave(double s) {
  double f = s - floor(s);
  if (f < 0.25) return 4.0 * f;
  if (f < 0.75) return 2.0 - 4.0 * f;
  return 4.0 * f - 4.0;
}

__device__ __forceinline__ double ramp_volts(const BatchFilm& f, long long step) {
  return f.amp * tri_wave((double)step / f.period);
}

__global__ void __launch_bounds__(256) k_batch_ramp(const BatchFilm* films, const BatchState* bs) {
  const BatchFilm f = films[blockIdx.y];
  if (!f.volt) return;
  const double v = ramp_volts(f, bs->step);
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < f.nxy; i += (long long)gridDim.x * 256) {
    if (f.fp32) static_cast<float*>(f.volt)[i] = (float)v;
    else static_cast<double*>(f.volt)[i] = v;
  }
}

constexpr int REC_THREADS = 256;

__global__ void __launch_bounds__(REC_THREADS) k_batch_record(const BatchFilm* films, int nfilms, int buf,
                                                              BatchState* bs, double* part, double* hist) {
  __shared__ double red[3][REC_THREADS / 32];
  __shared__ bool last;
  const long long step = bs->step;
  const bool rec = (step + 1) % bs->record_every == 0;
  const int fi = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
  const BatchFilm f = films[fi];
  double s[3] = {0.0, 0.0, 0.0};
  if (rec) {
    const long long chunk = (f.n + nb - 1) / nb;
    const long long lo = b * chunk, hi = min(f.n, lo + chunk);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (f.fp32) {
        const float* P = static_cast<const float*>(f.P[buf]) + c * f.n;
        for (long long i = lo + threadIdx.x; i < hi; i += REC_THREADS) s[c] += (double)P[i];
      } else {
        const double* P = static_cast<const double*>(f.P[buf]) + c * f.n;
        for (long long i = lo + threadIdx.x; i < hi; i += REC_THREADS) s[c] += P[i];
      }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s[c] = warp_sum(s[c]);
      if (lane == 0) red[c][wid] = s[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double t = 0.0;
        for (int w = 0; w < REC_THREADS / 32; ++w) t += red[c][w];
        part[((long long)fi * nb + b) * 3 + c] = t;
      }
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&bs->ticket, 1u) == (unsigned)(nb * nfilms - 1);
  }
  __syncthreads();
  if (!last) return;
  // the last block: every block has read the step counter and stored its sums
  if (rec) {
    const long long r = (step + 1) / bs->record_every - 1;
    for (int k = threadIdx.x; k < nfilms; k += REC_THREADS) {
      const BatchFilm g = films[k];
      double t[3] = {0.0, 0.0, 0.0};
      for (int j = 0; j < nb; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) t[c] += __ldcg(part + ((long long)k * nb + j) * 3 + c);
      if (r < bs->max_records) {
        double* h = hist + (r * nfilms + k) * 4;
        h[0] = g.volt ? ramp_volts(g, step) : 0.0;
        h[1] = t[0] / (double)g.n;
        h[2] = t[1] / (double)g.n;
        h[3] = t[2] / (double)g.n;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bs->ticket = 0u;
    if (rec) bs->records = (step + 1) / bs->record_every;
    bs->step = step + 1;
    __threadfence();
  }
}

void launch_batch_ramp(const BatchFilm* films, int nfilms, long long max_nxy, const BatchState* bs,
                       cudaStream_t st) {
  const long long bx = std::max<long long>(1, std::min<long long>((max_nxy + 255) / 256, 64));
  k_batch_ramp<<<dim3((unsigned)bx, (unsigned)nfilms), 256, 0, st>>>(films, bs);
}

void launch_batch_record(const BatchFilm* films, int nfilms, int buf, BatchState* bs, double* part, double* hist,
                         cudaStream_t st) {
  k_batch_record<<<dim3(BATCH_REC_BLOCKS, (unsigned)nfilms), REC_THREADS, 0, st>>>(films, nfilms, buf, bs, part,
                                                                                   hist);
}

}  // namespace pf
