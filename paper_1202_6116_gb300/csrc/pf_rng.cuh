// Counter-based normal variates for the thermal random force of Eq. TDGL.
//
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): ten rounds on a 4 x 32-bit counter with a
// 2 x 32-bit key; each round multiplies counter words 0 and 2 by the round
// multipliers into 64-bit products and recombines the halves with words 1
// and 3 and the key, and the key is bumped by the two Weyl constants between
// rounds.  Counter = (cell index, step index), key = seed, so every cell,
// step and seed has its own independent block of four words.  Normal
// variates come from the Box-Muller transform (Box & Muller 1958) of the two
// word pairs, the first word of a pair mapped to (0, 1], the second to [0, 1).
#pragma once

#include <stdint.h>

namespace pf {

__device__ __forceinline__ uint4 philox4x32_10(unsigned long long cell, unsigned long long step,
                                               unsigned long long seed) {
  unsigned c0 = (unsigned)cell, c1 = (unsigned)(cell >> 32), c2 = (unsigned)step, c3 = (unsigned)(step >> 32);
  unsigned k0 = (unsigned)seed, k1 = (unsigned)(seed >> 32);
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const unsigned lo2 = 0xCD9E8D57u * c2, hi2 = __umulhi(0xCD9E8D57u, c2);
    const unsigned n0 = hi2 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo2;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Three standard normal variates of (cell, step, seed) in the precision T.
template <typename T>
__device__ __forceinline__ void gauss3(unsigned long long cell, unsigned long long step, unsigned long long seed,
                                       T (&g)[3]);

template <>
__device__ __forceinline__ void gauss3<double>(unsigned long long cell, unsigned long long step,
                                               unsigned long long seed, double (&g)[3]) {
  const uint4 x = philox4x32_10(cell, step, seed);
  const double two32 = 4294967296.0, twopi = 6.283185307179586;
  const double r0 = sqrt(-2.0 * log(((double)x.x + 1.0) / two32));
  const double a0 = twopi * ((double)x.y / two32);
  const double r1 = sqrt(-2.0 * log(((double)x.z + 1.0) / two32));
  const double a1 = twopi * ((double)x.w / two32);
  g[0] = r0 * cos(a0);
  g[1] = r0 * sin(a0);
  g[2] = r1 * cos(a1);
}

template <>
__device__ __forceinline__ void gauss3<float>(unsigned long long cell, unsigned long long step,
                                              unsigned long long seed, float (&g)[3]) {
  const uint4 x = philox4x32_10(cell, step, seed);
  const float s32 = 2.3283064365386963e-10f;            // 2^-32
  const float r0 = sqrtf(-2.0f * logf(fmaf((float)x.x, s32, s32)));
  const float a0 = 6.2831853071795865f * ((float)x.y * s32);
  const float r1 = sqrtf(-2.0f * logf(fmaf((float)x.z, s32, s32)));
  const float a1 = 6.2831853071795865f * ((float)x.w * s32);
  float s0, c0, s1, c1;
  sincosf(a0, &s0, &c0);
  sincosf(a1, &s1, &c1);
  g[0] = r0 * c0;
  g[1] = r0 * s0;
  g[2] = r1 * c1;
}

}  // namespace pf
