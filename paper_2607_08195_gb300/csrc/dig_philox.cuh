// dig_philox.cuh -- the counter-based random numbers of every kernel:
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the uniform
// variates drawn from its words.  Every random number of the method is one
// word (or two) of philox(entity, sub, step, draw; seed_lo, seed_hi ^
// purpose << 24), so a result does not depend on launch shape or order.
#pragma once
#include <cstdint>

namespace dig {

__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                       uint32_t k1, uint32_t (&w)[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  w[0] = c0;
  w[1] = c1;
  w[2] = c2;
  w[3] = c3;
}

// uniform (0,1) from 23 bits of one word
__device__ __forceinline__ float u01f(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 1.1920928955078125e-07f; }

// uniform (0,1) from 52 bits of two words
__device__ __forceinline__ double u01d(uint32_t w0, uint32_t w1) {
  const unsigned long long k = ((unsigned long long)(w0 >> 4) << 24) | (unsigned long long)(w1 >> 8);
  return ((double)k + 0.5) * 2.220446049250313080847e-16;
}

}  // namespace dig
