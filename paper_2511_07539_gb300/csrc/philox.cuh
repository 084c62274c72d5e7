// Philox4x64-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11,
// "Parallel random numbers: as easy as 1, 2, 3"): ten rounds of two 64x64->128
// multiplications; the key is bumped by the Weyl constants between rounds.
// Key (seed, 0); counter (packet id, draw index, 0, 0).  Each draw gives four
// uniforms in [0,1) from the top 53 bits of each output word.
#pragma once
#include <stdint.h>

// XT_FIXEXP_HOST compiles the generator for the host (a CPU test checks it
// against an independent implementation); CUDA builds never define it.
#ifdef XT_FIXEXP_HOST
#include "fixexp_host.h"
#define XT_PX static inline
#else
#define XT_PX __device__ __forceinline__
#endif

namespace xt {

struct U4 { double u[4]; };

XT_PX void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1, uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll 1   // rolled: the kernels that draw are large, and instruction fetch stalls them
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// (x >> 11) 2^-53 assembled from its bits with integer operations only (exact).
XT_PX double u01(uint64_t x) {
  const uint64_t m = x >> 11;
  if (m == 0) return 0.0;
  const int b = 63 - __clzll((long long)m);          // top bit, 0..52
  const uint64_t bits = ((uint64_t)(b - 53 + 1023) << 52) | ((m << (52 - b)) & ((1ull << 52) - 1ull));
  return __longlong_as_double((long long)bits);
}

// Raw words of draw e of a packet (the uniforms are their top 53 bits).
XT_PX void draw_raw(uint64_t seed, int64_t packet, uint64_t e, uint64_t x[4]) {
  philox4x64_10((uint64_t)packet, e, 0, 0, seed, 0, x);
}

XT_PX U4 draw(uint64_t seed, int64_t packet, uint64_t e) {
  uint64_t x[4];
  philox4x64_10((uint64_t)packet, e, 0, 0, seed, 0, x);
  U4 r;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.u[i] = u01(x[i]);
  return r;
}

}  // namespace xt
