// e^-tau and 1 - e^-tau for tau > 0, computed on the integer pipe.
//
// GB300 executes FP64 arithmetic at about 1/64 of its FP32 rate, while 64-bit
// integer multiplies run on the wide integer pipe.  The attenuation factor of
// every line event is therefore evaluated in 63-bit fixed point:
//   tau = k ln2 + r,  0 <= r < ln2           (integer range reduction, ln2 to ~2^-117)
//   r   = j/64 + s,   0 <= s < 1/64          (table of e^-j/64, after Tang's
//                                             table-driven method, ACM TOMS 15, 1989)
//   e^-s by its Taylor series to s^9/9! (< 2^-72) in Horner form,
//   e^-tau = 2^-k e^-j/64 e^-s, rounded once to double.
// The complement 1 - e^-tau = 1 - 2^-k e^-r is formed in fixed point too (for
// tau < ln2 exactly, so it keeps full relative precision for small tau; for
// larger tau it is at least 1/2 and the dropped bits of 2^-k e^-r are below
// 2^-63).  Both results are within about one ulp of the correctly rounded
// values; tau >= 709 gives e^-tau = 0.  The tables are computed on the host
// (xt::fixexp_tables).
#pragma once
#include <math.h>
#include <stdint.h>

// XT_FIXEXP_HOST compiles these routines for the host (a CPU test checks them
// against extended-precision references); the header it includes defines the
// device intrinsics used below, and the FP32 approximations become the
// correctly rounded host operations.  CUDA builds never define it.
#ifdef XT_FIXEXP_HOST
#include "fixexp_host.h"
#define XT_FX static inline
#else
#define XT_FX __device__ __forceinline__
#endif

namespace xt {

struct FixExpTables {
  uint64_t tab[48];     // e^-j/64, j = 0..47, Q63
  uint64_t fact[10];    // 1/n!, n = 0..9, Q63
  uint64_t ln2_a;       // floor(ln2 2^53)
  uint64_t ln2_b;       // next 64 bits of ln2 2^53
};

struct FixTrigTables {
  uint64_t sin_t[65];   // sin(j pi/256), j = 0..64, Q63
  uint64_t cos_t[65];   // cos(j pi/256), Q63
  uint64_t pi4;         // pi/4 in Q63
  uint64_t inv[8];      // 1/(m(m+1)) for m = 1..8 (Taylor factors), Q63
};

// Tables of the fixed-point exponential (host).  ln2 from its series
// sum 1/(i 2^i) in Q127 integer arithmetic; 1/n! by exact integer division;
// e^-j/64 from the host's extended-precision expl (64 or more mantissa bits).
inline void fixexp_tables(FixExpTables* t) {
  typedef unsigned __int128 u128;
  u128 ln2 = 0;
  for (int i = 1; i < 127; ++i) ln2 += (((u128)1) << (127 - i)) / (u128)i;   // ln2 2^127
  t->ln2_a = (uint64_t)(ln2 >> 74);                    // ln2 2^53
  t->ln2_b = (uint64_t)(ln2 >> 10);                    // next 64 bits
  const u128 one = ((u128)1) << 63;
  u128 f = 1;
  for (int n = 0; n < 10; ++n) {
    if (n > 0) f *= (u128)n;
    t->fact[n] = (uint64_t)((one + f / 2) / f);
  }
  for (int j = 0; j < 48; ++j) {
    long double v = expl(-(long double)j / 64.0L) * 9223372036854775808.0L;
    t->tab[j] = (uint64_t)(v + 0.5L);
  }
}

// Tables of the fixed-point sine/cosine (host), from the host's
// extended-precision sinl/cosl and M_PIl; Taylor factors by integer division.
inline void fixtrig_tables(FixTrigTables* t) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double q63 = 9223372036854775808.0L;
  for (int j = 0; j <= 64; ++j) {
    t->sin_t[j] = (uint64_t)(sinl(pi * j / 256.0L) * q63 + 0.5L);
    t->cos_t[j] = (uint64_t)(cosl(pi * j / 256.0L) * q63 + 0.5L);
  }
  t->pi4 = (uint64_t)(pi / 4.0L * q63 + 0.5L);
  typedef unsigned __int128 u128;
  const u128 one = ((u128)1) << 63;
  for (int m = 1; m <= 8; ++m) {
    const u128 den = (u128)m * (u128)(m + 1);
    t->inv[m - 1] = (uint64_t)((one + den / 2) / den);
  }
}


XT_FX uint64_t mul_q63(uint64_t a, uint64_t b) {
  const uint64_t hi = __umul64hi(a, b), lo = a * b;
  return (hi << 1) | (lo >> 63);
}

// q * 2^-63 * 2^scale as a double, rounded to nearest even; 0 below 2^-1022.
XT_FX double q63_to_double(uint64_t q, int scale) {
  if (q == 0) return 0.0;
  const int b = 63 - __clzll((long long)q);
  int e = b - 63 + scale;
  uint64_t m;
  if (b > 52) {
    const int sh = b - 52;
    const uint64_t rem = q & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m = q >> sh;
    if (rem > half || (rem == half && (m & 1ull))) {
      m += 1ull;
      if (m >> 53) { m >>= 1; e += 1; }
    }
  } else {
    m = q << (52 - b);
  }
  if (e < -1022) return 0.0;
  return __longlong_as_double((long long)(((uint64_t)(e + 1023) << 52) | (m & ((1ull << 52) - 1ull))));
}

// tau > 0 (finite).  Writes e^-tau and 1 - e^-tau.
XT_FX void expneg(const FixExpTables& T, double tau, double& ex, double& ome) {
  // range tests on the bit pattern (tau > 0: integer order = numeric order)
  const uint64_t bits = (uint64_t)__double_as_longlong(tau);
  if (bits >= (uint64_t)__double_as_longlong(709.0)) { ex = 0.0; ome = 1.0; return; }
  const int eb = (int)(bits >> 52);                        // biased exponent (tau normal, > 0)
  const uint64_t m = (bits & ((1ull << 52) - 1ull)) | (1ull << 52);
  uint64_t R;                                              // r in Q63
  int k = 0;
  if (bits < (uint64_t)__double_as_longlong(0.6931471805599453)) {
    const int sh = eb - 1012;                              // tau 2^63 = m 2^(eb-1012)
    if (sh >= 0) R = m << sh;
    else if (sh > -64) R = (m >> (-sh)) + ((m >> (-sh - 1)) & 1ull);
    else R = 0;
  } else {
    const uint64_t T53 = m << (eb - 1022);                 // tau 2^53, exact (tau >= 0.69)
    // k = floor(tau / ln2) from a float estimate (off by at most one), then
    // corrected; r = tau - k ln2 with ln2 carried to 117 bits, in Q63
    const float tf = __int_as_float((int)((((uint32_t)(eb - 1023 + 127)) << 23) |
                                          ((uint32_t)(m >> 29) & 0x7FFFFFu)));
    k = (int)(tf * 1.44269504f);
    const uint64_t ln2_q63 = (T.ln2_a << 10) | (T.ln2_b >> 54);
    // r53 and rc below never under-estimate r (the dropped parts of k ln2 are
    // only subtracted truncated), so a k that is one too small always shows
    // r >= ln2 and the corrections cannot oscillate.
    int64_t Rs = 0;
    for (int it = 0; it < 4; ++it) {
      const uint64_t kk = (uint64_t)k;
      const int64_t r53 = (int64_t)(T53 - kk * T.ln2_a) - (int64_t)__umul64hi(kk, T.ln2_b);
      if (r53 < 0) { --k; continue; }
      if ((uint64_t)r53 > T.ln2_a + 1) { ++k; continue; }
      const int64_t rc = (r53 << 10) - (int64_t)((kk * T.ln2_b) >> 54);
      if (rc < 0) { --k; continue; }
      if ((uint64_t)rc > ln2_q63) { ++k; continue; }
      Rs = rc;
      break;
    }
    R = (uint64_t)Rs;
  }
  const int j = (int)(R >> 57);                            // R <= ln2 2^63 -> j <= 44
  const uint64_t s = R & ((1ull << 57) - 1ull);            // s < 2^-6 in Q63
  uint64_t p = T.fact[9];
#pragma unroll
  for (int n = 8; n >= 0; --n) p = T.fact[n] - mul_q63(s, p);   // all partial sums stay positive
  const uint64_t E = mul_q63(T.tab[j], p);                 // e^-r in Q63, in (1/2, 1]
  ex = q63_to_double(E, -k);
  ome = q63_to_double((1ull << 63) - (k < 64 ? E >> k : 0ull), 0);
}

// sin(2 pi u) and cos(2 pi u) for u = U 2^-53, 0 <= U < 2^53, in fixed point.
// The octant comes from the top three bits of U (exact); within it the angle
// beta <= pi/4 is split into j pi/256 (tables) plus delta < pi/256, whose sine
// and cosine are Taylor series to delta^8 (next term < 2^-72), combined by the
// angle-addition formulas; octant symmetries give the signs.  Results are
// within about one ulp of sin and cos of the exact angle 2 pi u.
// sincos_2pi_q63 leaves sin and cos of the angle within its quadrant in Q63
// and returns the quadrant (0..3); quadrant_signs maps them to the full angle.
XT_FX int sincos_2pi_q63(const FixTrigTables& T, uint64_t U, uint64_t& sa,
                                              uint64_t& ca) {
  const int oct = (int)(U >> 50);
  uint64_t g = U & ((1ull << 50) - 1ull);                  // fraction of the octant, Q50
  if (oct & 1) g = (1ull << 50) - g;                       // reflect: beta = pi/4 - theta
  const int j = (int)(g >> 44);                            // 0..64
  const uint64_t b = (g & ((1ull << 44) - 1ull)) << 13;    // Q63, < 2^-6
  const uint64_t d = mul_q63(b, T.pi4);                    // delta, Q63, < pi/256
  const uint64_t d2 = mul_q63(d, d);
  // sin delta = d (1 - d2/(2.3) (1 - d2/(4.5) (1 - d2/(6.7) (1 - d2/(8.9)))))
  uint64_t ps = (1ull << 63) - mul_q63(d2, T.inv[7]);
  ps = (1ull << 63) - mul_q63(mul_q63(d2, T.inv[5]), ps);
  ps = (1ull << 63) - mul_q63(mul_q63(d2, T.inv[3]), ps);
  ps = (1ull << 63) - mul_q63(mul_q63(d2, T.inv[1]), ps);
  const uint64_t sd = mul_q63(d, ps);
  // cos delta = 1 - d2/(1.2) (1 - d2/(3.4) (1 - d2/(5.6) (1 - d2/(7.8))))
  uint64_t pc = (1ull << 63) - mul_q63(d2, T.inv[6]);
  pc = (1ull << 63) - mul_q63(mul_q63(d2, T.inv[4]), pc);
  pc = (1ull << 63) - mul_q63(mul_q63(d2, T.inv[2]), pc);
  const uint64_t cd = (1ull << 63) - mul_q63(mul_q63(d2, T.inv[0]), pc);
  const uint64_t sb = mul_q63(T.sin_t[j], cd) + mul_q63(T.cos_t[j], sd);   // sin beta
  const uint64_t cb = mul_q63(T.cos_t[j], cd) - mul_q63(T.sin_t[j], sd);   // cos beta
  // angle within the quadrant: alpha = beta (even octant) or pi/2 - beta (odd)
  sa = (oct & 1) ? cb : sb;
  ca = (oct & 1) ? sb : cb;
  return oct >> 1;
}

// -x by flipping the sign bit (an FP64 negation would take a slot of the
// FP64 pipe)
XT_FX double neg_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

XT_FX void quadrant_signs(int q, double vs, double vc, double& s, double& c) {
  switch (q) {
    case 0: s = vs; c = vc; break;
    case 1: s = vc; c = neg_bits(vs); break;
    case 2: s = neg_bits(vs); c = neg_bits(vc); break;
    default: s = neg_bits(vc); c = vs; break;
  }
}

XT_FX void sincos_2pi(const FixTrigTables& T, uint64_t U, double& s, double& c) {
  uint64_t sa, ca;
  const int q = sincos_2pi_q63(T, U, sa, ca);
  quadrant_signs(q, q63_to_double(sa, 0), q63_to_double(ca, 0), s, c);
}

// ---- quotient and square root on the integer pipe ---------------------------
// Q63 value of 1/m for M = m 2^62, 1 <= m < 2.  The seed is the FP32 reciprocal
// approximation of m (rcp.approx, about 23 correct bits); two Newton-Raphson
// steps y <- y (2 - m y), each doubling the correct bits, run in 64-bit fixed
// point, whose truncations keep the result within about 2^-61 relative.
XT_FX uint64_t float_to_q63(float y) {     // 0.5 <= y <= 1
  const uint32_t yb = __float_as_uint(y);
  const int e = (int)(yb >> 23) - 127;                            // -1 or 0
  return (uint64_t)((yb & 0x7FFFFFu) | 0x800000u) << (40 + e);
}

XT_FX uint64_t rcp_q63(uint64_t M) {
  const float f = __uint_as_float((127u << 23) | (uint32_t)((M >> 39) & 0x7FFFFFu));
  float y;
#ifdef XT_FIXEXP_HOST
  y = 1.0f / f;
#else
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
#endif
  uint64_t Y = float_to_q63(y);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const uint64_t my = (__umul64hi(M, Y) << 1) | ((M * Y) >> 63);     // m y, Q62
    const uint64_t E = (1ull << 63) - my;                              // 2 - m y, Q62
    Y = (__umul64hi(Y, E) << 2) | ((Y * E) >> 62);                     // Q63
  }
  return Y;
}

// a / b for positive normal doubles: the significands' quotient from the
// reciprocal above and one 64 x 64-bit product, rounded once to nearest.  The
// reciprocal's error (< 2^-60) can move the rounding only for quotients within
// 2^-7 ulp of a midpoint, so the result is within 0.51 ulp of a / b.  A result
// outside the normal range (also an infinite or NaN b) is left to the IEEE
// division.  Zero, subnormal or negative operands are not handled: every
// caller's operands are positive normal by construction (frequencies, packet
// energies, wall spacings, optical depths >= 2^-10, rates), and a check here
// cost the trace kernel 3 % (measured).
XT_FX double div_pos(double a, double b) {
  const uint64_t ab = (uint64_t)__double_as_longlong(a), bb = (uint64_t)__double_as_longlong(b);
  const uint64_t frac = (1ull << 52) - 1ull;
  const uint64_t ma = (ab & frac) | (1ull << 52), mb = (bb & frac) | (1ull << 52);
  const uint64_t Y = rcp_q63(mb << 10);                // 2^115 / mb
  const uint64_t q = __umul64hi(ma << 11, Y);          // (ma / mb) 2^62, in (2^61, 2^63)
  int e = (int)(ab >> 52) - (int)(bb >> 52) + 1023;
  uint64_t m;
  if (q >> 62) {
    m = (q >> 10) + ((q >> 9) & 1ull);
  } else {
    m = (q >> 9) + ((q >> 8) & 1ull);
    --e;
  }
  if (m >> 53) { m >>= 1; ++e; }
  if (e <= 0 || e >= 2047) return a / b;
  return __longlong_as_double((long long)(((uint64_t)e << 52) | (m & frac)));
}

// beta_S(tau) (Eq. beta_Sobolev) and, if dbeta is not null, d beta_S / d tau,
// without FP64 transcendentals or divisions: for tau >= 2^-10, e^-tau and
// 1 - e^-tau in fixed point (expneg) and the quotients beta = (1 - e^-tau) / tau,
// beta' = -(1 - e^-tau - tau e^-tau) / tau^2 on the integer pipe (div_pos);
// below 2^-10 the Taylor series beta = sum (-tau)^k / (k+1)! and its derivative
// to the tau^4 terms (the next terms are below 2e-18 relative).  beta = 1 and
// beta' = 0 for tau <= 0 (no trapping).
XT_FX double sobolev_beta_fix(const FixExpTables& fx, double tau, double* dbeta) {
  const long long tb = __double_as_longlong(tau);
  if (tb <= 0) {                                   // tau <= +0 (or negative)
    if (dbeta) *dbeta = 0.0;
    return 1.0;
  }
  if (tb < __double_as_longlong(0x1p-10)) {
    if (dbeta) *dbeta = fma(tau, fma(tau, fma(tau, fma(tau, -1.0 / 144.0, 1.0 / 30.0), -0.125), 1.0 / 3.0), -0.5);
    return fma(tau, fma(tau, fma(tau, fma(tau, 1.0 / 120.0, -1.0 / 24.0), 1.0 / 6.0), -0.5), 1.0);
  }
  double ex, ome;
  expneg(fx, tau, ex, ome);
  if (dbeta) *dbeta = neg_bits(div_pos(fma(-tau, ex, ome), tau * tau));
  return div_pos(ome, tau);
}

// w 2^k rounded to FP32 (to nearest even) with integer operations: the
// exponent is shifted, the significand rounded from 52 bits to those FP32 keeps
// (23, or fewer for results in the subnormal range, as a plain conversion
// does); w must be finite and w 2^k < 2^127.
XT_FX float scaled_f32(double w, int k) {
  const uint64_t b = (uint64_t)__double_as_longlong(w);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return __uint_as_float(sign);
  const int ef = e - 1023 + k + 127;              // biased FP32 exponent
  const uint64_t M = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
  // keep M >> sh: sh = 29 for a normal result, 30 - ef below the normal range;
  // the FP32 bits are then (ef << 23) + kept (a carry out of the significand
  // steps the exponent, and a subnormal that rounds up to 2^-126 becomes normal)
  const int sh = ef > 0 ? 29 : 30 - ef;
  if (sh > 54) return __uint_as_float(sign);
  const uint64_t kept = M >> sh, rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  uint32_t m = (uint32_t)kept + ((rem > half || (rem == half && (kept & 1ull))) ? 1u : 0u);
  if (ef > 0) m += ((uint32_t)(ef - 1) << 23);   // the hidden bit of kept adds the last 1
  return __uint_as_float(sign | m);
}

// Direction of an isotropic emission from the 53-bit integers of its two
// uniforms, u = Umu 2^-53 and u' = Uphi 2^-53: mu = 2u - 1, phi = 2 pi u'.
// mu is exact; sin(theta) = sqrt(1 - mu^2) = 2^-52 sqrt(X) with the exact
// 106-bit X = Umu (2^53 - Umu); its square root comes from Newton-Raphson on
// 1/sqrt (FP32 seed, y <- y (3 - a y^2) / 2 twice) in fixed point, and
// n_x = sin(theta) cos(phi), n_y = sin(theta) sin(phi) are formed in Q63 and
// rounded once.  No FP64 arithmetic.
XT_FX void isotropic_fix(const FixTrigTables& T, uint64_t Umu, uint64_t Uphi,
                                              double n[3]) {
  const uint64_t two53 = 1ull << 53;
  const uint64_t t2 = 2 * Umu;
  const double mu_mag = q63_to_double(t2 >= two53 ? t2 - two53 : two53 - t2, 10);
  n[2] = t2 >= two53 ? mu_mag : neg_bits(mu_mag);
  uint64_t sa, ca;
  const int q = sincos_2pi_q63(T, Uphi, sa, ca);
  if (Umu == 0) { n[0] = 0.0; n[1] = 0.0; return; }  // mu = -1
  const uint64_t Uc = two53 - Umu;
  const uint64_t hi = __umul64hi(Umu, Uc), lo = Umu * Uc;              // X < 2^104
  const int top = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  int b0 = top - 63;
  b0 += b0 & 1;                                                          // even: X ~ xm 2^b0
  const uint64_t xm = b0 > 0 ? (hi << (64 - b0)) | (lo >> b0) : lo << (-b0);   // [2^62, 2^64)
  const int ea = (int)(xm >> 63);                                        // a = xm 2^-62 in [1, 4)
  const float f = __uint_as_float(((uint32_t)(127 + ea) << 23) |
                                  (uint32_t)((xm >> (39 + ea)) & 0x7FFFFFu));
  float y;
#ifdef XT_FIXEXP_HOST
  y = 1.0f / sqrtf(f);
#else
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
#endif
  uint64_t Y = float_to_q63(y);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const uint64_t Y2 = mul_q63(Y, Y);
    const uint64_t H = (__umul64hi(xm, Y2) << 1) | ((xm * Y2) >> 63);   // a y^2, Q62
    const uint64_t G = 0xC000000000000000ull - H;                        // 3 - a y^2, Q62
    Y = (__umul64hi(Y, G) << 1) | ((Y * G) >> 63);                       // y (3 - a y^2) / 2, Q63
  }
  const uint64_t S = (__umul64hi(xm, Y) << 1) | ((xm * Y) >> 63);       // sqrt(a), Q62
  const int sc = b0 / 2 - 20;                     // sin(theta) = S 2^-63 2^sc
  double vs, vc;
  quadrant_signs(q, q63_to_double(mul_q63(S, sa), sc), q63_to_double(mul_q63(S, ca), sc), vs, vc);
  n[0] = vc;
  n[1] = vs;
}

}  // namespace xt
