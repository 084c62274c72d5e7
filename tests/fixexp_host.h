// Host definitions of the CUDA device intrinsics that the fixed-point routines
// use, so that a CPU test can compile them unchanged (with XT_FIXEXP_HOST).
// Test infrastructure only.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

static inline uint64_t __umul64hi(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}
static inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
static inline long long __double_as_longlong(double x) { long long r; memcpy(&r, &x, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; memcpy(&r, &x, 8); return r; }
static inline unsigned int __float_as_uint(float x) { unsigned int r; memcpy(&r, &x, 4); return r; }
static inline float __uint_as_float(unsigned int x) { float r; memcpy(&r, &x, 4); return r; }
static inline float __int_as_float(int x) { float r; memcpy(&r, &x, 4); return r; }
