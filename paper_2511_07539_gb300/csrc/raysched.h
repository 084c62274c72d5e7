// Order in which the spherical walk's refill hands out ray ids (host and
// device code; shared with a CPU test).
#pragma once
#include <stdint.h>

namespace xt {

// The ray id taken at id v of a launch's range [p_begin, p_begin + n) of the
// RAYS sampler's ids (id = (cell rank nbin + bin) nview + viewer): within
// every cell's block of nbin x nview ids that the range holds whole, the ids
// go viewer by viewer, bin after bin within a viewer; ids of a block the range
// holds only in part are taken in order.  A bijection of the range onto
// itself.
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int64_t ray_id_in_range(int64_t v, int64_t p_begin, int64_t n, int64_t nbin, int64_t nview) {
  const int64_t per_cell = nbin * nview;
  const int64_t lo = (v / per_cell) * per_cell;
  if (nview <= 1 || lo < p_begin || lo + per_cell > p_begin + n) return v;
  const int64_t rem = v - lo, kv = rem / nbin;
  return lo + (rem - kv * nbin) * nview + kv;
}

}  // namespace xt
