// Packet quota of the emission (host code, shared with a CPU test).
#pragma once
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace xt {

// Largest-remainder integer quota of N packets over nc cells by luminosity L
// (serial host arithmetic in natural cell order): N L_c / sum L rounded down,
// the remaining packets to the largest fractional parts, ties to the lower
// cell.  Writes the prefix qoff [nc + 1]; frac [nc] and order [nc] are the
// caller's work space.  Allocates nothing.
inline void packet_quota(const double* L, int64_t nc, int64_t N, int64_t* qoff, double* frac,
                         int64_t* order) {
  double tot = 0.0;
  for (int64_t c = 0; c < nc; ++c) tot += L[c];
  int64_t used = 0;
  qoff[0] = 0;
  for (int64_t c = 0; c < nc; ++c) {
    const double q = tot > 0.0 ? ((double)N * L[c]) / tot : 0.0;
    const double fl = std::floor(q);
    qoff[c + 1] = (int64_t)fl;          // the cell's count until the prefix below
    frac[c] = q - fl;
    used += (int64_t)fl;
    order[c] = c;
  }
  const int64_t extra = std::min<int64_t>(N - used, nc);
  if (extra > 0) {
    // the extra packets go to the `extra` largest remainders, ties to the lower
    // cell (a total order, so selecting them needs no sort)
    auto cmp = [&](int64_t x, int64_t y) { return frac[x] > frac[y] || (frac[x] == frac[y] && x < y); };
    if (extra < nc) std::nth_element(order, order + (extra - 1), order + nc, cmp);
    for (int64_t k = 0; k < extra; ++k) qoff[order[k] + 1] += 1;
  }
  for (int64_t c = 0; c < nc; ++c) qoff[c + 1] += qoff[c];
}

// The same with vectors (run_transport).
inline void packet_quota(const std::vector<double>& L, int64_t N, std::vector<int64_t>& qoff) {
  const int64_t nc = (int64_t)L.size();
  std::vector<double> frac(nc);
  std::vector<int64_t> order(nc);
  qoff.assign(nc + 1, 0);
  packet_quota(L.data(), nc, N, qoff.data(), frac.data(), order.data());
}

}  // namespace xt
