// Packet quota of the emission (host code, shared with a CPU test).
#pragma once
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace xt {

// Largest-remainder integer quota of N packets over cells by luminosity
// (serial host arithmetic in natural cell order).
inline void packet_quota(const std::vector<double>& L, int64_t N, std::vector<int64_t>& qoff) {
  const int64_t nc = (int64_t)L.size();
  double tot = 0.0;
  for (int64_t c = 0; c < nc; ++c) tot += L[c];
  std::vector<int64_t> n(nc);
  std::vector<double> frac(nc);
  int64_t used = 0;
  for (int64_t c = 0; c < nc; ++c) {
    const double q = tot > 0.0 ? ((double)N * L[c]) / tot : 0.0;
    const double fl = std::floor(q);
    n[c] = (int64_t)fl;
    frac[c] = q - fl;
    used += n[c];
  }
  std::vector<int64_t> order(nc);
  std::iota(order.begin(), order.end(), 0);
  const int64_t extra = std::min<int64_t>(N - used, nc);
  if (extra > 0) {
    // the extra packets go to the `extra` largest remainders, ties to the lower
    // cell (a total order, so selecting them needs no sort)
    auto cmp = [&](int64_t x, int64_t y) { return frac[x] > frac[y] || (frac[x] == frac[y] && x < y); };
    if (extra < nc) std::nth_element(order.begin(), order.begin() + (extra - 1), order.end(), cmp);
    for (int64_t k = 0; k < extra; ++k) n[order[k]] += 1;
  }
  qoff.assign(nc + 1, 0);
  for (int64_t c = 0; c < nc; ++c) qoff[c + 1] = qoff[c] + n[c];
}

}  // namespace xt
