// Order of the line list by frequency (host code, shared with a CPU test).
#pragma once
#include <stdint.h>
#include <string.h>

#include <vector>

namespace xt {

// order[s] = the caller index of the line at rank s in descending frequency,
// ties in ascending caller index: a stable LSD radix sort (8-bit digits) of
// the complemented bit patterns of nu, starting from the caller order.  The
// frequencies must be positive (or +0), so that they order as their bit
// patterns; passes whose digit is the same for every line are skipped.
inline void sort_lines_by_frequency(const double* nu, int n, int* order) {
  std::vector<uint64_t> key(n), key2(n);
  std::vector<int> o2(n);
  for (int l = 0; l < n; ++l) {
    uint64_t b;
    memcpy(&b, &nu[l], sizeof(b));
    key[l] = ~b;
    order[l] = l;
  }
  int* ord = order;
  int* alt = o2.data();
  for (int sh = 0; sh < 64; sh += 8) {
    size_t cnt[257] = {0};
    for (int i = 0; i < n; ++i) cnt[((key[i] >> sh) & 255u) + 1]++;
    if (n == 0 || cnt[((key[0] >> sh) & 255u) + 1] == (size_t)n) continue;
    for (int d = 0; d < 256; ++d) cnt[d + 1] += cnt[d];
    for (int i = 0; i < n; ++i) {
      const size_t pos = cnt[(key[i] >> sh) & 255u]++;
      key2[pos] = key[i];
      alt[pos] = ord[i];
    }
    key.swap(key2);
    int* t = ord;
    ord = alt;
    alt = t;
  }
  if (ord != order) memcpy(order, ord, sizeof(int) * (size_t)n);
}

}  // namespace xt
