// Grouping policy of the request server (host code only, no CUDA): how many
// queued requests of the same problem join the one just admitted.  Kept apart
// from server.cu so it can be checked on the CPU.
#pragma once
#include <cstddef>

namespace hz {

// Largest group the host staging allows: the group's sources and solutions
// are staged on the host as N x size complex doubles each (16 bytes per
// value), at most 1 GiB each; group_max is a power of two.
inline int group_cap(int group_max, long long nodes) {
  int cap = group_max;
  while (cap > 1 && (double)nodes * cap * 16.0 > (double)(1u << 30)) cap >>= 1;
  return cap;
}

// The group size for a request admitted while `candidates` queued requests of
// its problem wait (already limited to cap - 1): the largest power of two k
// <= 1 + candidates whose context bytes, bytes_for(k), fit the budget once the
// request's own admitted bytes (held) are replaced by them; 1 = alone (also
// when bytes_for throws).  *bytes receives bytes_for(k) for k >= 2.
template <typename BytesFor>
int group_size_for(int candidates, std::size_t in_use, std::size_t held, std::size_t budget, BytesFor&& bytes_for,
                   std::size_t* bytes) {
  int k = 1;
  while (2 * k <= candidates + 1) k *= 2;
  for (; k >= 2; k /= 2) {
    std::size_t b = 0;
    try {
      b = bytes_for(k);
    } catch (...) {
      return 1;
    }
    if (in_use - held + b <= budget) {
      *bytes = b;
      return k;
    }
  }
  return 1;
}

}  // namespace hz
