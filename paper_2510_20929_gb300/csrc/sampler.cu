// Minibatch samplers (Pty-Chi Sec. 2.1: random, uniform and compact batches).
// Host code: they produce the `order` array the epoch entry points consume,
// whose consecutive chunks of `batch` entries are the minibatches.
//   random:  a seeded permutation (Fisher-Yates driven by SplitMix64).
//   compact: spatially connected clusters. The positions are split
//            recursively at an index along the longer side of their bounding
//            box (stable sort by that coordinate) so that every cluster but
//            the last holds exactly `batch` positions; each cluster is one
//            minibatch.
//   uniform: `batch` compact clusters of balanced size; minibatch t takes the
//            t-th position of every cluster, so each minibatch samples the
//            whole scan field evenly.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ptycho.h"

namespace ptycho {
namespace {

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): state += golden gamma, then
// two xor-shift-multiply rounds.
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

struct Range {
  int lo, hi;
};

// Splits idx[lo, hi) into `groups` spatial clusters. With `cap` > 0 the left
// part of every split holds exactly g1 * cap positions (full clusters first);
// otherwise the parts are proportional to the group counts.
void kd_split(const float* pos, std::vector<int>& idx, int lo, int hi, int groups, int cap, std::vector<Range>& out) {
  const int n = hi - lo;
  if (groups <= 1 || n <= 1) {
    out.push_back({lo, hi});
    return;
  }
  float ymin = pos[2 * idx[lo]], ymax = ymin, xmin = pos[2 * idx[lo] + 1], xmax = xmin;
  for (int i = lo + 1; i < hi; ++i) {
    const float y = pos[2 * idx[i]], x = pos[2 * idx[i] + 1];
    ymin = std::min(ymin, y); ymax = std::max(ymax, y);
    xmin = std::min(xmin, x); xmax = std::max(xmax, x);
  }
  const int axis = (ymax - ymin >= xmax - xmin) ? 0 : 1;
  std::stable_sort(idx.begin() + lo, idx.begin() + hi,
                   [&](int a, int b) { return pos[2 * a + axis] < pos[2 * b + axis]; });
  const int g1 = groups / 2, g2 = groups - g1;
  int n1 = cap > 0 ? std::min(n, g1 * cap) : (int)(((int64_t)n * g1 + groups / 2) / groups);
  kd_split(pos, idx, lo, lo + n1, g1, cap, out);
  kd_split(pos, idx, lo + n1, hi, g2, cap, out);
}

}  // namespace
}  // namespace ptycho

using namespace ptycho;

extern "C" ptycho_status ptycho_sampler_order(const float* pos, int32_t J, int32_t batch, int32_t kind, uint64_t seed,
                                              int32_t* order) {
  if (J < 0 || batch < 1 || (J > 0 && (!pos || !order))) return PTYCHO_ERR_ARG;
  if (kind != PTYCHO_SAMPLER_RANDOM && kind != PTYCHO_SAMPLER_UNIFORM && kind != PTYCHO_SAMPLER_COMPACT)
    return PTYCHO_ERR_ARG;
  for (int j = 0; j < 2 * J; ++j)
    if (!std::isfinite(pos[j])) return PTYCHO_ERR_ARG;
  std::vector<int> idx(J);
  for (int j = 0; j < J; ++j) idx[j] = j;
  if (kind == PTYCHO_SAMPLER_RANDOM) {
    SplitMix64 rng{seed};
    for (int i = J - 1; i > 0; --i) {
      const int k = (int)(rng.next() % (uint64_t)(i + 1));
      std::swap(idx[i], idx[k]);
    }
    for (int j = 0; j < J; ++j) order[j] = idx[j];
    return PTYCHO_OK;
  }
  std::vector<Range> groups;
  if (kind == PTYCHO_SAMPLER_COMPACT) {
    kd_split(pos, idx, 0, J, (J + batch - 1) / batch, batch, groups);
    for (int j = 0; j < J; ++j) order[j] = idx[j];
    return PTYCHO_OK;
  }
  // uniform: `batch` balanced clusters, read round-robin
  kd_split(pos, idx, 0, J, std::min(batch, std::max(J, 1)), 0, groups);
  int longest = 0;
  for (const Range& g : groups) longest = std::max(longest, g.hi - g.lo);
  int w = 0;
  for (int t = 0; t < longest; ++t)
    for (const Range& g : groups)
      if (g.lo + t < g.hi) order[w++] = idx[g.lo + t];
  return PTYCHO_OK;
}
