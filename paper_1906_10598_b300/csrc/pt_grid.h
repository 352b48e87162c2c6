// Grid shape of the objective launch (host side).
#pragma once

#include <algorithm>
#include <cstdint>

namespace pt {

// Tiles per CTA of an objective launch over `ntiles` tiles and `ny` candidate
// columns, with `slots` CTAs resident at once (SMs x CTAs per SM). A small
// block gets about two CTAs per slot in all (at most 32 tiles each). A block
// that fills more than that at 32 tiles per CTA takes the count from 32 to 48
// that ends soonest. The model charges each CTA its tiles plus about one
// tile's worth of set-up and staging, and counts whole waves of `slots` CTAs,
// so the last wave is not left mostly empty. (The 400K block against 4096
// candidates on 296 slots: 34 tiles, 1472 CTAs in 5 waves, instead of 32
// tiles and 1568 CTAs in 6.) `fits(t)` says whether t tiles fit the shared
// memory. The sums are exact fixed-point integers, so the choice never
// changes a result.
template <class Fits>
inline int objective_tiles_per_cta(int64_t ntiles, int ny, int slots, Fits fits) {
  const int64_t want = 2LL * slots;
  const int64_t t0 = std::max<int64_t>(1, std::min<int64_t>((ntiles * ny + want - 1) / want, 32));
  if (t0 < 32 || slots <= 0) return (int)t0;
  auto cost = [&](int64_t t) {
    const int64_t nx = (ntiles + t - 1) / t;
    return (nx * ny + slots - 1) / slots * (t + 1);
  };
  int64_t best = t0;
  for (int64_t t = 33; t <= 48; ++t)
    if (fits((int)t) && cost(t) < cost(best)) best = t;
  return (int)best;
}

}  // namespace pt
