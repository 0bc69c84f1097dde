// Compares the compile-time P2 prolongation weights of fe_kuhn.h with the
// host stencil tables of fe_stencils.h (entry by entry, every class of fine
// point inside a coarse cube, o in [0, 4)^3) and prints the number of
// mismatches, the number of entries compared and the largest sum of |8 w|.
#include <cmath>
#include <cstdio>
#include <vector>

#include "fe_kuhn.h"
#include "fe_stencils.h"

int main() {
  std::vector<int> start;
  std::vector<fe_stencil::Entry> ents;
  fe_stencil::prolongation(2, start, ents);
  int bad = 0, compared = 0, maxsum = 0;
  for (int q = 0; q + 1 < (int)start.size(); ++q) {
    const int ox = q % 4, oy = (q / 4) % 4, oz = q / 16;
    double ref[27] = {};
    for (int e = start[q]; e < start[q + 1]; ++e)
      ref[ents[e].d[0] + 3 * (ents[e].d[1] + 3 * ents[e].d[2])] += ents[e].w;
    int sum = 0;
    for (int n = 0; n < 27; ++n) {
      const int w8 = fe_kuhn::pro_w8(ox, oy, oz, n % 3, (n / 3) % 3, n / 9);
      sum += w8 < 0 ? -w8 : w8;
      ++compared;
      if (std::fabs(w8 / 8.0 - ref[n]) > 1e-15) ++bad;
    }
    if (sum > maxsum) maxsum = sum;
  }
  // the far faces (o = 4 on an axis) against o = 0 of the next cube: nodes shifted by 2
  for (int oz = 0; oz <= 4; ++oz)
    for (int oy = 0; oy <= 4; ++oy)
      for (int ox = 0; ox <= 4; ++ox) {
        if (ox < 4 && oy < 4 && oz < 4) continue;
        for (int n = 0; n < 27; ++n) {
          const int a = n % 3, b = (n / 3) % 3, d = n / 9;
          const int w = fe_kuhn::pro_w8(ox, oy, oz, a, b, d);
          const bool sx = ox == 4, sy = oy == 4, sz = oz == 4;
          const int a2 = sx ? a - 2 : a, b2 = sy ? b - 2 : b, d2 = sz ? d - 2 : d;
          const int w2 = (a2 < 0 || b2 < 0 || d2 < 0) ? 0 : fe_kuhn::pro_w8(sx ? 0 : ox, sy ? 0 : oy, sz ? 0 : oz, a2, b2, d2);
          ++compared;
          if (w != w2) ++bad;
        }
      }
  std::printf("%d %d %d\n", bad, compared, maxsum);
  return 0;
}
