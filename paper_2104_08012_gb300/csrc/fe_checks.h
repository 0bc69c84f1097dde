// Consistency check of a cell->dof map (host code, no CUDA types): the maps
// every cell kernel gathers and scatters through, laid out [nd][Cs] as int32
// with dof j >= 0 for a free dof and -1 - j for a Dirichlet dof.  The library
// runs it on every level's tet and cube maps after building them when the
// environment sets FE_DEBUG_CHECKS=1 (the bounds check that stands in for a
// memory sanitizer: a bad entry would make a kernel read or write outside its
// vectors).
#pragma once

#include <algorithm>
#include <vector>

namespace fe_check {

constexpr int kMaxMapRows = 64;  // (k+1)^3 cube map rows for P3

// Number of bad entries among cells 0..C-1: a decoded dof outside [0, n), an
// encoding that disagrees with the sorted boundary dof list `bnd` (a free dof
// flagged Dirichlet or the reverse), or a dof repeated within one cell.
// Returns -1 if nd is outside 1..kMaxMapRows.
inline long long bad_map_entries(const int* map, int nd, long long C, long long Cs, long long n,
                                 const std::vector<int>& bnd) {
  if (nd < 1 || nd > kMaxMapRows) return -1;
  long long bad = 0;
  for (long long c = 0; c < C; ++c) {
    long long dofs[kMaxMapRows];
    for (int j = 0; j < nd; ++j) {
      const int m = map[(size_t)j * Cs + c];
      const bool dirichlet = m < 0;
      const long long d = dirichlet ? -1LL - m : (long long)m;
      dofs[j] = -1;
      if (d < 0 || d >= n) {
        ++bad;
        continue;
      }
      if (dirichlet != std::binary_search(bnd.begin(), bnd.end(), (int)d)) ++bad;
      for (int i = 0; i < j; ++i)
        if (dofs[i] == d) ++bad;
      dofs[j] = d;
    }
  }
  return bad;
}

}  // namespace fe_check
