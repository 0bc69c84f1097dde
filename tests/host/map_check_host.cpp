// Host-only driver for tests/test_map_check_host.py: reads "nd C Cs n nb",
// then nb boundary dofs (sorted), then nd * Cs map entries ([nd][Cs]) from
// stdin and prints fe_check::bad_map_entries of that map.
#include <cstdio>
#include <vector>

#include "fe_checks.h"

int main() {
  int nd = 0;
  long long C = 0, Cs = 0, n = 0, nb = 0;
  if (std::scanf("%d %lld %lld %lld %lld", &nd, &C, &Cs, &n, &nb) != 5) return 2;
  std::vector<int> bnd((size_t)nb), map((size_t)nd * Cs);
  for (auto& b : bnd)
    if (std::scanf("%d", &b) != 1) return 2;
  for (auto& m : map)
    if (std::scanf("%d", &m) != 1) return 2;
  std::printf("%lld\n", fe_check::bad_map_entries(map.data(), nd, C, Cs, n, bnd));
  return 0;
}
