// Prints the library's integer P2 Kuhn-tet stiffness K120 (fe_kuhn.h) row by
// row, or with the argument "pair" the stiffness of two Kuhn tets that share
// a face (kuhn_pair_k, 14 x 14, times 4 so that it is in the units of K120),
// for tests/test_kuhn_host.py to compare with the oracle's element matrices.
#include <cstdio>
#include <cstring>

#include "fe_kuhn.h"

static_assert(fe_kuhn::kuhn_p2_k_ok(), "K120 properties");
static_assert(fe_kuhn::kuhn_pair_k_ok(), "pair stiffness properties");

int main(int argc, char** argv) {
  if (argc > 1 && std::strcmp(argv[1], "pair") == 0) {
    for (int m = 0; m < 14; ++m)
      for (int n = 0; n < 14; ++n) std::printf("%d%c", 4 * fe_kuhn::kuhn_pair_k(m, n), n == 13 ? '\n' : ' ');
    return 0;
  }
  for (int i = 0; i < 10; ++i) {
    for (int j = 0; j < 10; ++j) std::printf("%d%c", fe_kuhn::kuhn_p2_k120(i, j), j == 9 ? '\n' : ' ');
  }
  return 0;
}
