// Prints the library's integer P2 Kuhn-tet stiffness K120 (fe_kuhn.h) row by
// row, for tests/test_kuhn_host.py to compare with the oracle's element matrices.
#include <cstdio>

#include "fe_kuhn.h"

static_assert(fe_kuhn::kuhn_p2_k_ok(), "K120 properties");

int main() {
  for (int i = 0; i < 10; ++i) {
    for (int j = 0; j < 10; ++j) std::printf("%d%c", fe_kuhn::kuhn_p2_k120(i, j), j == 9 ? '\n' : ' ');
  }
  return 0;
}
