// Prints the library's integer P2 Kuhn-tet stiffness K120 (fe_kuhn.h) row by
// row, or with the argument "pair" the stiffness of two Kuhn tets that share
// a face (kuhn_pair_k, 14 x 14, times 4 so that it is in the units of K120),
// for tests/test_kuhn_host.py to compare with the oracle's element matrices.
// With the argument "limbs" it checks the exactness argument of the limb
// sums: for every row of K and of the pair matrix, limb values of the largest
// magnitude with an odd number of units (|A_j| = 2 - 2^-16 in units of 2^-16,
// |B_j| = 2^-17 + 2^-22 + 2^-33 in units of 2^-33, with the signs of the row,
// so that no partial sum is a multiple of a power of two) are summed by
// single-precision FMAs in column order, as the operator kernel does, and
// compared with the exact integer sum; prints the number of inexact rows and
// the largest |sum| in units of the limb.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "fe_kuhn.h"

static_assert(fe_kuhn::kuhn_p2_k_ok(), "K120 properties");
static_assert(fe_kuhn::kuhn_pair_k_ok(), "pair stiffness properties");

template <typename K>
static void limb_rows(int nd, K k, int& inexact, double& max_a, double& max_b) {
  const long long a_units = (1LL << 17) - 1;                // A_j: multiple of 2^-16, |A_j| <= 2
  const long long b_units = (1LL << 16) + (1LL << 11) + 1;  // B_j: multiple of 2^-33, |B_j| < 2^-17 + 2^-22
  const float a_mag = std::ldexp((float)a_units, -16), b_mag = std::ldexp((float)b_units, -33);
  for (int m = 0; m < nd; ++m)
    for (int sign = -1; sign <= 1; sign += 2) {
      volatile float ya = 0.0f, yb = 0.0f;  // volatile: one rounding per FMA, as on the device
      long long ea = 0, eb = 0;             // exact sums in units of 2^-16 and 2^-33
      for (int j = 0; j < nd; ++j) {
        const int c = k(m, j);
        if (c == 0) continue;
        const int s = (c > 0 ? 1 : -1) * sign;
        ya = std::fma((float)c, s * a_mag, (float)ya);
        yb = std::fma((float)c, s * b_mag, (float)yb);
        ea += (long long)c * s * a_units;
        eb += (long long)c * s * b_units;
      }
      if ((double)ya != std::ldexp((double)ea, -16) || (double)yb != std::ldexp((double)eb, -33)) ++inexact;
      max_a = std::fmax(max_a, std::fabs((double)ea));
      max_b = std::fmax(max_b, std::fabs((double)eb));
    }
}

int main(int argc, char** argv) {
  if (argc > 1 && std::strcmp(argv[1], "pair") == 0) {
    for (int m = 0; m < 14; ++m)
      for (int n = 0; n < 14; ++n) std::printf("%d%c", 4 * fe_kuhn::kuhn_pair_k(m, n), n == 13 ? '\n' : ' ');
    return 0;
  }
  if (argc > 1 && std::strcmp(argv[1], "limbs") == 0) {
    int inexact = 0;
    double max_a = 0.0, max_b = 0.0;
    limb_rows(10, [](int i, int j) { return fe_kuhn::kuhn_p2_k(i, j); }, inexact, max_a, max_b);
    limb_rows(14, [](int i, int j) { return fe_kuhn::kuhn_pair_k(i, j); }, inexact, max_a, max_b);
    std::printf("%d %.0f %.0f\n", inexact, max_a, max_b);
    return 0;
  }
  for (int i = 0; i < 10; ++i) {
    for (int j = 0; j < 10; ++j) std::printf("%d%c", fe_kuhn::kuhn_p2_k120(i, j), j == 9 ? '\n' : ' ');
  }
  return 0;
}
