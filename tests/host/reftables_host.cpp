// Host-only driver for tests/test_reftables_host.py: prints the library's
// reference-element tables (fe_reftables.h), one line per table:
// "<name> <values...>" in row-major order.
#include <cstdio>

#include "fe_reftables.h"

static void put(const char* name, const double* v, int n) {
  std::printf("%s", name);
  for (int i = 0; i < n; ++i) std::printf(" %.17g", v[i]);
  std::printf("\n");
}

int main() {
  double m1[16], m2[100];
  fe_ref::mass_tables(m1, m2);
  static double K3[210][6], M3[400];
  fe_ref::p3_tables(K3, M3);
  double xi[FE_QUAD_POINTS][3], w[FE_QUAD_POINTS], p1[FE_QUAD_POINTS][4], p2[FE_QUAD_POINTS][10];
  double p3[FE_QUAD_POINTS][20];
  fe_ref::quad_tables(xi, w, p1, p2, p3);
  put("m1", m1, 16);
  put("m2", m2, 100);
  put("K3", &K3[0][0], 210 * 6);
  put("M3", M3, 400);
  put("xi", &xi[0][0], FE_QUAD_POINTS * 3);
  put("w", w, FE_QUAD_POINTS);
  put("phi1", &p1[0][0], FE_QUAD_POINTS * 4);
  put("phi2", &p2[0][0], FE_QUAD_POINTS * 10);
  put("phi3", &p3[0][0], FE_QUAD_POINTS * 20);
  double t[5], gw[5];
  fe_ref::gauss_legendre01(5, t, gw);
  put("gl5_t", t, 5);
  put("gl5_w", gw, 5);
  return 0;
}
