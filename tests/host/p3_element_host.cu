// Host-only driver for tests/test_p3_element_host.py: reads "g0..g5 u0..u19" per
// line from stdin, writes the 20 values of the library's P3 element action
// (fe_p3.cuh, plain double arithmetic) with g taken as kappa G (the factor
// 1/161280 the library folds into its geometric factors is applied here).
#include <cstdio>

#include "fe_p3.cuh"

int main() {
  double g[6], u[20], y[20];
  while (true) {
    for (int k = 0; k < 6; ++k)
      if (std::scanf("%lf", &g[k]) != 1) return 0;
    for (int i = 0; i < 20; ++i)
      if (std::scanf("%lf", &u[i]) != 1) return 1;
    double gs[6];
    for (int k = 0; k < 6; ++k) gs[k] = g[k] / 161280.0;
    fe_p3::p3_element_grad<fe_p3::PlainOps<double>>(u, gs, y);
    for (int i = 0; i < 20; ++i) std::printf("%.17g%c", y[i], i == 19 ? '\n' : ' ');
  }
}
