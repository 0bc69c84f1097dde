// Host-only driver for tests/test_p3_element_host.py: counts the arithmetic of
// the library's P3 element formula (fe_p3.cuh) by running it once with an
// arithmetic type that tallies its operations (an FMA counts 1, each of the
// three rows of the 3 x 3 product G t is one multiply and two FMAs) and prints
// "add mul fma neg".
#include <cstdio>

#include "fe_p3.cuh"

#ifdef __CUDA_ARCH__
#define TALLY(x)
#else
#define TALLY(x) ++(x)
#endif

struct CountOps {
  using V = double;
  static long n_add, n_mul, n_fma, n_neg;
  __host__ __device__ static V zero() { return 0.0; }
  __host__ __device__ static V add(V a, V b) { TALLY(n_add); return a + b; }
  __host__ __device__ static V sub(V a, V b) { TALLY(n_add); return a - b; }
  __host__ __device__ static V neg(V a) { TALLY(n_neg); return -a; }
  __host__ __device__ static V muli(V a, int k) { TALLY(n_mul); return a * k; }
  __host__ __device__ static V fmai(V a, int k, V s) { TALLY(n_fma); return s + a * k; }
  __host__ __device__ static void gmul(const V (&g)[6], V t0, V t1, V t2, V& h0, V& h1, V& h2) {
#ifndef __CUDA_ARCH__
    n_mul += 3;
    n_fma += 6;
#endif
    h0 = g[0] * t0 + g[1] * t1 + g[2] * t2;
    h1 = g[1] * t0 + g[3] * t1 + g[4] * t2;
    h2 = g[2] * t0 + g[4] * t1 + g[5] * t2;
  }
};
long CountOps::n_add = 0, CountOps::n_mul = 0, CountOps::n_fma = 0, CountOps::n_neg = 0;

int main() {
  double u[20], y[20];
  const double g[6] = {1.0, 0.1, 0.2, 1.0, 0.3, 1.0};
  for (int i = 0; i < 20; ++i) u[i] = i;
  fe_p3::p3_element_grad<CountOps>(u, g, y);
  std::printf("%ld %ld %ld %ld\n", CountOps::n_add, CountOps::n_mul, CountOps::n_fma, CountOps::n_neg);
  return 0;
}
