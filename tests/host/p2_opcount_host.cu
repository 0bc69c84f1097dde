// Host-only driver for tests/test_p3_element_host.py: counts the arithmetic of
// the library's P2 element formula (p2_element in fe_internal.cuh, the formula
// of the native FP64 operator) with a scalar type that tallies additions,
// multiplications and negations, and prints "add mul neg".
#include <cstdio>

#include "fe_internal.cuh"

#ifdef __CUDA_ARCH__
#define TALLY(x)
#else
#define TALLY(x) ++(x)
#endif

struct Cnt {
  double v;
  static long n_add, n_mul, n_neg;
  __host__ __device__ Cnt() : v(0.0) {}
  __host__ __device__ explicit Cnt(double x) : v(x) {}
};
long Cnt::n_add = 0, Cnt::n_mul = 0, Cnt::n_neg = 0;
__host__ __device__ Cnt operator+(Cnt a, Cnt b) { TALLY(Cnt::n_add); return Cnt(a.v + b.v); }
__host__ __device__ Cnt operator-(Cnt a, Cnt b) { TALLY(Cnt::n_add); return Cnt(a.v - b.v); }
__host__ __device__ Cnt operator*(Cnt a, Cnt b) { TALLY(Cnt::n_mul); return Cnt(a.v * b.v); }
__host__ __device__ Cnt operator-(Cnt a) { TALLY(Cnt::n_neg); return Cnt(-a.v); }

int main() {
  Cnt u[10], g[6], y[10];
  for (int i = 0; i < 10; ++i) u[i] = Cnt(i);
  for (int i = 0; i < 6; ++i) g[i] = Cnt(1.0 + i);
  p2_element<Cnt>(u, g, y);
  std::printf("%ld %ld %ld\n", Cnt::n_add, Cnt::n_mul, Cnt::n_neg);
  return 0;
}
