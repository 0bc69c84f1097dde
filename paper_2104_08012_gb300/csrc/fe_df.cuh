// Double-float ("float pair") arithmetic shared by the FP64 operator kernels:
// a value is the unevaluated sum hi + lo of two floats; additions use Knuth's
// TwoSum, products FMA-based TwoProd (Dekker 1971; Hida, Li & Bailey's
// double-double algorithms restated for float pairs), about 48 significant
// bits.  FP64 values enter and leave through integer bit manipulation after a
// power-of-two normalisation, so the FP64 pipe is not used for conversions.
#pragma once

#include <type_traits>
#include <utility>

#include "fe_internal.cuh"
#include "fe_kuhn.h"

namespace fe_df {

struct DF {
  float hi, lo;
  __device__ __forceinline__ DF() : hi(0.0f), lo(0.0f) {}
  __device__ __forceinline__ explicit DF(float v) : hi(v), lo(0.0f) {}
  __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit DF(int v) : hi((float)v), lo(0.0f) {}
};

// |s| >= |e| assumed; s + e = h + l exactly.
__device__ __forceinline__ DF quick_two_sum(float s, float e) {
  const float h = __fadd_rn(s, e);
  return DF(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// a + b = s + e exactly (Knuth).
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return DF(s, e);
}

// The sum is left unnormalised: hi is the rounded sum of the leading terms and
// lo gathers that rounding error with the trailing terms, so |lo| stays within
// a few ulps of hi and a chain of k additions keeps about 47 - log2(k) bits
// (no quick_two_sum after every addition: 3 of 11 instructions saved).
__device__ __forceinline__ DF operator+(DF x, DF y) {
  const DF t = two_sum(x.hi, y.hi);
  return DF(t.hi, __fadd_rn(t.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF operator-(DF x) { return DF(-x.hi, -x.lo); }
__device__ __forceinline__ DF operator-(DF x, DF y) { return x + (-y); }

// Exact scaling by a power of two.
__device__ __forceinline__ DF scale2(DF x, float k) { return DF(__fmul_rn(x.hi, k), __fmul_rn(x.lo, k)); }
// x * k for a small integer k (TwoProd of the leading term).
__device__ __forceinline__ DF scalek(DF x, float k) {
  const float p = __fmul_rn(x.hi, k);
  const float e = __fmaf_rn(x.lo, k, __fmaf_rn(x.hi, k, -p));
  return quick_two_sum(p, e);
}

// a0 b0 + a1 b1 + a2 b2: the three leading products are summed exactly
// (TwoSum), every error term (product errors, cross terms, summation errors)
// is gathered in one float.
__device__ __forceinline__ DF dot3(DF a0, DF b0, DF a1, DF b1, DF a2, DF b2) {
  const float p0 = __fmul_rn(a0.hi, b0.hi), p1 = __fmul_rn(a1.hi, b1.hi), p2 = __fmul_rn(a2.hi, b2.hi);
  float e0 = __fmaf_rn(a0.hi, b0.hi, -p0), e1 = __fmaf_rn(a1.hi, b1.hi, -p1), e2 = __fmaf_rn(a2.hi, b2.hi, -p2);
  e0 = __fmaf_rn(a0.lo, b0.hi, __fmaf_rn(a0.hi, b0.lo, e0));
  e1 = __fmaf_rn(a1.lo, b1.hi, __fmaf_rn(a1.hi, b1.lo, e1));
  e2 = __fmaf_rn(a2.lo, b2.hi, __fmaf_rn(a2.hi, b2.lo, e2));
  const DF s1 = two_sum(p0, p1);
  const DF s2 = two_sum(s1.hi, p2);
  return DF(s2.hi, __fadd_rn(__fadd_rn(e0, e1), __fadd_rn(__fadd_rn(e2, s1.lo), s2.lo)));  // unnormalised, as +
}

// a * b with the leading product exact (TwoProd), unnormalised like +.
__device__ __forceinline__ DF mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return DF(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.hi, -p))));
}

// h = G t for the symmetric G stored (00, 01, 02, 11, 12, 22).
__device__ __forceinline__ void gmul(const DF (&g)[6], DF t0, DF t1, DF t2, DF& h0, DF& h1, DF& h2) {
  h0 = dot3(g[0], t0, g[1], t1, g[2], t2);
  h1 = dot3(g[1], t0, g[3], t1, g[4], t2);
  h2 = dot3(g[2], t0, g[4], t1, g[5], t2);
}

// The P2 vertex-gradient element of fe_internal.cuh written out without
// loops (u: 4 vertices then edges 01,02,03,12,13,23), so that every float
// pair stays in registers.
__device__ __forceinline__ void p2_element_df(const DF (&u)[10], const DF (&g)[6], DF (&y)[10]) {
  const DF f01 = scale2(u[4], 4.f), f02 = scale2(u[5], 4.f), f03 = scale2(u[6], 4.f);
  const DF f12 = scale2(u[7], 4.f), f13 = scale2(u[8], 4.f), f23 = scale2(u[9], 4.f);
  // c_wv = 4 u_wv - u_v, c_ww = 3 u_w;  d_w = (c_w1 - c_w0, c_w2 - c_w0, c_w3 - c_w0)
  const DF c00 = scalek(u[0], 3.f), c01 = f01 - u[1], c02 = f02 - u[2], c03 = f03 - u[3];
  const DF c10 = f01 - u[0], c11 = scalek(u[1], 3.f), c12 = f12 - u[2], c13 = f13 - u[3];
  const DF c20 = f02 - u[0], c21 = f12 - u[1], c22 = scalek(u[2], 3.f), c23 = f23 - u[3];
  const DF c30 = f03 - u[0], c31 = f13 - u[1], c32 = f23 - u[2], c33 = scalek(u[3], 3.f);
  const DF d00 = c01 - c00, d01 = c02 - c00, d02 = c03 - c00;
  const DF d10 = c11 - c10, d11 = c12 - c10, d12 = c13 - c10;
  const DF d20 = c21 - c20, d21 = c22 - c20, d22 = c23 - c20;
  const DF d30 = c31 - c30, d31 = c32 - c30, d32 = c33 - c30;
  const DF S0 = (d00 + d10) + (d20 + d30), S1 = (d01 + d11) + (d21 + d31), S2 = (d02 + d12) + (d22 + d32);
  DF b01, b02, b03, b11, b12, b13, b21, b22, b23, b31, b32, b33;  // cb_wv = h_w[v-1]
  gmul(g, S0 + d00, S1 + d01, S2 + d02, b01, b02, b03);
  gmul(g, S0 + d10, S1 + d11, S2 + d12, b11, b12, b13);
  gmul(g, S0 + d20, S1 + d21, S2 + d22, b21, b22, b23);
  gmul(g, S0 + d30, S1 + d31, S2 + d32, b31, b32, b33);
  const DF b00 = -(b01 + b02 + b03), b10 = -(b11 + b12 + b13), b20 = -(b21 + b22 + b23), b30 = -(b31 + b32 + b33);
  // y_v = 3 cb_vv - sum_{w != v} cb_wv;  y_(ab) = 4 (cb_ab + cb_ba)
  y[0] = scalek(b00, 3.f) - ((b10 + b20) + b30);
  y[1] = scalek(b11, 3.f) - ((b01 + b21) + b31);
  y[2] = scalek(b22, 3.f) - ((b02 + b12) + b32);
  y[3] = scalek(b33, 3.f) - ((b03 + b13) + b23);
  y[4] = scale2(b01 + b10, 4.f);
  y[5] = scale2(b02 + b20, 4.f);
  y[6] = scale2(b03 + b30, 4.f);
  y[7] = scale2(b12 + b21, 4.f);
  y[8] = scale2(b13 + b31, 4.f);
  y[9] = scale2(b23 + b32, 4.f);
}

// h = M t for the geometric matrix shared by every Kuhn tet, M = U^-1 U^-T =
// [[2,-1,0],[-1,2,-1],[0,-1,1]] (U the upper-triangular matrix of ones):
// v = U^-T t = (t0, t1 - t0, t2 - t1), then h = U^-1 v = (v0 - v1, v1 - v2, v2).
__device__ __forceinline__ void mmul(DF t0, DF t1, DF t2, DF& h0, DF& h1, DF& h2) {
  const DF v1 = t1 - t0, v2 = t2 - t1;
  h0 = t0 - v1;
  h1 = v1 - v2;
  h2 = v2;
}

// p2_element_df with G = c M (c = kappa h / 120 of the cell): the same vertex-
// gradient formula with the three-term G products replaced by mmul, the ten
// results multiplied by c at the end (the element map is linear).
__device__ __forceinline__ void p2_element_df_m(const DF (&u)[10], DF c, DF (&y)[10]) {
  const DF f01 = scale2(u[4], 4.f), f02 = scale2(u[5], 4.f), f03 = scale2(u[6], 4.f);
  const DF f12 = scale2(u[7], 4.f), f13 = scale2(u[8], 4.f), f23 = scale2(u[9], 4.f);
  const DF c00 = scalek(u[0], 3.f), c01 = f01 - u[1], c02 = f02 - u[2], c03 = f03 - u[3];
  const DF c10 = f01 - u[0], c11 = scalek(u[1], 3.f), c12 = f12 - u[2], c13 = f13 - u[3];
  const DF c20 = f02 - u[0], c21 = f12 - u[1], c22 = scalek(u[2], 3.f), c23 = f23 - u[3];
  const DF c30 = f03 - u[0], c31 = f13 - u[1], c32 = f23 - u[2], c33 = scalek(u[3], 3.f);
  const DF d00 = c01 - c00, d01 = c02 - c00, d02 = c03 - c00;
  const DF d10 = c11 - c10, d11 = c12 - c10, d12 = c13 - c10;
  const DF d20 = c21 - c20, d21 = c22 - c20, d22 = c23 - c20;
  const DF d30 = c31 - c30, d31 = c32 - c30, d32 = c33 - c30;
  const DF S0 = (d00 + d10) + (d20 + d30), S1 = (d01 + d11) + (d21 + d31), S2 = (d02 + d12) + (d22 + d32);
  DF b01, b02, b03, b11, b12, b13, b21, b22, b23, b31, b32, b33;
  mmul(S0 + d00, S1 + d01, S2 + d02, b01, b02, b03);
  mmul(S0 + d10, S1 + d11, S2 + d12, b11, b12, b13);
  mmul(S0 + d20, S1 + d21, S2 + d22, b21, b22, b23);
  mmul(S0 + d30, S1 + d31, S2 + d32, b31, b32, b33);
  const DF b00 = -(b01 + b02 + b03), b10 = -(b11 + b12 + b13), b20 = -(b21 + b22 + b23), b30 = -(b31 + b32 + b33);
  y[0] = mul(c, scalek(b00, 3.f) - ((b10 + b20) + b30));
  y[1] = mul(c, scalek(b11, 3.f) - ((b01 + b21) + b31));
  y[2] = mul(c, scalek(b22, 3.f) - ((b02 + b12) + b32));
  y[3] = mul(c, scalek(b33, 3.f) - ((b03 + b13) + b23));
  const DF c4 = scale2(c, 4.f);
  y[4] = mul(c4, b01 + b10);
  y[5] = mul(c4, b02 + b20);
  y[6] = mul(c4, b03 + b30);
  y[7] = mul(c4, b12 + b21);
  y[8] = mul(c4, b13 + b31);
  y[9] = mul(c4, b23 + b32);
}

__device__ __forceinline__ void p1_element_df_m(const DF (&u)[4], DF c, DF (&y)[4]) {
  DF h0, h1, h2;
  mmul(u[1] - u[0], u[2] - u[0], u[3] - u[0], h0, h1, h2);
  y[1] = mul(c, h0);
  y[2] = mul(c, h1);
  y[3] = mul(c, h2);
  y[0] = -((y[1] + y[2]) + y[3]);
}

__device__ __forceinline__ void p1_element_df(const DF (&u)[4], const DF (&g)[6], DF (&y)[4]) {
  DF h0, h1, h2;
  gmul(g, u[1] - u[0], u[2] - u[0], u[3] - u[0], h0, h1, h2);
  y[1] = h0;
  y[2] = h1;
  y[3] = h2;
  y[0] = -(h0 + h1 + h2);
}

// Consistent mass of a tet, y = s K u with s = |det J| / 2520 and the integer
// P2 matrix K of 2520 int_ref phi_i phi_j (vertices 6 on the diagonal, 1 off it;
// vertex-edge -4 if the edge holds the vertex, else -6; edge-edge 32 on the
// diagonal, 8 for the opposite edge, 16 otherwise), applied through sums:
// (K u)_v = 5 u_v + U - 6 E + 2 E_v,  (K u)_ab = 16 E + 16 u_ab - 8 u_opp - 6 U + 2 (u_a + u_b)
// with U the vertex sum, E the edge sum and E_v the sum over the edges at v.
__device__ __forceinline__ void p2_mass_df(const DF (&u)[10], DF s, DF (&y)[10]) {
  const DF U = (u[0] + u[1]) + (u[2] + u[3]);
  const DF E0 = (u[4] + u[5]) + u[6], E1 = (u[4] + u[7]) + u[8], E2 = (u[5] + u[7]) + u[9], E3 = (u[6] + u[8]) + u[9];
  const DF E = (E0 + u[7]) + (u[8] + u[9]);
  const DF W = U - (scale2(E, 4.f) + scale2(E, 2.f));                // U - 6E
  const DF Z = scale2(E, 16.f) - (scale2(U, 4.f) + scale2(U, 2.f));  // 16E - 6U
  y[0] = mul(s, ((scale2(u[0], 4.f) + u[0]) + W) + scale2(E0, 2.f));
  y[1] = mul(s, ((scale2(u[1], 4.f) + u[1]) + W) + scale2(E1, 2.f));
  y[2] = mul(s, ((scale2(u[2], 4.f) + u[2]) + W) + scale2(E2, 2.f));
  y[3] = mul(s, ((scale2(u[3], 4.f) + u[3]) + W) + scale2(E3, 2.f));
  // edges 01, 02, 03, 12, 13, 23; opposite pairs (01, 23), (02, 13), (03, 12)
  y[4] = mul(s, (Z + (scale2(u[4], 16.f) - scale2(u[9], 8.f))) + scale2(u[0] + u[1], 2.f));
  y[5] = mul(s, (Z + (scale2(u[5], 16.f) - scale2(u[8], 8.f))) + scale2(u[0] + u[2], 2.f));
  y[6] = mul(s, (Z + (scale2(u[6], 16.f) - scale2(u[7], 8.f))) + scale2(u[0] + u[3], 2.f));
  y[7] = mul(s, (Z + (scale2(u[7], 16.f) - scale2(u[6], 8.f))) + scale2(u[1] + u[2], 2.f));
  y[8] = mul(s, (Z + (scale2(u[8], 16.f) - scale2(u[5], 8.f))) + scale2(u[1] + u[3], 2.f));
  y[9] = mul(s, (Z + (scale2(u[9], 16.f) - scale2(u[4], 8.f))) + scale2(u[2] + u[3], 2.f));
}

// P1: 120 int_ref phi_i phi_j = 1 + delta_ij, so y_i = s (u_i + U) with s = |det J| / 120.
__device__ __forceinline__ void p1_mass_df(const DF (&u)[4], DF s, DF (&y)[4]) {
  const DF U = (u[0] + u[1]) + (u[2] + u[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) y[i] = mul(s, u[i] + U);
}

template <int DEG>
__device__ __forceinline__ void element_df(const DF (&u)[DEG == 1 ? 4 : 10], const DF (&g)[6],
                                           DF (&y)[DEG == 1 ? 4 : 10]) {
  if constexpr (DEG == 1)
    p1_element_df(u, g, y);
  else
    p2_element_df(u, g, y);
}

template <int DEG>
__device__ __forceinline__ void element_df_m(const DF (&u)[DEG == 1 ? 4 : 10], DF c, DF (&y)[DEG == 1 ? 4 : 10]) {
  if constexpr (DEG == 1)
    p1_element_df_m(u, c, y);
  else
    p2_element_df_m(u, c, y);
}

// ------------------------------------ P2 Kuhn tet by fixed-point limbs ---
// The integer element matrix K of a P2 Kuhn tet (fe_kuhn.h) applied to exact
// FP32 limbs of the float-pair products c x.
static_assert(fe_kuhn::kuhn_p2_k_ok(), "P2 Kuhn stiffness: integer, symmetric, zero row sums, row abs sums <= 62");
using fe_kuhn::kuhn_p2_k;

// Fixed-point limb evaluation of y = K x' for x'_j = cs u_j (float pairs,
// |x'_j| < 2): p2_kuhn_split forms the limbs, p2_kuhn_apply the products.  Each x'_j, held as the unnormalised product (p, e), is cut
// into three limbs by rounding against a magic constant (Dekker's splitting
// with a fixed exponent instead of a relative one):
//   A_j: a multiple of 2^-16, |A_j| <= 2;
//   B_j: a multiple of 2^-33, |B_j| < 2^-16.9;
//   C_j = x'_j - A_j - B_j, |C_j| < 2^-33.9.
// Sums of K_ij A_j are integers below 62 * 2^17 < 2^23 times 2^-16, and of
// K_ij B_j integers below 2^22.1 times 2^-33, so FP32 forms K A and K B
// exactly in any order; only K C (below 2^-28) is rounded (about 2^-49
// absolute).  The same holds for the stiffness of two tets that share a face
// (rows of |K| summing to at most 124: below 2^24 and 2^23.1 units).  Row i is handed to emit(i, y_i) as the float pair
// (fl(KA + KB), err + KC) as soon as it is formed, so no output array stays
// live.  The splitting costs 8 FP32 additions per dof and each limb product
// 82 FMAs with immediate integer coefficients, against about 80 float-pair
// additions of 8 instructions each for the same contraction through vertex
// gradients.
// One term K_ij (A_j, B_j, C_j) of row i, with K_ij a template argument so
// that zero terms vanish and the coefficient is an immediate operand.
template <int K>
__device__ __forceinline__ void kuhn_term(float a, float b, float c, float& ya, float& yb, float& yc) {
  if constexpr (K != 0) {
    ya = __fmaf_rn((float)K, a, ya);
    yb = __fmaf_rn((float)K, b, yb);
    yc = __fmaf_rn((float)K, c, yc);
  }
}
// The integer matrices applied by the limbs: one P2 Kuhn tet (10 dofs) and a
// pair of Kuhn tets with the same first axis (14 dofs, fe_kuhn.h).
// cells: consecutive cells of one unit; cell(n), local(n): the cell (0 or 1)
// and its local dof that unit dof n is read from.
struct KuhnTet {
  static constexpr int nd = 10, cells = 1;
  __host__ __device__ static constexpr int k(int i, int j) { return kuhn_p2_k(i, j); }
  __host__ __device__ static constexpr int cell(int) { return 0; }
  __host__ __device__ static constexpr int local(int n) { return n; }
};
struct KuhnPair {
  static constexpr int nd = 14, cells = 2;
  __host__ __device__ static constexpr int k(int i, int j) { return fe_kuhn::kuhn_pair_k(i, j); }
  __host__ __device__ static constexpr int cell(int n) { return n >= 10 ? 1 : 0; }
  __host__ __device__ static constexpr int local(int n) { return n >= 10 ? fe_kuhn::pair_second_local(n) : n; }
};
static_assert(fe_kuhn::kuhn_pair_k_ok(), "P2 Kuhn pair stiffness: symmetric, zero row sums, row abs sums <= 127");

template <typename Km, int I, int ND, int... J>
__device__ __forceinline__ void kuhn_row(const float (&A)[ND], const float (&B)[ND], const float (&C)[ND], float& ya,
                                         float& yb, float& yc, std::integer_sequence<int, J...>) {
  (kuhn_term<Km::k(I, J)>(A[J], B[J], C[J], ya, yb, yc), ...);
}
template <typename Km, int ND, int... I, typename Emit>
__device__ __forceinline__ void kuhn_rows(const float (&A)[ND], const float (&B)[ND], const float (&C)[ND],
                                          Emit& emit, std::integer_sequence<int, I...>) {
  auto row = [&](auto ic) {
    constexpr int i = decltype(ic)::value;
    float ya = 0.0f, yb = 0.0f, yc = 0.0f;
    kuhn_row<Km, i>(A, B, C, ya, yb, yc, std::make_integer_sequence<int, ND>{});
    const DF t = two_sum(ya, yb);
    emit(i, DF(t.hi, __fadd_rn(t.lo, yc)));
  };
  (row(std::integral_constant<int, I>{}), ...);
}

template <int ND>
__device__ __forceinline__ void p2_kuhn_split(const DF (&u)[ND], DF cs, float (&A)[ND], float (&B)[ND],
                                              float (&C)[ND]) {
  constexpr float kMagA = 192.0f;      // 1.5 * 2^7: fl(v + kMagA) has ulp 2^-16 for |v| <= 2
  constexpr float kMagB = 0x1.8p-10f;  // 1.5 * 2^-10: ulp 2^-33 for |v| < 2^-11
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const float p = __fmul_rn(cs.hi, u[j].hi);
    const float e = __fmaf_rn(cs.hi, u[j].lo, __fmaf_rn(cs.lo, u[j].hi, __fmaf_rn(cs.hi, u[j].hi, -p)));
    A[j] = __fsub_rn(__fadd_rn(p, kMagA), kMagA);
    const float r = __fsub_rn(p, A[j]);  // exact
    B[j] = __fsub_rn(__fadd_rn(__fadd_rn(r, e), kMagB), kMagB);
    C[j] = __fadd_rn(__fsub_rn(r, B[j]), e);  // r - B_j exact
  }
}
template <typename Km = KuhnTet, typename Emit>
__device__ __forceinline__ void p2_kuhn_apply(const float (&A)[Km::nd], const float (&B)[Km::nd],
                                              const float (&C)[Km::nd], Emit&& emit) {
  kuhn_rows<Km>(A, B, C, emit, std::make_integer_sequence<int, Km::nd>{});
}

// Whether cube-local node l already received a contribution from one of the
// tets 0..t-1 (decides at compile time between initialising and adding).
__host__ __device__ constexpr bool touched_before(int deg, int t, int l) {
  bool hit = false;
  for (int s = 0; s < t; ++s)
    for (int j = 0; j < (deg == 1 ? 4 : 10); ++j) hit = hit || cube_local(deg, s, j) == l;
  return hit;
}

// double -> float pair by bit manipulation, after scaling by 2^(1023 - emax)
// (emax: the largest biased exponent of the tet's dofs, so the largest dof
// maps to [1, 2)): hi keeps the leading 24 bits of the significand
// (truncated), lo the next 24 (rounded).  Dofs more than 2^126 below the
// tet's largest flush to 0 (negligible against it).
__device__ __forceinline__ DF split_scaled(double x, int emax) {
  const unsigned int h32 = (unsigned int)__double2hiint(x), l32 = (unsigned int)__double2loint(x);
  const int e = (int)((h32 >> 20) & 0x7FFu) - emax + 1023;  // exponent field of x * 2^(1023 - emax)
  const unsigned int sgn = h32 & 0x80000000u;
  if (((h32 >> 20) & 0x7FFu) == 0u || e <= 896) return DF(__uint_as_float(sgn), 0.0f);
  const unsigned int hb = sgn | ((unsigned int)(e - 896) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
  const float scale = e > 948 ? __uint_as_float((unsigned int)(e - 948) << 23) : 0.0f;  // 2^(e - 1075)
  const float lo = __fmul_rn(__uint2float_rn(l32 & 0x1FFFFFFFu), scale);
  return DF(__uint_as_float(hb), __uint_as_float(__float_as_uint(lo) | sgn));
}

// Largest biased exponent of the dofs (1023 if all are zero); 0x7FF if any is not finite.
template <int ND>
__device__ __forceinline__ int block_exponent(const double (&xv)[ND]) {
  int emax = 0;
#pragma unroll
  for (int j = 0; j < ND; ++j) emax = max(emax, (int)(((unsigned int)__double2hiint(xv[j]) >> 20) & 0x7FFu));
  return emax == 0 ? 1023 : emax;
}

// exact float -> double of f * 2^(emax - 1023) by bit manipulation; results
// below the normal double range become subnormal doubles (gradual underflow:
// the significand shifted right, bits below 2^-1074 truncated), results above
// it give inf
__device__ __forceinline__ double widen_scaled(float f, int emax) {
  const unsigned int b = __float_as_uint(f);
  const int ef = (int)((b >> 23) & 0xFFu);
  const unsigned int sgn = b & 0x80000000u;
  if (ef == 0) return __hiloint2double((int)sgn, 0);
  const int eh = ef + emax - 127;
  if (ef == 0xFF || eh >= 0x7FF) return __hiloint2double((int)(sgn | 0x7FF00000u | ((b & 0x7FFFFFu) >> 3)), 0);
  if (eh <= 0) {
    // value = m 2^(ef + emax - 1173) with the 24-bit significand m; as a
    // subnormal it is k 2^-1074 with k = m 2^sh, sh = ef + emax - 99 = eh + 28
    const unsigned long long m = 0x800000ull | (b & 0x7FFFFFu);
    const int sh = eh + 28;
    const unsigned long long k = sh >= 0 ? (m << sh) : (sh > -24 ? (m >> -sh) : 0ull);
    return __longlong_as_double((long long)(((unsigned long long)sgn << 32) | k));
  }
  return __hiloint2double((int)(sgn | ((unsigned int)eh << 20) | ((b & 0x7FFFFFu) >> 3)), (int)((b & 7u) << 29));
}


// widen_scaled for a tet whose exponent emax lies in [127, 1918]: then every
// normal float f maps to a normal double (biased exponent ef + emax - 127 in
// [1, 2045]) and zero or subnormal f (negligible against the tet's largest
// term) to +-0, so no range branches are needed.  kexp = (emax - 127) << 20.
__device__ __forceinline__ double widen_in_range(float f, unsigned int kexp) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int mag = b & 0x7FFFFFFFu, sgn = b & 0x80000000u;
  const bool normal = mag >= 0x00800000u;
  const unsigned int hi = normal ? (((mag >> 3) + kexp) | sgn) : sgn;
  const unsigned int lo = normal ? (b << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}

// Producer-side split of an FP64 value into the unscaled float pair that the
// operator kernels gather (hi holds the leading 24 significant bits, lo the
// next 24 rounded).  The pair is exact to 48 bits for 2^-64 <= |x| < 2^64; for
// larger, smaller (nonzero), subnormal or non-finite x it is the marker
// (NaN, 0), and a tet that gathers a marker splits its FP64 dofs itself with
// its own power-of-two scaling.
__device__ __forceinline__ float2 split_pair(double x) {
  const unsigned int h32 = (unsigned int)__double2hiint(x), l32 = (unsigned int)__double2loint(x);
  const unsigned int e = (h32 >> 20) & 0x7FFu;
  if (e - 959u < 128u) {  // biased exponent 959..1086: 2^-64 <= |x| < 2^64
    const DF p = split_scaled(x, 1023);
    return make_float2(p.hi, p.lo);
  }
  if (((h32 & 0x7FFFFFFFu) | l32) == 0u) return make_float2(__uint_as_float(h32 & 0x80000000u), 0.0f);
  return make_float2(__int_as_float(0x7fc00000), 0.0f);
}

}  // namespace fe_df
