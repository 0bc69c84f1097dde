// Float-pair arithmetic on two tets at once with Blackwell's packed FP32
// instructions (add/sub/mul/fma .rn.f32x2: one instruction, two independent
// IEEE single-precision operations).  Every value of fe_df.cuh becomes a pair
// of values, tet A in the low and tet B in the high half of a 64-bit register,
// and every scalar operation of the P2 element formula becomes one packed
// instruction applying the same rounding in both halves; the element results
// are the scalar formula's, tet by tet.  The double-float apply is bound by
// instruction issue, and the formula's 976 FP32 operations per tet then take
// 488 issue slots.
//
// PTX has no packed negation, so the formula is arranged to need none: the
// products of the 3-term dot products are formed with the negated geometric
// factors (exactly -p), each dot product is returned negated, and the
// downstream sums are reordered so that their (exact) negations cancel; the
// three edge outputs that stay negated are flipped when they are widened.
#pragma once

#include "fe_df.cuh"

namespace fe_df {

struct F2 {
  unsigned long long v;
};

__device__ __forceinline__ F2 f2_pack(float a, float b) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(F2 x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ F2 f2_const(float k) { return f2_pack(k, k); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
  F2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
  F2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
  F2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  F2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}

// A float pair (hi + lo) for each of the two tets.
struct DF2 {
  F2 hi, lo;
};

// Knuth's TwoSum in both halves: a + b = s + e exactly.
__device__ __forceinline__ DF2 two_sum2(F2 a, F2 b) {
  const F2 s = add2(a, b);
  const F2 v = sub2(s, a);
  return DF2{s, add2(sub2(a, sub2(s, v)), sub2(b, v))};
}

// x + y, unnormalised like fe_df's operator+.
__device__ __forceinline__ DF2 operator+(DF2 x, DF2 y) {
  const DF2 t = two_sum2(x.hi, y.hi);
  return DF2{t.hi, add2(t.lo, add2(x.lo, y.lo))};
}

// x - y: fe_df computes x + (-y); TwoSum of (a, -b) is written with
// subtractions (RN(-b - v) = -RN(b + v)), which gives the same bits.
__device__ __forceinline__ DF2 operator-(DF2 x, DF2 y) {
  const F2 s = sub2(x.hi, y.hi);
  const F2 v = sub2(s, x.hi);
  const F2 e = sub2(sub2(x.hi, sub2(s, v)), add2(y.hi, v));
  return DF2{s, add2(e, sub2(x.lo, y.lo))};
}

// Exact scaling by a power of two.
__device__ __forceinline__ DF2 scale2(DF2 x, float k) {
  const F2 kk = f2_const(k);
  return DF2{mul2(x.hi, kk), mul2(x.lo, kk)};
}

// fe_df's scalek (TwoProd of the leading term, quick_two_sum) with the rounded
// product formed negated, pn = RN(-k hi) = -p: fma(hi, k, -p) = fma(hi, k, pn),
// RN(p + e) = RN(e - pn), RN(h - p) = RN(h + pn).
__device__ __forceinline__ DF2 scalek(DF2 x, float k) {
  const F2 kk = f2_const(k);
  const F2 pn = mul2(x.hi, f2_const(-k));
  const F2 e = fma2(x.lo, kk, fma2(x.hi, kk, pn));
  const F2 h = sub2(e, pn);
  return DF2{h, sub2(e, add2(h, pn))};
}

// -(a0 b0 + a1 b1 + a2 b2) for the geometric factors a (with their negated
// leading parts an) and b: fe_df's dot3 with every product negated (exact);
// the two TwoSums of the negated products give the negated sums, and the
// error terms' sum is subtracted instead of added.
__device__ __forceinline__ DF2 neg_dot3(DF2 a0, F2 an0, DF2 b0, DF2 a1, F2 an1, DF2 b1, DF2 a2, F2 an2, DF2 b2) {
  const F2 pn0 = mul2(an0, b0.hi), pn1 = mul2(an1, b1.hi), pn2 = mul2(an2, b2.hi);
  F2 e0 = fma2(a0.hi, b0.hi, pn0), e1 = fma2(a1.hi, b1.hi, pn1), e2 = fma2(a2.hi, b2.hi, pn2);
  e0 = fma2(a0.lo, b0.hi, fma2(a0.hi, b0.lo, e0));
  e1 = fma2(a1.lo, b1.hi, fma2(a1.hi, b1.lo, e1));
  e2 = fma2(a2.lo, b2.hi, fma2(a2.hi, b2.lo, e2));
  const DF2 s1 = two_sum2(pn0, pn1);   // = -(p0 + p1)
  const DF2 s2 = two_sum2(s1.hi, pn2);  // = -(s1 + p2)
  return DF2{s2.hi, sub2(add2(sub2(s1.lo, e2), s2.lo), add2(e0, e1))};
}

// -G t for the symmetric G stored (00, 01, 02, 11, 12, 22).
__device__ __forceinline__ void neg_gmul(const DF2 (&g)[6], const F2 (&gn)[6], DF2 t0, DF2 t1, DF2 t2, DF2& h0,
                                         DF2& h1, DF2& h2) {
  h0 = neg_dot3(g[0], gn[0], t0, g[1], gn[1], t1, g[2], gn[2], t2);
  h1 = neg_dot3(g[1], gn[1], t0, g[3], gn[3], t1, g[4], gn[4], t2);
  h2 = neg_dot3(g[2], gn[2], t0, g[4], gn[4], t1, g[5], gn[5], t2);
}

// fe_df's p2_element_df for two tets.  With B = -b (the negated products
// G t) the outputs are rewritten without negations: y_v = R_v - 3 B_vv (v >
// 0), y_0 = 3 S_0 - R_0, y_(0w) = 4 (S_w - B_0w) where S_w = B_w1 + B_w2 +
// B_w3, and the edges between two non-zero vertices come out negated:
// ny_(ab) = 4 (B_ab + B_ba) = -y_(ab) for outputs 7, 8, 9.
__device__ __forceinline__ void p2_element_df2(const DF2 (&u)[10], const DF2 (&g)[6], const F2 (&gn)[6],
                                               DF2 (&y)[10]) {
  const DF2 f01 = scale2(u[4], 4.f), f02 = scale2(u[5], 4.f), f03 = scale2(u[6], 4.f);
  const DF2 f12 = scale2(u[7], 4.f), f13 = scale2(u[8], 4.f), f23 = scale2(u[9], 4.f);
  const DF2 c00 = scalek(u[0], 3.f), c01 = f01 - u[1], c02 = f02 - u[2], c03 = f03 - u[3];
  const DF2 c10 = f01 - u[0], c11 = scalek(u[1], 3.f), c12 = f12 - u[2], c13 = f13 - u[3];
  const DF2 c20 = f02 - u[0], c21 = f12 - u[1], c22 = scalek(u[2], 3.f), c23 = f23 - u[3];
  const DF2 c30 = f03 - u[0], c31 = f13 - u[1], c32 = f23 - u[2], c33 = scalek(u[3], 3.f);
  const DF2 d00 = c01 - c00, d01 = c02 - c00, d02 = c03 - c00;
  const DF2 d10 = c11 - c10, d11 = c12 - c10, d12 = c13 - c10;
  const DF2 d20 = c21 - c20, d21 = c22 - c20, d22 = c23 - c20;
  const DF2 d30 = c31 - c30, d31 = c32 - c30, d32 = c33 - c30;
  const DF2 S0 = (d00 + d10) + (d20 + d30), S1 = (d01 + d11) + (d21 + d31), S2 = (d02 + d12) + (d22 + d32);
  DF2 B01, B02, B03, B11, B12, B13, B21, B22, B23, B31, B32, B33;  // B_wv = -cb_wv
  neg_gmul(g, gn, S0 + d00, S1 + d01, S2 + d02, B01, B02, B03);
  neg_gmul(g, gn, S0 + d10, S1 + d11, S2 + d12, B11, B12, B13);
  neg_gmul(g, gn, S0 + d20, S1 + d21, S2 + d22, B21, B22, B23);
  neg_gmul(g, gn, S0 + d30, S1 + d31, S2 + d32, B31, B32, B33);
  // cb_w0 = -(cb_w1 + cb_w2 + cb_w3) = (B_w1 + B_w2) + B_w3 = SB_w
  const DF2 SB0 = (B01 + B02) + B03, SB1 = (B11 + B12) + B13, SB2 = (B21 + B22) + B23, SB3 = (B31 + B32) + B33;
  y[0] = scalek(SB0, 3.f) - ((SB1 + SB2) + SB3);
  y[1] = ((B01 + B21) + B31) - scalek(B11, 3.f);
  y[2] = ((B02 + B12) + B32) - scalek(B22, 3.f);
  y[3] = ((B03 + B13) + B23) - scalek(B33, 3.f);
  y[4] = scale2(SB1 - B01, 4.f);
  y[5] = scale2(SB2 - B02, 4.f);
  y[6] = scale2(SB3 - B03, 4.f);
  y[7] = scale2(B12 + B21, 4.f);  // negated
  y[8] = scale2(B13 + B31, 4.f);  // negated
  y[9] = scale2(B23 + B32, 4.f);  // negated
}

}  // namespace fe_df
