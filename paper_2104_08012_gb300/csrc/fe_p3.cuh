// P3 element action through the gradient at the P2 nodes (degree 3 is the
// paper's Poisson discretisation, Section 2; the bilinear form is Eq. 4).
//
// For u in P3 the reference gradient is quadratic, so it equals its P2
// interpolant: grad u = sum_n psi_n d_n over the 10 P2 nodes n (vertices, edge
// midpoints) with d_n = grad u(x_n).  In barycentric form d_n = (c_n1 - c_n0,
// c_n2 - c_n0, c_n3 - c_n0) with c_nv = du/dlambda_v at x_n, and
//   a(u, w) = sum_{n,m} Mq_nm d_n(w)^T G d_m(u),   Mq = int_ref psi_n psi_m,
// so y = D^T (Mq (x) G) D u.  The barycentric derivatives of the P3 basis at the
// P2 nodes are k/8 with small integers k (148 nonzeros of 800), and Mq = K/2520
// with the integer P2 mass matrix K (vertex diagonal 6, vertex-vertex 1,
// vertex-edge -4 or -6, edge-edge 32, 16 or 8 for the opposite edge).  With
// c, d and the transposed map scaled by 8, the geometric factors carry
// kappa G / (64 * 2520) = kappa G / 161280 and every other coefficient is a
// small integer: about 590 operations per tet against 1680 FMAs for the
// element matrix.  Zero coefficients are removed at compile time.
//
// Ops supplies the arithmetic: plain float/double, or float pairs (fe_df.cuh).
#pragma once

#include <utility>

#include "fe_df.cuh"

namespace fe_p3 {

// P2 edge (a, b) of index e in the order (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).
__host__ __device__ constexpr int ea(int e) { return e < 3 ? 0 : (e < 5 ? 1 : 2); }
__host__ __device__ constexpr int eb(int e) { return e == 0 ? 1 : (e == 1 || e == 3) ? 2 : 3; }

// 2 * lambda_v at P2 node n (0, 1 or 2).
__host__ __device__ constexpr int node_l(int n, int v) {
  return n < 4 ? (n == v ? 2 : 0) : ((v == ea(n - 4) || v == eb(n - 4)) ? 1 : 0);
}

// 8 * d phi_i / d lambda_v at P2 node n, P3 local dof i (vertices; per edge the
// node nearer its first vertex, then the other; faces opposite vertex 0..3):
// vertex w: 27 l^2 - 36 l + 8 (v = w); edge node nearer p (other vertex q):
// 18 l_q (3 l_p - 1) (v = p), 9 l_p (3 l_p - 2) (v = q); face (a, b, c):
// 54 l_b l_c (v = a, the other two for b and c).  l = 2 lambda.
__host__ __device__ constexpr int dphi8(int i, int v, int n) {
  if (i < 4) {
    const int l = node_l(n, i);
    return v == i ? 27 * l * l - 36 * l + 8 : 0;
  }
  if (i < 16) {
    const int e = (i - 4) / 2, h = (i - 4) % 2;
    const int p = h ? eb(e) : ea(e), q = h ? ea(e) : eb(e);
    const int lp = node_l(n, p), lq = node_l(n, q);
    if (v == p) return 18 * lq * (3 * lp - 1);
    if (v == q) return 9 * lp * (3 * lp - 2);
    return 0;
  }
  const int f = i - 16;  // face opposite vertex f
  if (v == f) return 0;
  int o[2] = {0, 0}, k = 0;
  for (int w = 0; w < 4; ++w)
    if (w != f && w != v) o[k++] = w;
  return 54 * node_l(n, o[0]) * node_l(n, o[1]);
}

// ------------------------------------------------------------ arithmetic
template <typename T>
struct PlainOps {
  using V = T;
  __host__ __device__ static V zero() { return T(0); }
  __host__ __device__ static V add(V a, V b) { return a + b; }
  __host__ __device__ static V sub(V a, V b) { return a - b; }
  __host__ __device__ static V neg(V a) { return -a; }
  __host__ __device__ static V muli(V a, int k) { return a * T(k); }
  __host__ __device__ static V fmai(V a, int k, V s) { return s + a * T(k); }
  // G t for symmetric G (00, 01, 02, 11, 12, 22)
  __host__ __device__ static void gmul(const V (&g)[6], V t0, V t1, V t2, V& h0, V& h1, V& h2) {
    h0 = g[0] * t0 + g[1] * t1 + g[2] * t2;
    h1 = g[1] * t0 + g[3] * t1 + g[4] * t2;
    h2 = g[2] * t0 + g[4] * t1 + g[5] * t2;
  }
  // M t for M = [[2,-1,0],[-1,2,-1],[0,-1,1]], the geometric matrix of every Kuhn tet (G = c M)
  __host__ __device__ static void mmul(V t0, V t1, V t2, V& h0, V& h1, V& h2) {
    const V v1 = t1 - t0, v2 = t2 - t1;
    h0 = t0 - v1;
    h1 = v1 - v2;
    h2 = v2;
  }
  __host__ __device__ static V mul(V a, V b) { return a * b; }
};

struct DFOps {
  using V = fe_df::DF;
  __device__ static V zero() { return V(0.0f); }
  __device__ static V add(V a, V b) { return a + b; }
  __device__ static V sub(V a, V b) { return a - b; }
  __device__ static V neg(V a) { return -a; }
  // exact products by small integers (TwoProd of the leading term); powers of two scale exactly
  __device__ static V muli(V a, int k) {
    if ((k & (k - 1)) == 0 && k > 0) return fe_df::scale2(a, (float)k);
    return fe_df::scalek(a, (float)k);
  }
  __device__ static V fmai(V a, int k, V s) { return s + muli(a, k); }
  __device__ static void gmul(const V (&g)[6], V t0, V t1, V t2, V& h0, V& h1, V& h2) {
    fe_df::gmul(g, t0, t1, t2, h0, h1, h2);
  }
  __device__ static void mmul(V t0, V t1, V t2, V& h0, V& h1, V& h2) { fe_df::mmul(t0, t1, t2, h0, h1, h2); }
  __device__ static V mul(V a, V b) { return fe_df::mul(a, b); }
};

// ------------------------------------------------------- compile-time folds
template <typename Ops, int n, int v, int i>
__host__ __device__ __forceinline__ void c_term(typename Ops::V& s, bool& any, const typename Ops::V* u) {
  constexpr int k = dphi8(i, v, n);
  if constexpr (k != 0) {
    if constexpr (k == 1)
      s = any ? Ops::add(s, u[i]) : u[i];
    else if constexpr (k == -1)
      s = any ? Ops::sub(s, u[i]) : Ops::neg(u[i]);
    else
      s = any ? Ops::fmai(u[i], k, s) : Ops::muli(u[i], k);
    any = true;
  }
}

// 8 c_nv = sum_i 8 dphi_i/dlambda_v (x_n) u_i
template <typename Ops, int n, int v, int... I>
__host__ __device__ __forceinline__ typename Ops::V c_val(const typename Ops::V* u, std::integer_sequence<int, I...>) {
  typename Ops::V s = Ops::zero();
  bool any = false;
  (c_term<Ops, n, v, I>(s, any, u), ...);
  return s;
}

template <typename Ops, int i, int n, int v>
__host__ __device__ __forceinline__ void y_term(typename Ops::V& s, bool& any, const typename Ops::V (&hh)[10][4]) {
  constexpr int k = dphi8(i, v, n);
  if constexpr (k != 0) {
    if constexpr (k == 1)
      s = any ? Ops::add(s, hh[n][v]) : hh[n][v];
    else if constexpr (k == -1)
      s = any ? Ops::sub(s, hh[n][v]) : Ops::neg(hh[n][v]);
    else
      s = any ? Ops::fmai(hh[n][v], k, s) : Ops::muli(hh[n][v], k);
    any = true;
  }
}

// y_i = sum_{n, v} 8 dphi_i/dlambda_v (x_n) hh_nv  (J = 4 n + v)
template <typename Ops, int i, int... J>
__host__ __device__ __forceinline__ typename Ops::V y_val(const typename Ops::V (&hh)[10][4], std::integer_sequence<int, J...>) {
  typename Ops::V s = Ops::zero();
  bool any = false;
  (y_term<Ops, i, J / 4, J % 4>(s, any, hh), ...);
  return s;
}

template <typename Ops, int n>
__host__ __device__ __forceinline__ void grad_at_node(const typename Ops::V* u, typename Ops::V (&d)[10][3]) {
  using Seq = std::make_integer_sequence<int, 20>;
  const typename Ops::V c0 = c_val<Ops, n, 0>(u, Seq{});
  d[n][0] = Ops::sub(c_val<Ops, n, 1>(u, Seq{}), c0);
  d[n][1] = Ops::sub(c_val<Ops, n, 2>(u, Seq{}), c0);
  d[n][2] = Ops::sub(c_val<Ops, n, 3>(u, Seq{}), c0);
}

template <typename Ops, int... N>
__host__ __device__ __forceinline__ void grads(const typename Ops::V* u, typename Ops::V (&d)[10][3],
                                      std::integer_sequence<int, N...>) {
  (grad_at_node<Ops, N>(u, d), ...);
}

template <typename Ops, int... I>
__host__ __device__ __forceinline__ void outputs(const typename Ops::V (&hh)[10][4], typename Ops::V* y,
                                        std::integer_sequence<int, I...>) {
  ((y[I] = y_val<Ops, I>(hh, std::make_integer_sequence<int, 40>{})), ...);
}

// w = K x for the integer P2 mass matrix K through vertex and edge sums:
// (K x)_v = 5 x_v + U - 6 E + 2 E_v, (K x)_ab = 16 E + 16 x_ab - 8 x_opp - 6 U + 2 (x_a + x_b)
// with U the vertex sum, E the edge sum, E_v the sum over the edges at v.
template <typename Ops>
__host__ __device__ __forceinline__ void p2_mass_int(const typename Ops::V (&x)[10], typename Ops::V (&w)[10]) {
  using V = typename Ops::V;
  const V U = Ops::add(Ops::add(x[0], x[1]), Ops::add(x[2], x[3]));
  const V E0 = Ops::add(Ops::add(x[4], x[5]), x[6]), E1 = Ops::add(Ops::add(x[4], x[7]), x[8]);
  const V E2 = Ops::add(Ops::add(x[5], x[7]), x[9]), E3 = Ops::add(Ops::add(x[6], x[8]), x[9]);
  const V E = Ops::add(Ops::add(E0, x[7]), Ops::add(x[8], x[9]));
  const V W = Ops::sub(U, Ops::muli(E, 6));                 // U - 6E
  const V Z = Ops::sub(Ops::muli(E, 16), Ops::muli(U, 6));  // 16E - 6U
  const V Ev[4] = {E0, E1, E2, E3};
#pragma unroll
  for (int v = 0; v < 4; ++v) w[v] = Ops::add(Ops::add(Ops::muli(x[v], 5), W), Ops::muli(Ev[v], 2));
  // edges 01, 02, 03, 12, 13, 23; opposite pairs (01, 23), (02, 13), (03, 12)
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int opp = 5 - e;
    w[4 + e] = Ops::add(Ops::add(Z, Ops::sub(Ops::muli(x[4 + e], 16), Ops::muli(x[4 + opp], 8))),
                        Ops::muli(Ops::add(x[ea(e)], x[eb(e)]), 2));
  }
}

// y = A_K u for one P3 tet; g = kappa G / 161280 (symmetric, 00 01 02 11 12 22),
// or with UNI g[0] = c for G = c M (the Kuhn tets' shared matrix, see mmul).
template <typename Ops, bool UNI = false>
__host__ __device__ __forceinline__ void p3_element_grad(const typename Ops::V* u, const typename Ops::V (&g)[6],
                                                typename Ops::V* y) {
  using V = typename Ops::V;
  V d[10][3];
  grads<Ops>(u, d, std::make_integer_sequence<int, 10>{});
  V hh[10][4];
  {
    V x[10], w[3][10];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int n = 0; n < 10; ++n) x[n] = d[n][a];
      p2_mass_int<Ops>(x, w[a]);
    }
#pragma unroll
    for (int n = 0; n < 10; ++n) {
      V h0, h1, h2;
      if constexpr (UNI)
        Ops::mmul(w[0][n], w[1][n], w[2][n], h0, h1, h2);
      else
        Ops::gmul(g, w[0][n], w[1][n], w[2][n], h0, h1, h2);
      hh[n][0] = Ops::neg(Ops::add(Ops::add(h0, h1), h2));
      hh[n][1] = h0;
      hh[n][2] = h1;
      hh[n][3] = h2;
    }
  }
  outputs<Ops>(hh, y, std::make_integer_sequence<int, 20>{});
  if constexpr (UNI) {
#pragma unroll
    for (int i = 0; i < 20; ++i) y[i] = Ops::mul(g[0], y[i]);
  }
}

}  // namespace fe_p3
