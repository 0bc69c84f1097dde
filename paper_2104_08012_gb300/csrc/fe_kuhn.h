// Integer tables of P2 on Kuhn tets, computed at compile time (host and
// device code, no CUDA types, so that host tests compile it with g++): the
// element stiffness of a Kuhn tet and the prolongation weights between nested
// Kuhn meshes.
//
// Every tet of the Kuhn split of UnitCubeMesh has J = h P U (P a permutation,
// U the upper-triangular matrix of ones), hence G = |det J| J^-1 J^-T = h M
// with M = U^-1 U^-T = [[2,-1,0],[-1,2,-1],[0,-1,1]] for every cell, and the P2
// element matrix of the bilinear form (Section 2, Eq. 4, phi quadratic) is
// kappa h / 120 times one integer matrix
//   K120_ij = 120 int_ref grad phi_i^T M grad phi_j,
// computed here from grad phi_v = (4 lambda_v - 1) g_v, grad phi_ab =
// 4 (lambda_a g_b + lambda_b g_a) with g_a = grad lambda_a (constant:
// g_0 = -(1, 1, 1), g_k = e_k) and the reference moments
// 120 int lambda_a lambda_b = 1 + delta_ab, 120 int lambda_a = 5, 120 vol = 20.
// Local dof order: vertices 0..3, then the edges (0,1), (0,2), (0,3), (1,2),
// (1,3), (2,3) as dofs 4..9.
#pragma once

#ifdef __CUDACC__
#define FE_KUHN_HD __host__ __device__
#else
#define FE_KUHN_HD
#endif

namespace fe_kuhn {

// end points of the edge dof j (4..9)
FE_KUHN_HD constexpr int edge_first(int j) { return j <= 6 ? 0 : (j <= 8 ? 1 : 2); }
FE_KUHN_HD constexpr int edge_second(int j) { return j <= 6 ? j - 3 : (j <= 8 ? j - 5 : 3); }

// m_ab = g_a^T M g_b
FE_KUHN_HD constexpr int kuhn_m(int a, int b) {
  int s = 0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      const int mkl = k == l ? (k == 2 ? 1 : 2) : (k + l == 1 || k + l == 3 ? -1 : 0);
      s += (a == 0 ? -1 : (a - 1 == k ? 1 : 0)) * mkl * (b == 0 ? -1 : (b - 1 == l ? 1 : 0));
    }
  return s;
}

// 120 int lambda_a lambda_b over the reference tet
FE_KUHN_HD constexpr int lam2(int a, int b) { return a == b ? 2 : 1; }

FE_KUHN_HD constexpr int kuhn_p2_k120(int i, int j) {
  return i < 4 && j < 4 ? kuhn_m(i, j) * (16 * lam2(i, j) - 20)
         : i >= 4 && j >= 4
             ? 16 * (lam2(edge_first(i), edge_first(j)) * kuhn_m(edge_second(i), edge_second(j)) +
                     lam2(edge_first(i), edge_second(j)) * kuhn_m(edge_second(i), edge_first(j)) +
                     lam2(edge_second(i), edge_first(j)) * kuhn_m(edge_first(i), edge_second(j)) +
                     lam2(edge_second(i), edge_second(j)) * kuhn_m(edge_first(i), edge_first(j)))
         : i >= 4 ? kuhn_p2_k120(j, i)
                  : 4 * (kuhn_m(i, edge_second(j)) * (4 * lam2(i, edge_first(j)) - 5) +
                         kuhn_m(i, edge_first(j)) * (4 * lam2(i, edge_second(j)) - 5));
}

// K120 = 4 K; the limb sums of the operator kernel rely on every row of |K|
// summing to at most 62.
FE_KUHN_HD constexpr int kuhn_p2_k(int i, int j) { return kuhn_p2_k120(i, j) / 4; }

FE_KUHN_HD constexpr bool kuhn_p2_k_ok() {
  for (int i = 0; i < 10; ++i) {
    int row = 0, absrow = 0;
    for (int j = 0; j < 10; ++j) {
      if (kuhn_p2_k120(i, j) % 4 != 0 || kuhn_p2_k120(i, j) != kuhn_p2_k120(j, i)) return false;
      row += kuhn_p2_k(i, j);
      absrow += kuhn_p2_k(i, j) < 0 ? -kuhn_p2_k(i, j) : kuhn_p2_k(i, j);
    }
    if (row != 0 || absrow > 62) return false;  // constants in the kernel: rows sum to 0
  }
  return true;
}

// Two Kuhn tets of a cube whose permutations share the first axis, (p0, p1,
// p2) and (p0, p2, p1) (cells 6q + 2k and 6q + 2k + 1), share the vertices
// v0, v1 = v0 + e_p0 and v3 and the edges (0,1), (0,3), (1,3): the face that
// separates them.  Their 14 distinct P2 dofs, as a pair: pair dof n < 10 is
// local dof n of the first tet; the second tet's vertex 2 and its edges
// (0,2), (1,2), (2,3) (local dofs 2, 5, 7, 9) are pair dofs 10..13, and its
// other local dofs are the first tet's with the same number.
FE_KUHN_HD constexpr int pair_second_local(int n) {  // the second tet's local dof at pair dof n, -1 if none
  return n >= 10 ? (n == 10 ? 2 : n == 11 ? 5 : n == 12 ? 7 : 9)
                 : (n == 2 || n == 5 || n == 7 || n == 9 ? -1 : n);
}

// The stiffness of such a pair with one c for both tets, divided by 4 c: the
// two integer element matrices K added on the 14 pair dofs.
FE_KUHN_HD constexpr int kuhn_pair_k(int m, int n) {
  const int sm = pair_second_local(m), sn = pair_second_local(n);
  return (m < 10 && n < 10 ? kuhn_p2_k(m, n) : 0) + (sm >= 0 && sn >= 0 ? kuhn_p2_k(sm, sn) : 0);
}

// The pair's limb sums stay exact while every row of |K_pair| sums to at most
// 127 (127 * 2^17 < 2^24, the integers FP32 holds exactly).
FE_KUHN_HD constexpr int kuhn_pair_k_absrow_max() {
  int mx = 0;
  for (int m = 0; m < 14; ++m) {
    int absrow = 0;
    for (int n = 0; n < 14; ++n) absrow += kuhn_pair_k(m, n) < 0 ? -kuhn_pair_k(m, n) : kuhn_pair_k(m, n);
    mx = absrow > mx ? absrow : mx;
  }
  return mx;
}
FE_KUHN_HD constexpr bool kuhn_pair_k_ok() {
  for (int m = 0; m < 14; ++m) {
    int row = 0;
    for (int n = 0; n < 14; ++n) {
      if (kuhn_pair_k(m, n) != kuhn_pair_k(n, m)) return false;
      row += kuhn_pair_k(m, n);
    }
    if (row != 0) return false;
  }
  return kuhn_pair_k_absrow_max() <= 127;
}

// P2 prolongation weights on nested Kuhn meshes, times 8 (integers): the
// coarse P2 function of a cube evaluated at the fine P2 node o / 4 of that
// cube (o in [0, 4]^3, fine lattice units), as the sum over the basis
// functions of the Kuhn tet containing the point: the tet follows the
// descending order of the coordinates (ties resolved by axis order; the
// basis functions of the shared face agree there), its barycentrics are
// L / 4 with integer L, a vertex function is L (L - 2) / 8 and an edge
// function 2 L_i L_j / 8.  (a, b, d) in [0, 2]^3 is the coarse node, in
// coarse P2 lattice units from the cube's corner.
FE_KUHN_HD constexpr int pro_w8(int ox, int oy, int oz, int a, int b, int d) {
  const int s[3] = {ox, oy, oz};
  int sg[3] = {0, 1, 2};
  // stable descending sort of the three coordinates
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j + 1 < 3 - i; ++j)
      if (s[sg[j + 1]] > s[sg[j]]) {
        const int t = sg[j];
        sg[j] = sg[j + 1];
        sg[j + 1] = t;
      }
  const int L[4] = {4 - s[sg[0]], s[sg[0]] - s[sg[1]], s[sg[1]] - s[sg[2]], s[sg[2]]};
  int v[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
  v[1][sg[0]] = 1;
  v[2][sg[0]] = 1;
  v[2][sg[1]] = 1;
  const int n[3] = {a, b, d};
  for (int k = 0; k < 4; ++k)
    if (n[0] == 2 * v[k][0] && n[1] == 2 * v[k][1] && n[2] == 2 * v[k][2]) return L[k] * (L[k] - 2);
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (n[0] == v[i][0] + v[j][0] && n[1] == v[i][1] + v[j][1] && n[2] == v[i][2] + v[j][2]) return 2 * L[i] * L[j];
  return 0;
}

}  // namespace fe_kuhn
