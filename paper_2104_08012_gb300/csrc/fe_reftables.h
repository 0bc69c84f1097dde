// Reference-element tables of the Lagrange P1/P2/P3 bases of the paper's
// function spaces (Section 2); host code, no CUDA types: the consistent mass
// matrices of the reference tet, the reference P3 stiffness coefficients, and
// the quadrature rule of the load vector with the basis values at its points.
// fe_kernels.cu uploads them to constant memory.
//
// Local dof order: vertices 0..3; P2 edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
// as dofs 4..9; P3 per edge in that order the node nearer its first vertex,
// then the other (dofs 4..15), then the face opposite vertex 0..3 (16..19).
#pragma once

#include <cmath>

#include "fe.h"

namespace fe_ref {

// P2 local dof of edge (a, b)
constexpr int edge_dof(int a, int b) {
  return a > b ? edge_dof(b, a) : (a == 0 ? 3 + b : (a == 1 ? 5 + b : 9));
}

// k-th vertex (k = 0, 1, 2) of the face opposite vertex f
constexpr int face_vertex(int f, int k) { return k + (k >= f ? 1 : 0); }

inline double fact(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

// int_ref phi_i phi_j on the reference tet for P1 (4 x 4) and P2 (10 x 10).
// Every P1/P2 basis function is a homogeneous polynomial in the barycentrics
// (P1: lambda_i; P2: lambda_v^2 - sum_{w!=v} lambda_v lambda_w and
// 4 lambda_a lambda_b), and int_ref lambda^alpha = alpha! / (|alpha| + 3)!.
inline void mass_tables(double m1[16], double m2[100]) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) m1[i * 4 + j] = (i == j ? 2.0 : 1.0) / 120.0;
  // P2 basis as symmetric quadratic forms Q[i][a][b] in the barycentrics
  double Q[10][4][4] = {};
  for (int v = 0; v < 4; ++v) {
    Q[v][v][v] = 1.0;
    for (int w = 0; w < 4; ++w)
      if (w != v) {
        Q[v][v][w] -= 0.5;
        Q[v][w][v] -= 0.5;
      }
  }
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b) {
      const int e = edge_dof(a, b);
      Q[e][a][b] = 2.0;
      Q[e][b][a] = 2.0;
    }
  for (int i = 0; i < 10; ++i)
    for (int j = 0; j < 10; ++j) {
      double s = 0.0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          for (int c = 0; c < 4; ++c)
            for (int d = 0; d < 4; ++d) {
              const double q = Q[i][a][b] * Q[j][c][d];
              if (q == 0.0) continue;
              int al[4] = {0, 0, 0, 0};
              al[a]++;
              al[b]++;
              al[c]++;
              al[d]++;
              s += q * fact(al[0]) * fact(al[1]) * fact(al[2]) * fact(al[3]) / fact(7);
            }
      m2[i * 10 + j] = s;
    }
}

// P3 Lagrange basis on the reference tet at xi:
// vertex v: lam (3 lam - 1)(3 lam - 2) / 2; the edge node nearer p on edge
// (p, q): 9/2 lam_p lam_q (3 lam_p - 1); face (a, b, c): 27 lam_a lam_b lam_c.
inline void p3_basis(const double xi[3], double phi[20], double dphi[20][3]) {
  const double lam[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
  const double dl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int v = 0; v < 4; ++v) {
    const double L = lam[v];
    phi[v] = 0.5 * L * (3 * L - 1) * (3 * L - 2);
    for (int a = 0; a < 3; ++a) dphi[v][a] = 0.5 * (27 * L * L - 18 * L + 2) * dl[v][a];
  }
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b) {
      const int e = edge_dof(a, b) - 4;
      for (int h = 0; h < 2; ++h) {
        const int p = h ? b : a, q = h ? a : b, i = 4 + 2 * e + h;
        phi[i] = 4.5 * lam[p] * lam[q] * (3 * lam[p] - 1);
        for (int c = 0; c < 3; ++c)
          dphi[i][c] = 4.5 * (lam[q] * (6 * lam[p] - 1) * dl[p][c] + lam[p] * (3 * lam[p] - 1) * dl[q][c]);
      }
    }
  for (int f = 0; f < 4; ++f) {
    const int a = face_vertex(f, 0), b = face_vertex(f, 1), c = face_vertex(f, 2);
    phi[16 + f] = 27 * lam[a] * lam[b] * lam[c];
    for (int d = 0; d < 3; ++d)
      dphi[16 + f][d] = 27 * (lam[b] * lam[c] * dl[a][d] + lam[a] * lam[c] * dl[b][d] + lam[a] * lam[b] * dl[c][d]);
  }
}

// The load vector's rule: Gauss-Legendre with 3 nodes on [0, 1] per direction,
// collapsed to the reference tet (xi = u, eta = (1-u) v, zeta = (1-u)(1-v) w,
// weight w_u w_v w_w (1-u)^2 (1-v)), points ordered u slowest, w fastest; and
// the P1/P2/P3 basis values there.
inline void quad_tables(double xi[FE_QUAD_POINTS][3], double w[FE_QUAD_POINTS], double phi1[FE_QUAD_POINTS][4],
                        double phi2[FE_QUAD_POINTS][10], double phi3[FE_QUAD_POINTS][20]) {
  const double r = std::sqrt(0.6);
  const double t[3] = {0.5 * (1.0 - r), 0.5, 0.5 * (1.0 + r)};
  const double wt[3] = {0.5 * 5.0 / 9.0, 0.5 * 8.0 / 9.0, 0.5 * 5.0 / 9.0};
  int q = 0;
  for (int iu = 0; iu < 3; ++iu)
    for (int iv = 0; iv < 3; ++iv)
      for (int iw = 0; iw < 3; ++iw, ++q) {
        const double u = t[iu], v = t[iv], ww = t[iw];
        xi[q][0] = u;
        xi[q][1] = (1.0 - u) * v;
        xi[q][2] = (1.0 - u) * (1.0 - v) * ww;
        w[q] = wt[iu] * wt[iv] * wt[iw] * (1.0 - u) * (1.0 - u) * (1.0 - v);
        const double lam[4] = {1.0 - xi[q][0] - xi[q][1] - xi[q][2], xi[q][0], xi[q][1], xi[q][2]};
        for (int k = 0; k < 4; ++k) {
          phi1[q][k] = lam[k];
          phi2[q][k] = lam[k] * (2.0 * lam[k] - 1.0);
        }
        int e = 4;
        for (int a = 0; a < 4; ++a)
          for (int b2 = a + 1; b2 < 4; ++b2) phi2[q][e++] = 4.0 * lam[a] * lam[b2];
        double d[20][3];
        p3_basis(xi[q], phi3[q], d);
      }
}

// Gauss-Legendre nodes and weights on [0, 1] (Newton's method on the
// three-term Legendre recurrence, P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1)).
inline void gauss_legendre01(int n, double* t, double* w) {
  for (int i = 0; i < n; ++i) {
    double x = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    t[i] = 0.5 * (x + 1.0);
    w[i] = 1.0 / ((1.0 - x * x) * dp * dp);  // half the [-1, 1] weight 2 / ((1 - x^2) P_n'(x)^2)
  }
}

// Reference P3 stiffness coefficients and mass matrix, by the conical-product
// Gauss rule with 5 points per direction (exact to degree 7; the integrands
// have degree 4 and 6).  K[p] for the dof pair p = (i <= j, row-major upper
// triangle) holds int d_0 phi_i d_0 phi_j, int (d_0 phi_i d_1 phi_j + d_1 phi_i
// d_0 phi_j), the same for (0, 2), then (1, 1), (1, 2), (2, 2): the element
// matrix is sum_k G_k K[p][k] for the symmetric 3 x 3 factors G = |det J|
// J^-1 J^-T in the order 00, 01, 02, 11, 12, 22.  M = int phi_i phi_j, 20 x 20.
inline void p3_tables(double K[210][6], double M[400]) {
  double t[5], w[5];
  gauss_legendre01(5, t, w);
  for (int p = 0; p < 210; ++p)
    for (int k = 0; k < 6; ++k) K[p][k] = 0.0;
  for (int i = 0; i < 400; ++i) M[i] = 0.0;
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b)
      for (int c = 0; c < 5; ++c) {
        const double u = t[a], v = t[b], z = t[c];
        const double xi[3] = {u, (1 - u) * v, (1 - u) * (1 - v) * z};
        const double wq = w[a] * w[b] * w[c] * (1 - u) * (1 - u) * (1 - v);
        double phi[20], d[20][3];
        p3_basis(xi, phi, d);
        for (int i = 0, p = 0; i < 20; ++i)
          for (int j = i; j < 20; ++j, ++p) {
            K[p][0] += wq * d[i][0] * d[j][0];
            K[p][1] += wq * (d[i][0] * d[j][1] + d[i][1] * d[j][0]);
            K[p][2] += wq * (d[i][0] * d[j][2] + d[i][2] * d[j][0]);
            K[p][3] += wq * d[i][1] * d[j][1];
            K[p][4] += wq * (d[i][1] * d[j][2] + d[i][2] * d[j][1]);
            K[p][5] += wq * d[i][2] * d[j][2];
          }
        for (int i = 0; i < 20; ++i)
          for (int j = 0; j < 20; ++j) M[i * 20 + j] += wq * phi[i] * phi[j];
      }
}

}  // namespace fe_ref
