// Transfer stencils between the P_k spaces of nested Kuhn meshes (host code,
// no CUDA types; fe_api.cu uploads them).
//
// Prolongation is exact interpolation of the coarse P_k function at the fine
// nodes (Section 3, the MeshHierarchy transfers).  A fine lattice point
// (spacing h / 2k) is 2k B + o with B its coarse cube and o in [0, 2k)^3 its
// class; its position o / 2k inside the cube lies in the Kuhn tet given by the
// descending order of the coordinates, whose barycentrics are exact dyadic
// numbers, and the coarse basis functions of that tet at the point give the
// entries (o, d, w): fine value += w * coarse value at k B + d.  Restriction
// is the transpose: coarse point c receives w * r(2 c + o - 2 d) from every
// entry with d = c (mod k) per axis.
#pragma once

#include <algorithm>
#include <vector>

namespace fe_stencil {

struct Entry {
  int o[3];  // class of the fine point (offset inside the coarse cube, fine lattice units)
  int d[3];  // coarse lattice point relative to k B
  double w;
};

struct Tap {
  int off[3];  // fine point relative to 2 c
  double w;
};

// Entries of every prolongation class, classes in the order o_x fastest, then
// o_y, o_z; class q holds ents[start[q] .. start[q + 1]).  Zero weights are
// left out.
inline void prolongation(int deg, std::vector<int>& start, std::vector<Entry>& ents) {
  const int K2 = 2 * deg;
  start.assign(1, 0);
  ents.clear();
  for (int oz = 0; oz < K2; ++oz)
    for (int oy = 0; oy < K2; ++oy)
      for (int ox = 0; ox < K2; ++ox) {
        const int o[3] = {ox, oy, oz};
        const double s[3] = {ox / (double)K2, oy / (double)K2, oz / (double)K2};
        int sig[3] = {0, 1, 2};
        std::stable_sort(sig, sig + 3, [&](int a, int b) { return s[a] > s[b]; });
        const double lam[4] = {1.0 - s[sig[0]], s[sig[0]] - s[sig[1]], s[sig[1]] - s[sig[2]], s[sig[2]]};
        int v[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 1}};
        v[1][sig[0]] = 1;
        v[2][sig[0]] = 1;
        v[2][sig[1]] = 1;
        auto push = [&](const int d[3], double w) {
          if (w == 0.0) return;
          ents.push_back(Entry{{o[0], o[1], o[2]}, {d[0], d[1], d[2]}, w});
        };
        if (deg == 1) {
          for (int i = 0; i < 4; ++i) push(v[i], lam[i]);
        } else if (deg == 3) {
          // barycentrics l/6 with integer l: the P3 basis values are l-polynomials over
          // powers of two (vertex l(l-2)(l-4)/48, edge l_p l_q (l_p - 2)/16, face
          // l_a l_b l_c / 8), so the weights and their zeros are exact
          int sv[3] = {o[0], o[1], o[2]};
          std::sort(sv, sv + 3, [](int a, int b) { return a > b; });
          const int l[4] = {K2 - sv[0], sv[0] - sv[1], sv[1] - sv[2], sv[2]};
          for (int i = 0; i < 4; ++i) {
            const int d[3] = {3 * v[i][0], 3 * v[i][1], 3 * v[i][2]};
            push(d, (double)(l[i] * (l[i] - 2) * (l[i] - 4)) / 48.0);
          }
          for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
              for (int h = 0; h < 2; ++h) {
                const int pp = h ? b : a, q = h ? a : b;
                const int d[3] = {2 * v[pp][0] + v[q][0], 2 * v[pp][1] + v[q][1], 2 * v[pp][2] + v[q][2]};
                push(d, (double)(l[pp] * l[q] * (l[pp] - 2)) / 16.0);
              }
          for (int f = 0; f < 4; ++f) {
            // the face opposite vertex f: its k-th vertex is k + (k >= f)
            const int a = f == 0 ? 1 : 0, b = f <= 1 ? 2 : 1, c = f <= 2 ? 3 : 2;
            const int d[3] = {v[a][0] + v[b][0] + v[c][0], v[a][1] + v[b][1] + v[c][1], v[a][2] + v[b][2] + v[c][2]};
            push(d, (double)(l[a] * l[b] * l[c]) / 8.0);
          }
        } else {
          for (int i = 0; i < 4; ++i) {
            const int d[3] = {2 * v[i][0], 2 * v[i][1], 2 * v[i][2]};
            push(d, lam[i] * (2.0 * lam[i] - 1.0));
          }
          for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
              const int d[3] = {v[a][0] + v[b][0], v[a][1] + v[b][1], v[a][2] + v[b][2]};
              push(d, 4.0 * lam[a] * lam[b]);
            }
        }
        start.push_back((int)ents.size());
      }
}

// Restriction taps grouped by the class code (c_x mod k) + k (c_y mod k) +
// k^2 (c_z mod k) of the coarse point c; class q holds taps[start[q] .. start[q + 1]).
inline void restriction(int deg, const std::vector<Entry>& pro, std::vector<int>& start, std::vector<Tap>& taps) {
  start.assign(1, 0);
  taps.clear();
  for (int cls = 0; cls < deg * deg * deg; ++cls) {
    for (const Entry& e : pro) {
      const int code = (e.d[0] % deg) + deg * ((e.d[1] % deg) + deg * (e.d[2] % deg));
      if (code != cls) continue;
      taps.push_back(Tap{{e.o[0] - 2 * e.d[0], e.o[1] - 2 * e.d[1], e.o[2] - 2 * e.d[2]}, e.w});
    }
    start.push_back((int)taps.size());
  }
}

}  // namespace fe_stencil
