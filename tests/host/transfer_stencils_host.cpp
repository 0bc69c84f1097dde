// Host-only driver for tests/test_transfer_stencils_host.py: prints the
// library's transfer stencils (fe_stencils.h) for the degree given as argv[1],
// one line per prolongation entry ("p class dx dy dz w") and per restriction
// tap ("r class ox oy oz w").
#include <cstdio>
#include <cstdlib>

#include "fe_stencils.h"

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  const int deg = std::atoi(argv[1]);
  std::vector<int> ps, rs;
  std::vector<fe_stencil::Entry> pro;
  std::vector<fe_stencil::Tap> res;
  fe_stencil::prolongation(deg, ps, pro);
  fe_stencil::restriction(deg, pro, rs, res);
  for (size_t q = 0; q + 1 < ps.size(); ++q)
    for (int e = ps[q]; e < ps[q + 1]; ++e)
      std::printf("p %zu %d %d %d %.17g\n", q, pro[e].d[0], pro[e].d[1], pro[e].d[2], pro[e].w);
  for (size_t q = 0; q + 1 < rs.size(); ++q)
    for (int e = rs[q]; e < rs[q + 1]; ++e)
      std::printf("r %zu %d %d %d %.17g\n", q, res[e].off[0], res[e].off[1], res[e].off[2], res[e].w);
  return 0;
}
