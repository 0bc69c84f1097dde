// Cell-loop kernels of the matrix-free operator (paper Section 2, Eq. 4),
// mass, diagonal, adjoint cell gradient, mesh construction, and the
// multigrid transfer and smoother vector kernels (paper Section 3).
#include <array>
#include <cmath>
#include <mutex>
#include <vector>
#include <type_traits>

#include "fe_df.cuh"
#include "fe_kuhn.h"
#include "fe_internal.cuh"
#include "fe_p3.cuh"
#include "fe_reftables.h"

// Reference P1/P2/P3 mass matrices int_ref phi_i phi_j (fe_reftables.h),
// uploaded when the first hierarchy is created on each device.
__constant__ double c_mref1[16];
__constant__ double c_mref2[100];
__constant__ double c_mref3[400];
// P3 reference stiffness: for the symmetric pairs p = (i <= j) of the 20
// local dofs (row-major packed upper triangle), the coefficients of the six
// components (00, 01, 02, 11, 12, 22) of G = |det J| J^-1 J^-T:
// A_K[i][j] = kappa_K sum_k G_k c_K3[p][k], with c_K3[p][k] = int_ref
// d_a phi_i d_b phi_j (+ d_b phi_i d_a phi_j for a != b).  The operator applies
// the element through the gradient at the P2 nodes (fe_p3.cuh); these entries
// serve the diagonal, the coarse assembly and the patch matrices.
__constant__ double c_K3[210][6];
// P3 vertex-star patch slots: lattice offsets from 3 V on the 3N lattice of
// the vertex (0), the two nodes of each of its 14 edges (d, 2 d) and the
// centroids of its 36 faces (d1 + d2); filled by launch_patch_setup_p3.
__constant__ int c_p3slot[65][3];
// Quadrature rule of the load vector (conical-product Gauss, 3 points per
// direction, FE_QUAD_POINTS = 27 per tet): reference points, weights, basis values.
__constant__ double c_qxi[FE_QUAD_POINTS][3];
__constant__ double c_qw[FE_QUAD_POINTS];
__constant__ double c_qphi1[FE_QUAD_POINTS][4];
__constant__ double c_qphi2[FE_QUAD_POINTS][10];
__constant__ double c_qphi3[FE_QUAD_POINTS][20];

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ int decode(int m, bool& bd) {
  bd = m < 0;
  return bd ? -1 - m : m;
}

// Diagonal entry A_K[i][i] of the P3 element (g = kappa G / 161280 as stored).
__device__ __forceinline__ double p3_diag_entry(const double* g, int i) {
  const int p = 20 * i - i * (i - 1) / 2;
  return 161280.0 * (g[0] * c_K3[p][0] + g[1] * c_K3[p][1] + g[2] * c_K3[p][2] + g[3] * c_K3[p][3] +
                     g[4] * c_K3[p][4] + g[5] * c_K3[p][5]);
}

template <int DEG, typename T>
__device__ __forceinline__ void tet_element(const T* u, const T* g, T* y) {
  if constexpr (DEG == 3) {
    const T gg[6] = {g[0], g[1], g[2], g[3], g[4], g[5]};
    fe_p3::p3_element_grad<fe_p3::PlainOps<T>>(u, gg, y);
  } else {
    element_apply<DEG, T>(u, g, y);
  }
}

// The same with G = c M (every Kuhn tet shares M = [[2,-1,0],[-1,2,-1],[0,-1,1]]).
template <int DEG, typename T>
__device__ __forceinline__ void tet_element_m(const T* u, T c, T* y) {
  if constexpr (DEG == 3) {
    const T gg[6] = {c, T(0), T(0), T(0), T(0), T(0)};
    fe_p3::p3_element_grad<fe_p3::PlainOps<T>, true>(u, gg, y);
  } else {
    const T g[6] = {T(2) * c, -c, T(0), T(2) * c, -c, c};
    element_apply<DEG, T>(u, g, y);
  }
}

// Geometric factors are stored as kappa G / w: w = 6 (P1), 120 (P2) and
// 161280 = 64 x 2520 (P3) fold the element formulas' reference integrals.
template <int DEG>
__host__ __device__ constexpr double geo_weight() { return DEG == 1 ? 6.0 : DEG == 2 ? 120.0 : 161280.0; }

// ------------------------------------------------------ mesh construction
template <int DEG>
__global__ void k_build_map(Numbering num, int C, int Cs, int* __restrict__ map) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int N = num.N;
  const int q = c / 6, t = c - 6 * (c / 6);
  const int ci = q % N, cj = (q / N) % N, ck = q / (N * N);
  int p0, p1, p2;
  kuhn_perm(t, p0, p1, p2);
  int v[4][3];
  v[0][0] = ci; v[0][1] = cj; v[0][2] = ck;
#pragma unroll
  for (int a = 0; a < 3; ++a) v[1][a] = v[0][a] + (a == p0);
#pragma unroll
  for (int a = 0; a < 3; ++a) v[2][a] = v[1][a] + (a == p1);
#pragma unroll
  for (int a = 0; a < 3; ++a) v[3][a] = v[0][a] + 1;
  const int m = num.m;
  auto put = [&](int j, int x, int y, int z) {
    const int dof = lattice_to_dof(num, x, y, z);
    const bool bd = x == 0 || y == 0 || z == 0 || x == m || y == m || z == m;
    map[(size_t)j * Cs + c] = bd ? -1 - dof : dof;
  };
  if (DEG == 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) put(k, v[k][0], v[k][1], v[k][2]);
  } else if (DEG == 3) {
#pragma unroll
    for (int k = 0; k < 4; ++k) put(k, 3 * v[k][0], 3 * v[k][1], 3 * v[k][2]);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a + 1; b < 4; ++b) {
        const int e = p2_edge(a, b) - 4;
        put(4 + 2 * e, 2 * v[a][0] + v[b][0], 2 * v[a][1] + v[b][1], 2 * v[a][2] + v[b][2]);
        put(5 + 2 * e, v[a][0] + 2 * v[b][0], v[a][1] + 2 * v[b][1], v[a][2] + 2 * v[b][2]);
      }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int a = p3_face_vertex(f, 0), b = p3_face_vertex(f, 1), d = p3_face_vertex(f, 2);
      put(16 + f, v[a][0] + v[b][0] + v[d][0], v[a][1] + v[b][1] + v[d][1], v[a][2] + v[b][2] + v[d][2]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) put(k, 2 * v[k][0], 2 * v[k][1], 2 * v[k][2]);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a + 1; b < 4; ++b)
        put(p2_edge(a, b), v[a][0] + v[b][0], v[a][1] + v[b][1], v[a][2] + v[b][2]);
  }
}

// P3: coordinates of every lattice point indexed by its dof, so that the map
// rows of the tet vertices index them as they index the vertices for P1/P2.
__global__ void k_build_coords_lattice(Numbering num, int n, double* __restrict__ vx, double* __restrict__ vy,
                                       double* __restrict__ vz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x, y, z;
  dof_to_lattice(num, i, x, y, z);
  const double m = (double)num.m;
  vx[i] = x / m;
  vy[i] = y / m;
  vz[i] = z / m;
}

__global__ void k_build_coords(int N, int V, double* __restrict__ vx, double* __restrict__ vy, double* __restrict__ vz) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int n1 = N + 1;
  const double dn = (double)N;
  vx[v] = (v % n1) / dn;
  vy[v] = ((v / n1) % n1) / dn;
  vz[v] = (v / (n1 * n1)) / dn;
}

// ----------------------------------------------------------- geometry
template <int DEG>
__global__ void k_geometry(int C, int Cs, const int* __restrict__ map, const double* __restrict__ vx,
                           const double* __restrict__ vy, const double* __restrict__ vz,
                           const double* __restrict__ kappa, double* __restrict__ geo64, float* __restrict__ geo32,
                           double* __restrict__ detj) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double p[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    bool bd;
    const int v = decode(map[(size_t)k * Cs + c], bd);  // vertex dofs are numbered first
    p[k][0] = vx[v];
    p[k][1] = vy[v];
    p[k][2] = vz[v];
  }
  double g[6], adet;
  tet_metric<double>(p, g, adet);
  const double s = kappa[c] / geo_weight<DEG>();
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    geo64[(size_t)a * Cs + c] = g[a] * s;
    geo32[(size_t)a * Cs + c] = (float)(g[a] * s);
  }
  detj[c] = adet;
}

// geo64 = c M for every cell (M = [[2,-1,0],[-1,2,-1],[0,-1,1]] in the stored
// order 00, 01, 02, 11, 12, 22), c = geo64[22]; a cell whose G differs from
// c M by more than 1e-12 |c| sets bit 0 of the flag, an odd cell whose c
// differs from that of the cell before it (the other tet of its pair) bit 1.
__global__ void k_uniform_geometry(int C, int Cs, const double* __restrict__ geo64, float* __restrict__ c32,
                                   float2* __restrict__ cdf, int* __restrict__ flag) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C) return;
  const double c = geo64[(size_t)5 * Cs + t];
  const double m[5] = {2.0, -1.0, 0.0, 2.0, -1.0};
  bool ok = c >= 0x1p-100 && c <= 0x1p100;  // the float-pair kernels normalise c.hi by its exponent field
#pragma unroll
  for (int a = 0; a < 5; ++a) ok = ok && fabs(geo64[(size_t)a * Cs + t] - m[a] * c) <= 1e-12 * c;
  if (!ok) atomicOr(flag, 1);
  if ((t & 1) && c != geo64[(size_t)5 * Cs + t - 1]) atomicOr(flag, 2);
  c32[t] = (float)c;
  const float hi = (float)c;
  cdf[t] = make_float2(hi, (float)(c - (double)hi));
}

// ------------------------------------------------------ operator apply
// One thread per tet: gather the cell dofs through the cell->dof map
// (coalesced: the map is stored [dof][cell]), contract with the cell's
// geometric factors, scatter-add with atomics.  Extra threads past the last
// cell copy x -> y on the Dirichlet dofs (identity rows).
// UNI: only row 5 of geo is read, c = G_22 with G = c M (see Level).
template <int DEG, typename T, bool UNI>
__global__ void __launch_bounds__(kBlock) k_apply(int C, int Cs, int Cpad, const int* __restrict__ map,
                                                  const T* __restrict__ geo, const T* __restrict__ x,
                                                  T* __restrict__ y, int nb, const int* __restrict__ bnd) {
  constexpr int ND = tet_ndof(DEG);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < C) {
    int idx[ND];
    T u[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      idx[j] = __ldg(map + (size_t)j * Cs + t);
      u[j] = idx[j] >= 0 ? __ldg(x + idx[j]) : T(0);
    }
    T out[ND];
    if constexpr (UNI) {
      tet_element_m<DEG, T>(u, __ldg(geo + (size_t)5 * Cs + t), out);
    } else {
      T g[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) g[a] = __ldg(geo + (size_t)a * Cs + t);
      tet_element<DEG, T>(u, g, out);
    }
#pragma unroll
    for (int j = 0; j < ND; ++j)
      if (idx[j] >= 0) atomicAdd(y + idx[j], out[j]);
  } else if (t >= Cpad && t - Cpad < nb) {
    const int i = bnd[t - Cpad];
    y[i] = x[i];
  }
}

// Lift of inhomogeneous Dirichlet data (symmetric elimination of u = g on the
// boundary): b_i -= (A g)_i on every interior dof i, where g holds the
// Dirichlet values on the boundary dofs and 0 inside.  Only tets with a
// Dirichlet dof contribute; the others leave after reading their map rows.
// FP64 FMAs: it runs once per solve, on the boundary layer of cells.
template <int DEG>
__global__ void __launch_bounds__(kBlock) k_bc_lift(int C, int Cs, const int* __restrict__ map,
                                                    const double* __restrict__ geo, const double* __restrict__ g,
                                                    double* __restrict__ b) {
  constexpr int ND = tet_ndof(DEG);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C) return;
  int idx[ND];
  double u[ND];
  bool any = false;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    idx[j] = __ldg(map + (size_t)j * Cs + t);
    any = any || idx[j] < 0;
    u[j] = idx[j] < 0 ? __ldg(g + (-1 - idx[j])) : 0.0;
  }
  if (!any) return;
  double gg[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) gg[a] = __ldg(geo + (size_t)a * Cs + t);
  double out[ND];
  tet_element<DEG, double>(u, gg, out);
#pragma unroll
  for (int j = 0; j < ND; ++j)
    if (idx[j] >= 0) atomicAdd(b + idx[j], -out[j]);
}

// Cube-aggregated apply: one thread per cube gathers the cube's (k+1)^3 dofs
// once, applies its six Kuhn tets into register accumulators and scatters
// (k+1)^3 atomics instead of 6 * nd (27 instead of 60 for P2).
constexpr int kCubeBlock = 128;
// The uniform-geometry FP32 cube kernel is gather-latency-bound: compiled for 6 resident blocks per SM (80
// registers, 60 bytes of spill) it ran 0.134 ms at P2 128^3 against 0.138 ms for 5 (96 registers) and 0.148 ms
// for 4 (109 registers); streaming cache hints on the cube map and c made it slower (0.167 ms).
constexpr int kCubeMinBlocksUni = 6;  // 4 blocks of 128 per SM at 128 registers: 5% faster than 2 of 256

// UNI: geo is c32 (one value per cell, geometric factors c M, see Level)
// instead of the six stored factors per cell.
template <int DEG, bool FUSE, bool UNI>
__global__ void __launch_bounds__(kCubeBlock, UNI ? kCubeMinBlocksUni : 4) k_apply_cube(int Q, int Qs, int Cs, int Qpad,
                                                            const int* __restrict__ cmap,
                                                            const float* __restrict__ geo, const float* x,
                                                            float* __restrict__ y, int nb, const int* __restrict__ bnd,
                                                            ChebFuse<float> cf) {
  constexpr int NL = DEG == 1 ? 8 : 27, ND = DEG == 1 ? 4 : 10;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < Q) {
    float xv[NL], acc[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int i = __ldg(cmap + (size_t)l * Qs + q);
      // with FUSE, x changes during the launch (each dof once, after its last reader)
      xv[l] = i >= 0 ? (FUSE ? x[i] : __ldg(x + i)) : 0.0f;
      acc[l] = 0.0f;
    }
    // The cube's six tets are cells 6q .. 6q+5, contiguous in every row of
    // geo: one 8-byte load fetches G_a (or c) of two tets.
    constexpr int NR = UNI ? 1 : 6;
    float2 gp[NR][3];
#pragma unroll
    for (int a = 0; a < NR; ++a)
#pragma unroll
      for (int h = 0; h < 3; ++h) gp[a][h] = __ldg(reinterpret_cast<const float2*>(geo + (size_t)a * Cs + 6 * q) + h);
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      float u[ND], g[6], o[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) u[j] = xv[cube_local(DEG, t, j)];
      if constexpr (UNI) {
        const float c = (t & 1) ? gp[0][t >> 1].y : gp[0][t >> 1].x;
        g[0] = 2.0f * c, g[1] = -c, g[2] = 0.0f, g[3] = 2.0f * c, g[4] = -c, g[5] = c;
      } else {
#pragma unroll
        for (int a = 0; a < 6; ++a) g[a] = (t & 1) ? gp[a][t >> 1].y : gp[a][t >> 1].x;
      }
      element_apply<DEG, float>(u, g, o);
#pragma unroll
      for (int j = 0; j < ND; ++j) acc[cube_local(DEG, t, j)] += o[j];
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int i = __ldg(cmap + (size_t)l * Qs + q);
      if (i >= 0) atomicAdd(y + i, acc[l]);
    }
    if constexpr (FUSE) {
      // this cube's contributions reach L2 before its countdowns do; the cube
      // that ends a dof's countdown therefore reads the complete y_i
      fence_acq_rel_gpu();
      for (int l = 0; l < NL; ++l) {
        const int i = __ldg(cmap + (size_t)l * Qs + q);
        if (i >= 0 && atomicSub(cf.cnt + i, 1u) == 1u) {
          fence_acq_rel_gpu();
          cf.cnt[i] = __ldg(cf.val + i);
          cheb_update(i, __ldcg(y + i), cf.b, cf.dinv, cf.x, cf.d, cf.c1, cf.c2, cf.store_d);
        }
      }
    }
  } else if (q >= Qpad && q - Qpad < nb) {
    const int i = bnd[q - Qpad];
    const float xi = x[i];
    y[i] = xi;
    if constexpr (FUSE) cheb_update(i, xi, cf.b, cf.dinv, cf.x, cf.d, cf.c1, cf.c2, cf.store_d);
  }
}

// The uniform-geometry FP32 cube apply as a persistent loop over cubes: each
// thread's cube map rows two cubes ahead are copied into shared memory by
// cp.async ([buffer][node][thread], three buffers), and the next cube's dofs
// and c values are gathered into registers while the current cube is
// contracted, so the dependent map -> x gathers no longer stall every cube.
// 128 threads, 4 resident blocks per SM (128 registers, 41 KB of staged map per
// block): P2 applications measured 0.1305 / 0.0269 ms at 128^3 / 64^3, against
// 0.1513 / 0.0287 ms at 5 blocks (96 registers, spills) and 0.131-0.134 /
// 0.0297 ms for the one-cube-per-thread kernel without staging (k_apply_cube).
constexpr int kCubeLpBlock = 128;
constexpr int kCubeLpMinBlocks = 4;

template <int DEG>
__global__ void __launch_bounds__(kCubeLpBlock, DEG == 1 ? 8 : kCubeLpMinBlocks)
    k_apply_cube_lp32(int Q, int Qs, int Cs, const int* __restrict__ cmap, const float* __restrict__ c32,
                      const float* __restrict__ x, float* __restrict__ y, int nb, const int* __restrict__ bnd) {
  constexpr int NL = DEG == 1 ? 8 : 27, ND = DEG == 1 ? 4 : 10;
  __shared__ int smap[3][NL][kCubeLpBlock];
  const int tx = threadIdx.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < nb; i += stride) y[bnd[i]] = x[bnd[i]];  // Dirichlet rows: identity
  int q = tid;
  if (q >= Q) return;
  auto copy_map = [&](int cube, int buf) {
    if (cube < Q) {
#pragma unroll
      for (int l = 0; l < NL; ++l) cp_async4(&smap[buf][l][tx], cmap + (size_t)l * Qs + cube);
    }
    cp_async_commit();
  };
  auto gather = [&](int cube, int buf, float (&xv)[NL], float2 (&cv)[3]) {
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int i = smap[buf][l][tx];
      xv[l] = i >= 0 ? __ldg(x + i) : 0.0f;
    }
    // the cube's six tets are cells 6q .. 6q+5: three 8-byte loads of c
#pragma unroll
    for (int h = 0; h < 3; ++h) cv[h] = __ldg(reinterpret_cast<const float2*>(c32 + 6 * (size_t)cube) + h);
  };
  copy_map(q, 0);
  copy_map(q + stride, 1);
  cp_async_wait_all();
  float xv[NL];
  float2 cv[3];
  gather(q, 0, xv, cv);
  int b = 0;
  while (true) {
    const int qn = q + stride;
    const bool more = qn < Q;
    const int bn = b == 2 ? 0 : b + 1, bnn = bn == 2 ? 0 : bn + 1;
    float xn[NL];
    float2 cn[3];
    if (more) {
      cp_async_wait_all();  // the next cube's map rows (copied one iteration ago)
      gather(qn, bn, xn, cn);
      copy_map(qn + stride, bnn);
    }
    float acc[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) acc[l] = 0.0f;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      float u[ND], g[6], o[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) u[j] = xv[cube_local(DEG, t, j)];
      const float c = (t & 1) ? cv[t >> 1].y : cv[t >> 1].x;
      g[0] = 2.0f * c, g[1] = -c, g[2] = 0.0f, g[3] = 2.0f * c, g[4] = -c, g[5] = c;
      element_apply<DEG, float>(u, g, o);
#pragma unroll
      for (int j = 0; j < ND; ++j) acc[cube_local(DEG, t, j)] += o[j];
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int i = smap[b][l][tx];
      if (i >= 0) atomicAdd(y + i, acc[l]);
    }
    if (!more) break;
    q = qn;
    b = bn;
#pragma unroll
    for (int l = 0; l < NL; ++l) xv[l] = xn[l];
#pragma unroll
    for (int h = 0; h < 3; ++h) cv[h] = cn[h];
  }
  cp_async_wait_all();
}

// Contributors per interior dof: cells (nd map rows) or cubes (cube map rows).
__global__ void k_valence(int C, int Cs, int rows, const int* __restrict__ map, unsigned* __restrict__ v) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  for (int j = 0; j < rows; ++j) {
    const int m = map[(size_t)j * Cs + c];
    if (m >= 0) atomicAdd(v + m, 1u);
  }
}

template <int DEG>
__global__ void k_build_cube_map(Numbering num, int Q, int Qs, int* __restrict__ cmap) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const int N = num.N, m = num.m;
  const int ci = q % N, cj = (q / N) % N, ck = q / (N * N);
  constexpr int K = DEG + 1;
  for (int l = 0; l < K * K * K; ++l) {
    const int x = DEG * ci + l % K, y = DEG * cj + (l / K) % K, z = DEG * ck + l / (K * K);
    const int dof = lattice_to_dof(num, x, y, z);
    const bool bd = x == 0 || y == 0 || z == 0 || x == m || y == m || z == m;
    cmap[(size_t)l * Qs + q] = bd ? -1 - dof : dof;
  }
}

// ------------------------------------------------------------ mass
template <int DEG>
__global__ void k_mass(int C, int Cs, const int* __restrict__ map, const double* __restrict__ detj,
                       const double* __restrict__ x, double* __restrict__ y) {
  constexpr int ND = tet_ndof(DEG);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int idx[ND];
  double u[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    bool bd;
    idx[j] = decode(map[(size_t)j * Cs + c], bd);
    u[j] = x[idx[j]];
  }
  const double s = detj[c];
  const double* M = DEG == 1 ? c_mref1 : DEG == 2 ? c_mref2 : c_mref3;
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < ND; ++j) acc += M[i * ND + j] * u[j];
    atomicAdd(y + idx[i], s * acc);
  }
}

// ------------------------------------------------------ quadrature load
// Physical quadrature points x = p0 + J xi of every cell: xyz [C][27][3].
__global__ void k_quad_points(int C, int Cs, const int* __restrict__ map, const double* __restrict__ vx,
                              const double* __restrict__ vy, const double* __restrict__ vz, double* __restrict__ xyz) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double p[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    bool bd;
    const int v = decode(map[(size_t)k * Cs + c], bd);  // vertex dofs index the vertices
    p[k][0] = vx[v];
    p[k][1] = vy[v];
    p[k][2] = vz[v];
  }
  for (int q = 0; q < FE_QUAD_POINTS; ++q)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      xyz[((size_t)c * FE_QUAD_POINTS + q) * 3 + a] = p[0][a] + (p[1][a] - p[0][a]) * c_qxi[q][0] +
                                                       (p[2][a] - p[0][a]) * c_qxi[q][1] +
                                                       (p[3][a] - p[0][a]) * c_qxi[q][2];
}

// b_i += sum_q w_q |det J| f(x_q) phi_i(xi_q) for the cell's dofs (boundary rows are zeroed afterwards).
template <int DEG>
__device__ __forceinline__ double qphi(int q, int i) {
  if constexpr (DEG == 1)
    return c_qphi1[q][i];
  else if constexpr (DEG == 2)
    return c_qphi2[q][i];
  else
    return c_qphi3[q][i];
}

template <int DEG>
__global__ void k_load_quad(int C, int Cs, const int* __restrict__ map, const double* __restrict__ detj,
                            const double* __restrict__ fq, double* __restrict__ b) {
  constexpr int ND = tet_ndof(DEG);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double acc[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) acc[i] = 0.0;
  const double dj = detj[c];
  for (int q = 0; q < FE_QUAD_POINTS; ++q) {
    const double sq = c_qw[q] * dj * __ldg(fq + (size_t)c * FE_QUAD_POINTS + q);
#pragma unroll
    for (int i = 0; i < ND; ++i) acc[i] += sq * qphi<DEG>(q, i);
  }
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    bool bd;
    atomicAdd(b + decode(map[(size_t)i * Cs + c], bd), acc[i]);
  }
}

// ------------------------------------------------------------ diagonal
template <int DEG>
__global__ void k_diag(int C, int Cs, const int* __restrict__ map, const double* __restrict__ geo, double* __restrict__ diag) {
  constexpr int ND = tet_ndof(DEG);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double g[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) g[a] = geo[(size_t)a * Cs + c];
  if constexpr (DEG == 3) {  // straight from the reference coefficients
    for (int i = 0; i < ND; ++i) {
      const int m = map[(size_t)i * Cs + c];
      if (m >= 0) atomicAdd(diag + m, p3_diag_entry(g, i));
    }
  } else {  // the element applied to unit vectors
    for (int i = 0; i < ND; ++i) {
      const int m = map[(size_t)i * Cs + c];
      if (m < 0) continue;
      double u[ND], out[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) u[j] = (j == i) ? 1.0 : 0.0;
      tet_element<DEG, double>(u, g, out);
      atomicAdd(diag + m, out[i]);
    }
  }
}

__global__ void k_diag_finish(int n, int nb, const int* __restrict__ bnd, double* __restrict__ diag) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nb) diag[bnd[t]] = 1.0;
}

__global__ void k_invert(int n, const double* __restrict__ diag, double* __restrict__ d64, float* __restrict__ d32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = 1.0 / diag[i];
  d64[i] = v;
  d32[i] = (float)v;
}

// ---------------------------------------------------- adjoint gradient
// g_K = int_K grad(lambda) . grad(u) = lambda_K^T A_K(kappa=1) u_K, with the
// Dirichlet dofs of u and lambda taken as 0.
template <int DEG>
__global__ void k_gradient(int C, int Cs, const int* __restrict__ map, const double* __restrict__ vx,
                           const double* __restrict__ vy, const double* __restrict__ vz, const double* __restrict__ u,
                           const double* __restrict__ lam, double* __restrict__ g) {
  constexpr int ND = tet_ndof(DEG);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double uu[ND], ll[ND];
  double p[4][3];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    bool bd;
    const int i = decode(map[(size_t)j * Cs + c], bd);
    uu[j] = bd ? 0.0 : u[i];
    ll[j] = bd ? 0.0 : lam[i];
    if (j < 4) {
      p[j][0] = vx[i];
      p[j][1] = vy[i];
      p[j][2] = vz[i];
    }
  }
  double G[6], adet;
  tet_metric<double>(p, G, adet);
  const double s = 1.0 / geo_weight<DEG>();
#pragma unroll
  for (int a = 0; a < 6; ++a) G[a] *= s;
  double out[ND];
  tet_element<DEG, double>(uu, G, out);
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < ND; ++j) acc += ll[j] * out[j];
  g[c] = acc;
}

// ------------------------------------------------------ mesh queries
__global__ void k_dof_coords(Numbering num, int n, double* __restrict__ xyz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x, y, z;
  dof_to_lattice(num, i, x, y, z);
  const double m = (double)num.m;
  xyz[3 * (size_t)i + 0] = x / m;
  xyz[3 * (size_t)i + 1] = y / m;
  xyz[3 * (size_t)i + 2] = z / m;
}

__global__ void k_centroids(int C, int Cs, const int* __restrict__ map, const double* __restrict__ vx,
                            const double* __restrict__ vy, const double* __restrict__ vz, double* __restrict__ xyz) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double s[3] = {0, 0, 0};
  for (int k = 0; k < 4; ++k) {
    bool bd;
    const int v = decode(map[(size_t)k * Cs + c], bd);
    s[0] += vx[v];
    s[1] += vy[v];
    s[2] += vz[v];
  }
  for (int a = 0; a < 3; ++a) xyz[3 * (size_t)c + a] = 0.25 * s[a];
}

__global__ void k_bmask(Numbering num, int n, unsigned char* __restrict__ m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x, y, z;
  dof_to_lattice(num, i, x, y, z);
  m[i] = (x == 0 || y == 0 || z == 0 || x == num.m || y == num.m || z == num.m) ? 1 : 0;
}

// coarse kappa = mean of the 8 child cells (fixed summation order)
__global__ void k_coarsen_kappa(int Nc, int Cc, const int* __restrict__ children, const double* __restrict__ kf,
                                double* __restrict__ kc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Cc) return;
  const int q = c / 6, T = c - 6 * q;
  const int ci = q % Nc, cj = (q / Nc) % Nc, ck = q / (Nc * Nc);
  const int Nf = 2 * Nc;
  double s = 0.0;
  for (int k = 0; k < 8; ++k) {
    const int e = children[T * 8 + k];
    const int code = e >> 3, tf = e & 7;
    const int fi = 2 * ci + (code & 1), fj = 2 * cj + ((code >> 1) & 1), fk = 2 * ck + ((code >> 2) & 1);
    s += kf[6 * (fi + Nf * (fj + Nf * fk)) + tf];
  }
  kc[c] = 0.125 * s;
}

__global__ void k_check_positive(const double* __restrict__ v, int n, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = v[i];
  if (!(a > 0.0) || !isfinite(a)) atomicOr(flag, 1);
}

// ----------------------------------------------------------- transfers
// Prolongation: fine lattice point L splits as L = 2k*c + o (c the coarse cube,
// o in [0,2k)^3); the class o selects a stencil of (coarse lattice point
// DEG*c + offset, weight) pairs built on the host by evaluating the coarse
// basis.  The per-level index table gives each entry's coarse dof as
// t.x + cx + t.y cy + t.z cz (affine in the cube coordinates).
template <int DEG, typename T>
__global__ void k_prolong(Numbering nf, int n_f, const int* __restrict__ start, const int4* __restrict__ tab,
                          const T* __restrict__ w, const T* __restrict__ xc, T* __restrict__ xf, int accumulate,
                          float2* __restrict__ xs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_f) return;
  int x, y, z;
  dof_to_lattice(nf, i, x, y, z);
  constexpr int K2 = 2 * DEG;
  const int cx = x / K2, cy = y / K2, cz = z / K2;
  const int cls = (x - K2 * cx) + K2 * ((y - K2 * cy) + K2 * (z - K2 * cz));
  T s = T(0);
  const int e0 = __ldg(start + cls), ne = __ldg(start + cls + 1) - e0;
  // at most 2 (P1), 10 (P2), 20 (P3) coarse dofs per fine dof: unrolled and
  // predicated, so all the gathers of a fine dof are in flight together
  constexpr int MAXE = tet_ndof(DEG) == 4 ? 2 : tet_ndof(DEG);
  // x stride of the coarse dof in the cube index: P1 and P2 (halved
  // coordinates of its class) 1, P3 (lexicographic, base point 3 c) 3
  constexpr int KP = DEG == 3 ? 3 : 1;
#pragma unroll
  for (int k = 0; k < MAXE; ++k) {
    if (k < ne) {
      const int4 t = __ldg(tab + e0 + k);
      const int j = t.x + KP * cx + t.y * cy + t.z * cz;
      s += __ldg(w + e0 + k) * __ldg(xc + j);
    }
  }
  const T v = accumulate ? xf[i] + s : s;
  xf[i] = v;
  if constexpr (sizeof(T) == 8)
    if (xs) xs[i] = fe_df::split_pair(v);  // the operator's next input, ready as a float pair
}

// P2 prolongation per coarse cube and fine row: a thread takes coarse cube
// (cx, cy, cz) and one row (OY, OZ) of the cube's fine points (4 per row, 5 in
// the last cube along x; rows OY = 4 or OZ = 4 only in the last cube along y
// or z), loads the coarse values the row needs once, and forms each fine value
// with the compile-time weights of fe_kuhn.h (pro_w8: about 3.8 terms per
// point).  The table-driven kernel above spent some 250 instructions per fine
// point on recovering lattice coordinates and classes from the dof index and
// on loading stencil entries; here the indices are affine in the cube
// coordinates (the P2 numbering is class-major by lattice parity) and the
// weights are immediates.  Blocks of 32 x 4 cubes share one row, so the row's
// template instance is chosen by a uniform branch.
// Compile-time weights (template constants, so that nothing of pro_w8 is left
// to run on the device) and the coarse nodes a row needs.
template <int OX, int OY, int OZ, int N>
struct ProW8 {
  static constexpr int v = fe_kuhn::pro_w8(OX, OY, OZ, N % 3, (N / 3) % 3, N / 9);
};
template <int OY, int OZ, int N>
struct ProNeed {
  static constexpr bool v = ProW8<0, OY, OZ, N>::v != 0 || ProW8<1, OY, OZ, N>::v != 0 ||
                            ProW8<2, OY, OZ, N>::v != 0 || ProW8<3, OY, OZ, N>::v != 0 || ProW8<4, OY, OZ, N>::v != 0;
};

__host__ __device__ constexpr int p2_class(int px, int py, int pz) {
  return (px | (py << 1) | (pz << 2)) == 3 ? 4 : ((px | (py << 1) | (pz << 2)) == 4 ? 3 : (px | (py << 1) | (pz << 2)));
}

template <int OY, int OZ, int N, typename T>
__device__ __forceinline__ void pro_load(const Numbering& nc, int cx, int cy, int cz, const T* __restrict__ xc,
                                         T (&v)[27]) {
  if constexpr (ProNeed<OY, OZ, N>::v) {
    constexpr int a = N % 3, b = (N / 3) % 3, d = N / 9, c = p2_class(a & 1, b & 1, d & 1);
    v[N] = __ldg(xc + nc.off[c] + (cx + (a >> 1)) + nc.sx[c] * ((cy + (b >> 1)) + nc.sy[c] * (cz + (d >> 1))));
  }
}
template <int OX, int OY, int OZ, int N, typename T>
__device__ __forceinline__ void pro_term(const T (&v)[27], T& s) {
  if constexpr (ProW8<OX, OY, OZ, N>::v != 0) s += T(ProW8<OX, OY, OZ, N>::v * 0.125) * v[N];
}
template <int OX, int OY, int OZ, typename T, int... N>
__device__ __forceinline__ T pro_sum(const T (&v)[27], std::integer_sequence<int, N...>) {
  T s = T(0);
  (pro_term<OX, OY, OZ, N>(v, s), ...);
  return s;
}
template <int OX, int OY, int OZ, typename T>
__device__ __forceinline__ void pro_point(const T (&v)[27], int base0, int base1, T* __restrict__ xf, int accumulate,
                                          float2* __restrict__ xs) {
  const T s = pro_sum<OX, OY, OZ, T>(v, std::make_integer_sequence<int, 27>{});
  const int i = (OX & 1 ? base1 : base0) + (OX >> 1);
  const T r = accumulate ? xf[i] + s : s;
  xf[i] = r;
  if constexpr (sizeof(T) == 8)
    if (xs) xs[i] = fe_df::split_pair(r);  // the operator's next input, ready as a float pair
}
template <int OY, int OZ, typename T, int... N>
__device__ __forceinline__ void pro_loads(const Numbering& nc, int cx, int cy, int cz, const T* __restrict__ xc,
                                          T (&v)[27], std::integer_sequence<int, N...>) {
  (pro_load<OY, OZ, N>(nc, cx, cy, cz, xc, v), ...);
}

template <int OY, int OZ, typename T>
__device__ __forceinline__ void pro_row(const Numbering& nc, const Numbering& nf, int Nc, int cx, int cy, int cz,
                                        const T* __restrict__ xc, T* __restrict__ xf, int accumulate,
                                        float2* __restrict__ xs) {
  T v[27];
  pro_loads<OY, OZ>(nc, cx, cy, cz, xc, v, std::make_integer_sequence<int, 27>{});
  // fine dofs of the row: parity class by ox & 1, the y and z parts fixed
  const int fy = 2 * cy + (OY >> 1), fz = 2 * cz + (OZ >> 1);
  constexpr int c0 = p2_class(0, OY & 1, OZ & 1), c1 = p2_class(1, OY & 1, OZ & 1);
  const int base0 = nf.off[c0] + 2 * cx + nf.sx[c0] * (fy + nf.sy[c0] * fz);
  const int base1 = nf.off[c1] + 2 * cx + nf.sx[c1] * (fy + nf.sy[c1] * fz);
  pro_point<0, OY, OZ>(v, base0, base1, xf, accumulate, xs);
  pro_point<1, OY, OZ>(v, base0, base1, xf, accumulate, xs);
  pro_point<2, OY, OZ>(v, base0, base1, xf, accumulate, xs);
  pro_point<3, OY, OZ>(v, base0, base1, xf, accumulate, xs);
  if (cx == Nc - 1) pro_point<4, OY, OZ>(v, base0, base1, xf, accumulate, xs);
}

template <int R, typename T>
__device__ __forceinline__ void pro_row_dispatch(int row, const Numbering& nc, const Numbering& nf, int Nc, int cx,
                                                 int cy, int cz, const T* xc, T* xf, int accumulate, float2* xs) {
  if (row == R)
    pro_row<R % 5, R / 5, T>(nc, nf, Nc, cx, cy, cz, xc, xf, accumulate, xs);
  else if constexpr (R + 1 < 25)
    pro_row_dispatch<R + 1, T>(row, nc, nf, Nc, cx, cy, cz, xc, xf, accumulate, xs);
}

template <typename T>
__global__ void __launch_bounds__(128) k_prolong_cube(Numbering nc, Numbering nf, int Nc, int nby,
                                                      const T* __restrict__ xc, T* __restrict__ xf, int accumulate,
                                                      float2* __restrict__ xs) {
  const int row = blockIdx.y / nby;  // uniform per block
  const int cx = blockIdx.x * 32 + threadIdx.x, cy = (blockIdx.y - row * nby) * 4 + threadIdx.y, cz = blockIdx.z;
  if (cx >= Nc || cy >= Nc) return;
  const int oy = row % 5, oz = row / 5;
  if ((oy == 4 && cy != Nc - 1) || (oz == 4 && cz != Nc - 1)) return;
  pro_row_dispatch<0, T>(row, nc, nf, Nc, cx, cy, cz, xc, xf, accumulate, xs);
}

// Restriction = exact transpose: coarse point Lc gathers fine points
// 2 Lc + o for the stencil entries of its class (Lc mod k per axis); the index
// table gives the fine dof as t.x + KX X + t.y Y + t.z Z (KX = 1 for P2, whose
// classes halve the coordinates, 2 for the lexicographic P1/P3) and the
// offset o packed in t.w, unpacked for the bounds test only by coarse points
// within `margin` of the boundary.  With yf != null the restricted vector is
// the residual bf - yf.  A block holds 32 consecutive coarse points (one per
// lane, so every gather of a warp reads consecutive fine entries of one class
// array) and TPC warps: warp w takes every TPC-th stencil entry (a P2 vertex
// gathers 125 fine points) and the partial sums meet in shared memory.
template <int DEG, typename T, int TPC>
__global__ void __launch_bounds__(32 * TPC) k_restrict(int mf, Numbering nc, int n_c, int margin,
                                                       const int* __restrict__ start, const int4* __restrict__ tab,
                                                       const T* __restrict__ w, const T* __restrict__ bf,
                                                       const T* __restrict__ yf, T* __restrict__ rc, int zero_bd) {
  __shared__ T part[TPC][32];
  constexpr int KX = DEG == 2 ? 1 : 2;
  const int lane = threadIdx.x & 31, sub = threadIdx.x >> 5;
  const int J = blockIdx.x * 32 + lane;
  T s = T(0);
  if (J < n_c) {
    int X, Y, Z;
    dof_to_lattice(nc, J, X, Y, Z);
    const int mc = nc.m;
    const bool bd = X == 0 || Y == 0 || Z == 0 || X == mc || Y == mc || Z == mc;
    if (!(bd && zero_bd)) {
      const bool near = min(min(X, Y), Z) < margin || max(max(X, Y), Z) > mc - margin;
      const int cls = DEG == 1 ? 0 : (X % DEG) + DEG * ((Y % DEG) + DEG * (Z % DEG));
      const int e1 = __ldg(start + cls + 1);
      const int base = KX * X;
#pragma unroll 2
      for (int e = __ldg(start + cls) + sub; e < e1; e += TPC) {
        const int4 t = __ldg(tab + e);
        if (near) {
          const int fx = 2 * X + (t.w & 255) - 8, fy = 2 * Y + ((t.w >> 8) & 255) - 8,
                    fz = 2 * Z + ((t.w >> 16) & 255) - 8;
          if (fx < 0 || fy < 0 || fz < 0 || fx > mf || fy > mf || fz > mf) continue;
        }
        const int i = t.x + base + t.y * Y + t.z * Z;
        T v = __ldg(bf + i);
        if (yf) v -= __ldg(yf + i);
        s += __ldg(w + e) * v;
      }
    }
  }
  part[sub][lane] = s;
  __syncthreads();
  if (sub == 0 && J < n_c) {
    T t = part[0][lane];
#pragma unroll
    for (int k = 1; k < TPC; ++k) t += part[k][lane];
    rc[J] = t;
  }
}

// --------------------------------------------------------- vector ops
// Chebyshev step: d = c1 d + c2 D^-1 (b - y); x += d  (y = A x).  With
// first_from_zero (x = 0, y unused): d = c2 D^-1 b; x = d.
template <typename T>
__global__ void k_cheb_step(int n, const T* __restrict__ b, const T* __restrict__ y, const T* __restrict__ dinv,
                            T* __restrict__ x, T* __restrict__ d, T c1, T c2, int first_from_zero, int store_d,
                            float2* __restrict__ xs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T xn;
  if (first_from_zero) {
    const T dn = c2 * dinv[i] * b[i];
    if (store_d) d[i] = dn;
    xn = dn;
  } else {
    const T dn = (c1 != T(0) ? c1 * d[i] : T(0)) + c2 * dinv[i] * (b[i] - y[i]);
    if (store_d) d[i] = dn;  // the last step of a sweep does not need d again
    xn = x[i] + dn;
  }
  x[i] = xn;
  if constexpr (sizeof(T) == 8)
    if (xs) xs[i] = fe_df::split_pair(xn);  // the operator's next input, ready as a float pair
}

// The FP64 step with two dofs per thread: 16-byte loads and stores (every
// pointer 16-byte aligned), so a warp keeps twice the bytes in flight per
// load instruction; the last thread takes the odd dof of an odd n.
__global__ void k_cheb_step2(int n, const double* __restrict__ b, const double* __restrict__ y,
                             const double* __restrict__ dinv, double* __restrict__ x, double* __restrict__ d, double c1,
                             double c2, int first_from_zero, int store_d, float2* __restrict__ xs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = 2 * t;
  if (i >= n) return;
  if (i + 1 == n) {  // the odd last dof
    double xn;
    if (first_from_zero) {
      const double dn = c2 * dinv[i] * b[i];
      if (store_d) d[i] = dn;
      xn = dn;
    } else {
      const double dn = (c1 != 0.0 ? c1 * d[i] : 0.0) + c2 * dinv[i] * (b[i] - y[i]);
      if (store_d) d[i] = dn;
      xn = x[i] + dn;
    }
    x[i] = xn;
    if (xs) xs[i] = fe_df::split_pair(xn);
    return;
  }
  const double2 bb = *reinterpret_cast<const double2*>(b + i), dd = *reinterpret_cast<const double2*>(dinv + i);
  double2 xn;
  if (first_from_zero) {
    const double2 dn = make_double2(c2 * dd.x * bb.x, c2 * dd.y * bb.y);
    if (store_d) *reinterpret_cast<double2*>(d + i) = dn;
    xn = dn;
  } else {
    const double2 yy = *reinterpret_cast<const double2*>(y + i), xo = *reinterpret_cast<const double2*>(x + i);
    const double2 dp = c1 != 0.0 ? *reinterpret_cast<const double2*>(d + i) : make_double2(0.0, 0.0);
    const double2 dn = make_double2((c1 != 0.0 ? c1 * dp.x : 0.0) + c2 * dd.x * (bb.x - yy.x),
                                    (c1 != 0.0 ? c1 * dp.y : 0.0) + c2 * dd.y * (bb.y - yy.y));
    if (store_d) *reinterpret_cast<double2*>(d + i) = dn;
    xn = make_double2(xo.x + dn.x, xo.y + dn.y);
  }
  *reinterpret_cast<double2*>(x + i) = xn;
  if (xs) {
    const float2 p0 = fe_df::split_pair(xn.x), p1 = fe_df::split_pair(xn.y);
    *reinterpret_cast<float4*>(xs + i) = make_float4(p0.x, p0.y, p1.x, p1.y);
  }
}

template <typename Ti, typename To>
__global__ void k_convert(int n, const Ti* __restrict__ in, To* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (To)in[i];
}

__global__ void k_set_boundary(int nb, const int* __restrict__ bnd, const double* __restrict__ src,
                               double* __restrict__ dst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nb) dst[bnd[t]] = src ? src[bnd[t]] : 0.0;
}

__global__ void k_random(int n, uint64_t seed, double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // splitmix64 of (seed, i) -> uniform(-1, 1)
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  v[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// Dense interior coarse operator, P3: A[ii][jj] += A_K[i][j] straight from
// the reference coefficients (the P1/P2 assembly in fe_coarse.cu applies the
// element to unit vectors).
__global__ void k_coarse_assemble_p3(int C, int Cs, const int* __restrict__ map, const double* __restrict__ geo,
                                     const int* __restrict__ dof2int, int nci, double* __restrict__ A, int band) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int ii[20];
  double g[6];
  for (int j = 0; j < 20; ++j) {
    const int m = map[(size_t)j * Cs + c];
    ii[j] = m >= 0 ? dof2int[m] : -1;
  }
  for (int a = 0; a < 6; ++a) g[a] = geo[(size_t)a * Cs + c];
  for (int i = 0; i < 20; ++i) {
    if (ii[i] < 0) continue;
    for (int j = 0; j < 20; ++j) {
      if (ii[j] < 0) continue;
      const int lo = min(i, j), hi = max(i, j);
      const int p = 20 * lo - lo * (lo - 1) / 2 + (hi - lo);
      if (band >= 0 && ii[j] > ii[i]) continue;  // band storage keeps the lower triangle
      double a = 0.0;
      for (int k = 0; k < 6; ++k) a += g[k] * c_K3[p][k];
      const size_t at = band >= 0 ? (size_t)ii[i] * (band + 1) + (ii[j] - ii[i] + band) : (size_t)ii[i] * nci + ii[j];
      atomicAdd(A + at, 161280.0 * a);  // g = kappa G / 161280
    }
  }
}

// P3 vertex-star patch: one block per vertex assembles A_p (65 x 65, shared
// memory) from the element-matrix entries of the tets around V that couple two
// dofs of V's open star (per tet: V, the 6 nodes of its 3 edges at V, the 3
// face nodes of its faces at V), gives inactive slots (outside, Dirichlet) an
// identity row, inverts A_p in place by Gauss-Jordan (SPD: no pivoting) and
// stores the packed upper triangle patch-major [P][2145] as float pairs (the
// FP64 product) and FP32 for the warp-per-patch product.
constexpr int kNS3 = 65, kNP3 = kNS3 * (kNS3 + 1) / 2;
__device__ int p3_slot_of(int dx, int dy, int dz) {
  for (int s = 0; s < kNS3; ++s)
    if (c_p3slot[s][0] == dx && c_p3slot[s][1] == dy && c_p3slot[s][2] == dz) return s;
  return -1;
}

__global__ void __launch_bounds__(128) k_patch_setup_p3(Numbering num, int P, int Cs, const double* __restrict__ geo64,
                                                        int* __restrict__ pdof, float2* __restrict__ pinvdf,
                                                        float* __restrict__ pinv32, int* __restrict__ flag) {
  __shared__ double A[kNS3][kNS3];
  __shared__ double fcol[kNS3];
  __shared__ int sdof[kNS3];
  const int v = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int N = num.N, n1 = N + 1, m = num.m;
  const int V[3] = {v % n1, (v / n1) % n1, v / (n1 * n1)};
  for (int sl = tid; sl < kNS3; sl += nt) {
    const int x = 3 * V[0] + c_p3slot[sl][0], y = 3 * V[1] + c_p3slot[sl][1], z = 3 * V[2] + c_p3slot[sl][2];
    const bool active = x > 0 && y > 0 && z > 0 && x < m && y < m && z < m;
    sdof[sl] = active ? lattice_to_dof(num, x, y, z) : -1;
    pdof[(size_t)v * kNS3 + sl] = sdof[sl];
  }
  for (int e = tid; e < kNS3 * kNS3; e += nt) A[e / kNS3][e % kNS3] = 0.0;
  __syncthreads();
  // work item: (cube around V, tet, pair of the tet's 10 star dofs)
  for (int item = tid; item < 8 * 6 * 100; item += nt) {
    const int c8 = item / 600, t = (item / 100) % 6, pr = item % 100;
    const int ox = V[0] - 1 + (c8 & 1), oy = V[1] - 1 + ((c8 >> 1) & 1), oz = V[2] - 1 + (c8 >> 2);
    if (ox < 0 || oy < 0 || oz < 0 || ox >= N || oy >= N || oz >= N) continue;
    int p0, p1, p2;
    kuhn_perm(t, p0, p1, p2);
    int w[4][3] = {{ox, oy, oz}, {ox, oy, oz}, {ox, oy, oz}, {ox + 1, oy + 1, oz + 1}};
    w[1][p0] += 1;
    w[2][p0] += 1;
    w[2][p1] += 1;
    int a = -1;
    for (int k = 0; k < 4; ++k)
      if (w[k][0] == V[0] && w[k][1] == V[1] && w[k][2] == V[2]) a = k;
    if (a < 0) continue;
    // the tet's 10 star dofs: local index and lattice offset from 3 V
    int loc[10], off[10][3], n = 0;
    loc[n] = a;
    off[n][0] = off[n][1] = off[n][2] = 0;
    ++n;
    for (int b = 0; b < 4; ++b) {
      if (b == a) continue;
      const int lo = min(a, b), hi = max(a, b), e = p2_edge(lo, hi) - 4;
      for (int h = 0; h < 2; ++h) {  // node 4 + 2e + h at (2 - h) w_lo + (1 + h) w_hi
        loc[n] = 4 + 2 * e + h;
        for (int d = 0; d < 3; ++d) off[n][d] = (2 - h) * w[lo][d] + (1 + h) * w[hi][d] - 3 * V[d];
        ++n;
      }
    }
    for (int f = 0; f < 4; ++f) {
      if (f == a) continue;
      loc[n] = 16 + f;
      for (int d = 0; d < 3; ++d)
        off[n][d] = w[p3_face_vertex(f, 0)][d] + w[p3_face_vertex(f, 1)][d] + w[p3_face_vertex(f, 2)][d] - 3 * V[d];
      ++n;
    }
    const int ii = pr / 10, jj = pr % 10;
    const int si = p3_slot_of(off[ii][0], off[ii][1], off[ii][2]), sj = p3_slot_of(off[jj][0], off[jj][1], off[jj][2]);
    if (si < 0 || sj < 0) {
      atomicOr(flag, 1);
      continue;
    }
    if (sdof[si] < 0 || sdof[sj] < 0) continue;
    const int lo = min(loc[ii], loc[jj]), hi = max(loc[ii], loc[jj]);
    const int p = 20 * lo - lo * (lo - 1) / 2 + (hi - lo);
    const int cell = 6 * (ox + N * (oy + N * oz)) + t;
    double aij = 0.0;
    for (int k = 0; k < 6; ++k) aij += geo64[(size_t)k * Cs + cell] * c_K3[p][k];
    atomicAdd(&A[si][sj], 161280.0 * aij);  // geo64 = kappa G / 161280
  }
  __syncthreads();
  for (int sl = tid; sl < kNS3; sl += nt)
    if (sdof[sl] < 0) A[sl][sl] = 1.0;
  __syncthreads();
  for (int k = 0; k < kNS3; ++k) {
    const double pk = A[k][k];
    if (!(pk > 0.0)) {  // uniform: every thread reads the same pivot
      if (tid == 0) atomicOr(flag, 2);
      return;
    }
    __syncthreads();
    for (int j = tid; j < kNS3; j += nt) A[k][j] = (j == k ? 1.0 : A[k][j]) / pk;
    for (int i = tid; i < kNS3; i += nt) fcol[i] = i == k ? 0.0 : A[i][k];
    __syncthreads();
    for (int e = tid; e < kNS3 * kNS3; e += nt) {
      const int i = e / kNS3, j = e % kNS3;
      if (i != k) A[i][j] = (j == k ? 0.0 : A[i][j]) - fcol[i] * A[k][j];
    }
    __syncthreads();
  }
  for (int i = 0; i < kNS3; ++i)
    for (int j = i + tid; j < kNS3; j += nt) {
      const int p = kNS3 * i - i * (i - 1) / 2 + (j - i);
      const double e = 0.5 * (A[i][j] + A[j][i]);
      const size_t o = (size_t)v * kNP3 + p;
      const float h = (float)e;  // P3 products use the float-pair and FP32 copies only
      pinvdf[o] = make_float2(h, (float)(e - (double)h));
      pinv32[o] = h;
    }
}

}  // namespace

// ===================================================================== host
void launch_patch_setup_p3(Level& L, cudaStream_t s) {
  static std::mutex mu;
  static std::vector<char> uploaded;  // per device: constant memory lives in each device's context
  int dev = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  std::unique_lock<std::mutex> lock(mu);
  if (dev >= (int)uploaded.size()) uploaded.resize(dev + 1, 0);
  if (!uploaded[dev]) {  // the 65 slot offsets of a Kuhn vertex star, from the six tets of the 8 cubes around it
    int tab[65][3] = {{0, 0, 0}};
    int ns = 1;
    std::vector<std::array<int, 3>> edges, faces;
    auto add = [](std::vector<std::array<int, 3>>& v, std::array<int, 3> d) {
      for (auto& x : v)
        if (x == d) return;
      v.push_back(d);
    };
    for (int c8 = 0; c8 < 8; ++c8)
      for (int t = 0; t < 6; ++t) {
        const int o[3] = {-1 + (c8 & 1), -1 + ((c8 >> 1) & 1), -1 + (c8 >> 2)};
        int p0, p1, p2;
        kuhn_perm(t, p0, p1, p2);
        int w[4][3] = {{o[0], o[1], o[2]}, {o[0], o[1], o[2]}, {o[0], o[1], o[2]}, {o[0] + 1, o[1] + 1, o[2] + 1}};
        w[1][p0] += 1;
        w[2][p0] += 1;
        w[2][p1] += 1;
        int a = -1;
        for (int k = 0; k < 4; ++k)
          if (w[k][0] == 0 && w[k][1] == 0 && w[k][2] == 0) a = k;
        if (a < 0) continue;
        for (int b = 0; b < 4; ++b)
          if (b != a) add(edges, {w[b][0], w[b][1], w[b][2]});
        for (int b = 0; b < 4; ++b)
          for (int c = b + 1; c < 4; ++c)
            if (b != a && c != a) add(faces, {w[b][0] + w[c][0], w[b][1] + w[c][1], w[b][2] + w[c][2]});
      }
    FE_REQUIRE(edges.size() == 14 && faces.size() == 36, FE_ERR_CUDA, "unexpected Kuhn vertex star");
    for (auto& d : edges) {
      for (int k = 0; k < 3; ++k) tab[ns][k] = d[k];
      ++ns;
      for (int k = 0; k < 3; ++k) tab[ns][k] = 2 * d[k];
      ++ns;
    }
    for (auto& d : faces) {
      for (int k = 0; k < 3; ++k) tab[ns][k] = d[k];
      ++ns;
    }
    CUDA_CHECK(cudaMemcpyToSymbol(c_p3slot, tab, sizeof(tab)));
    uploaded[dev] = 1;
  }
  lock.unlock();
  const int P = L.V;
  if (L.pdof.n != (size_t)kNS3 * P) {
    L.pdof.alloc((size_t)kNS3 * P);
    L.pinvdf.alloc((size_t)kNP3 * P);
    L.pinv32.alloc((size_t)kNP3 * P);
  }
  DBuf<int> flag;
  flag.alloc(1);
  CUDA_CHECK(cudaMemsetAsync(flag, 0, sizeof(int), s));
  k_patch_setup_p3<<<P, 128, 0, s>>>(L.num, P, L.Cs, L.geo64, L.pdof, L.pinvdf, L.pinv32, flag);
  LAUNCH_CHECK();
  int hflag = 0;
  CUDA_CHECK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  FE_REQUIRE(hflag == 0, FE_ERR_CUDA, "P3 patch setup failed (non-positive pivot or unknown star node)");
}

void launch_coarse_assemble_p3(const Level& L0, const int* dof2int, int nci, double* A, int band, cudaStream_t s) {
  k_coarse_assemble_p3<<<ceil_div(L0.C, kBlock), kBlock, 0, s>>>(L0.C, L0.Cs, L0.map, L0.geo64, dof2int, nci, A,
                                                                 band);
  LAUNCH_CHECK();
}

// Calls f with std::integral_constant<int, deg> for deg = 1, 2, 3.
template <class F>
static void by_degree(int deg, F&& f) {
  if (deg == 1)
    f(std::integral_constant<int, 1>{});
  else if (deg == 2)
    f(std::integral_constant<int, 2>{});
  else
    f(std::integral_constant<int, 3>{});
}

void launch_build_level(Level& L, cudaStream_t s) {
  by_degree(L.deg, [&](auto D) {
    k_build_map<D.value><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.num, L.C, L.Cs, L.map);
    LAUNCH_CHECK();
    k_build_cube_map<D.value><<<ceil_div(L.Q, kBlock), kBlock, 0, s>>>(L.num, L.Q, L.Qs, L.cmap);
    LAUNCH_CHECK();
  });
  if (L.deg == 3)  // coordinates of every lattice point, indexed by dof (the vertices' dofs are not 0..V-1)
    k_build_coords_lattice<<<ceil_div(L.n, kBlock), kBlock, 0, s>>>(L.num, L.n, L.vx, L.vy, L.vz);
  else
    k_build_coords<<<ceil_div(L.V, kBlock), kBlock, 0, s>>>(L.N, L.V, L.vx, L.vy, L.vz);
  LAUNCH_CHECK();
}

void launch_uniform_geometry(Level& L, int* dflag, cudaStream_t s) {
  if (!L.c32.p) {  // rows of Cs (a multiple of 128 cells): the tensor-core operator stages c32 by TMA tiles
    L.c32.alloc(L.Cs);
    L.cdf.alloc(L.Cs);
  }
  CUDA_CHECK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
  k_uniform_geometry<<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.geo64, L.c32, L.cdf, dflag);
  LAUNCH_CHECK();
  int hflag = 1;
  CUDA_CHECK(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  L.uniform = (hflag & 1) == 0 ? 1 : 0;
  L.pair_uniform = hflag == 0 ? 1 : 0;
}

void launch_geometry(Level& L, cudaStream_t s) {
  by_degree(L.deg, [&](auto D) {
    k_geometry<D.value><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.vx, L.vy, L.vz, L.kappa, L.geo64,
                                                                L.geo32, L.detj);
  });
  LAUNCH_CHECK();
}

template <typename T>
static void apply_impl(const Level& L, const T* geo, const T* x, T* y, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)L.n, s));
  const int Cpad = ceil_div(L.C, kBlock) * kBlock;
  const int grid = ceil_div((long long)Cpad + L.nb, kBlock);
  by_degree(L.deg, [&](auto D) {
    if (L.uniform)
      k_apply<D.value, T, true><<<grid, kBlock, 0, s>>>(L.C, L.Cs, Cpad, L.map, geo, x, y, L.nb, L.bnd);
    else
      k_apply<D.value, T, false><<<grid, kBlock, 0, s>>>(L.C, L.Cs, Cpad, L.map, geo, x, y, L.nb, L.bnd);
  });
  LAUNCH_CHECK();
}

template <bool FUSE>
static void apply_cube32(const Level& L, const float* x, float* y, const ChebFuse<float>& cf, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(float) * (size_t)L.n, s));
  const int Qpad = ceil_div(L.Q, kCubeBlock) * kCubeBlock;
  const int grid = ceil_div((long long)Qpad + L.nb, kCubeBlock);
  // c32 rows start at multiples of 24 bytes per cube: the UNI kernel's float2 loads stay 8-byte aligned
  if (L.deg == 1 && L.uniform)
    k_apply_cube<1, FUSE, true><<<grid, kCubeBlock, 0, s>>>(L.Q, L.Qs, L.Cs, Qpad, L.cmap, L.c32, x, y, L.nb, L.bnd, cf);
  else if (L.deg == 1)
    k_apply_cube<1, FUSE, false><<<grid, kCubeBlock, 0, s>>>(L.Q, L.Qs, L.Cs, Qpad, L.cmap, L.geo32, x, y, L.nb, L.bnd,
                                                             cf);
  else if (L.uniform && !FUSE) {
    static int g2 = 0;
    if (!g2) g2 = resident_grid(k_apply_cube_lp32<2>, kCubeLpBlock, 1 << 30);
    k_apply_cube_lp32<2><<<std::min(g2, ceil_div(std::max(L.Q, L.nb), kCubeLpBlock)), kCubeLpBlock, 0, s>>>(
        L.Q, L.Qs, L.Cs, L.cmap, L.c32, x, y, L.nb, L.bnd);
  } else if (L.uniform)
    k_apply_cube<2, FUSE, true><<<grid, kCubeBlock, 0, s>>>(L.Q, L.Qs, L.Cs, Qpad, L.cmap, L.c32, x, y, L.nb, L.bnd, cf);
  else
    k_apply_cube<2, FUSE, false><<<grid, kCubeBlock, 0, s>>>(L.Q, L.Qs, L.Cs, Qpad, L.cmap, L.geo32, x, y, L.nb, L.bnd,
                                                             cf);
  LAUNCH_CHECK();
}

void launch_apply_cheb32(const Level& L, const float* b, float* x, float* y, float* d, double c1, double c2,
                         bool store_d, cudaStream_t s) {
  const ChebFuse<float> cf{b, L.dinv32, x, d, L.val_cube, L.cnt_cube, (float)c1, (float)c2, store_d ? 1 : 0};
  apply_cube32<true>(L, x, y, cf, s);
}

void launch_build_valence(Level& L, cudaStream_t s) {
  L.val_tet.alloc(L.n);
  L.cnt_tet.alloc(L.n);
  L.val_cube.alloc(L.n);
  L.cnt_cube.alloc(L.n);
  CUDA_CHECK(cudaMemsetAsync(L.val_tet, 0, sizeof(unsigned) * (size_t)L.n, s));
  CUDA_CHECK(cudaMemsetAsync(L.val_cube, 0, sizeof(unsigned) * (size_t)L.n, s));
  k_valence<<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.nd, L.map, L.val_tet);
  LAUNCH_CHECK();
  const int K = L.deg + 1;
  k_valence<<<ceil_div(L.Q, kBlock), kBlock, 0, s>>>(L.Q, L.Qs, K * K * K, L.cmap, L.val_cube);
  LAUNCH_CHECK();
  CUDA_CHECK(cudaMemcpyAsync(L.cnt_tet, L.val_tet, sizeof(unsigned) * (size_t)L.n, cudaMemcpyDeviceToDevice, s));
  CUDA_CHECK(cudaMemcpyAsync(L.cnt_cube, L.val_cube, sizeof(unsigned) * (size_t)L.n, cudaMemcpyDeviceToDevice, s));
}

void launch_apply64(const Level& L, const double* x, double* y, cudaStream_t s) { apply_impl<double>(L, L.geo64, x, y, s); }
void launch_apply32(const Level& L, const float* x, float* y, cudaStream_t s) {
  if (L.deg == 3)  // P3: one thread per tet (a P3 cube holds 64 dofs and 6 x 20 x 20 products)
    apply_impl<float>(L, L.geo32, x, y, s);
  else
    apply_cube32<false>(L, x, y, ChebFuse<float>{}, s);
}

void launch_mass(const Level& L, const double* x, double* y, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)L.n, s));
  by_degree(L.deg, [&](auto D) {
    k_mass<D.value><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.detj, x, y);
  });
  LAUNCH_CHECK();
}

void launch_diag(Level& L, double* diag, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(diag, 0, sizeof(double) * (size_t)L.n, s));
  by_degree(L.deg, [&](auto D) {
    k_diag<D.value><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.geo64, diag);
  });
  LAUNCH_CHECK();
  if (L.nb > 0) {
    k_diag_finish<<<ceil_div(L.nb, kBlock), kBlock, 0, s>>>(L.n, L.nb, L.bnd, diag);
    LAUNCH_CHECK();
  }
  k_invert<<<ceil_div(L.n, kBlock), kBlock, 0, s>>>(L.n, diag, L.dinv64, L.dinv32);
  LAUNCH_CHECK();
}

void launch_gradient(const Level& L, const double* u, const double* lam, double* g, cudaStream_t s) {
  by_degree(L.deg, [&](auto D) {
    k_gradient<D.value><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.vx, L.vy, L.vz, u, lam, g);
  });
  LAUNCH_CHECK();
}

void launch_dof_coords(const Level& L, double* xyz, cudaStream_t s) {
  k_dof_coords<<<ceil_div(L.n, kBlock), kBlock, 0, s>>>(L.num, L.n, xyz);
  LAUNCH_CHECK();
}

void launch_centroids(const Level& L, double* xyz, cudaStream_t s) {
  k_centroids<<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.vx, L.vy, L.vz, xyz);
  LAUNCH_CHECK();
}

void launch_bmask(const Level& L, unsigned char* m, cudaStream_t s) {
  k_bmask<<<ceil_div(L.n, kBlock), kBlock, 0, s>>>(L.num, L.n, m);
  LAUNCH_CHECK();
}

void launch_coarsen_kappa(const Level& Lc, const Level& Lf, const int* children, cudaStream_t s) {
  k_coarsen_kappa<<<ceil_div(Lc.C, kBlock), kBlock, 0, s>>>(Lc.N, Lc.C, children, Lf.kappa, Lc.kappa);
  LAUNCH_CHECK();
}

int launch_check_positive(const double* v, int n, int* dflag, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
  k_check_positive<<<ceil_div(n, kBlock), kBlock, 0, s>>>(v, n, dflag);
  LAUNCH_CHECK();
  int hflag = 0;
  CUDA_CHECK(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  return hflag;
}

// Stencil weights in the precision of the vectors (exact in both).
template <typename T>
static const T* tt_weights(const DBuf<double>& wd, const DBuf<float>& wf);
template <>
const double* tt_weights<double>(const DBuf<double>& wd, const DBuf<float>&) { return wd.p; }
template <>
const float* tt_weights<float>(const DBuf<double>&, const DBuf<float>& wf) { return wf.p; }

template <typename T>
void launch_prolong(const fe_hierarchy* h, int lf, const T* xc, T* xf, bool accumulate, cudaStream_t s, float2* xs) {
  const Level& F = h->L[lf];
  const TransferTables& t = h->tt;
  // the per-cube kernel's blocks span 32 cubes along x: on coarse levels with
  // fewer cubes the table-driven kernel keeps every lane busy (P2 16^3 -> 32^3:
  // 10.5 against 12.5 us; 32^3 -> 64^3: 48.8 against 31.1 us)
  if (h->deg == 2 && h->L[lf - 1].N >= 32) {
    const Level& Cl = h->L[lf - 1];
    const int Nc = Cl.N, nby = ceil_div(Nc, 4);
    const dim3 grid(ceil_div(Nc, 32), nby * 25, Nc), block(32, 4);
    k_prolong_cube<T><<<grid, block, 0, s>>>(Cl.num, F.num, Nc, nby, xc, xf, accumulate, xs);
    LAUNCH_CHECK();
    return;
  }
  by_degree(h->deg, [&](auto D) {
    k_prolong<D.value, T><<<ceil_div(F.n, kBlock), kBlock, 0, s>>>(F.num, F.n, t.pro_start, F.ptab,
                                                                  tt_weights<T>(t.pro_w, t.pro_wf), xc, xf, accumulate,
                                                                  xs);
  });
  LAUNCH_CHECK();
}

// Coarse levels below this many dofs restrict with 32 warps per 32 coarse
// points instead of 8: with fewer blocks than SMs there, a P2 vertex's 125
// entries in chains of 16 per thread left them latency-bound (P2 16^3 -> 8^3,
// 4,913 coarse dofs: 16.5 -> 9.1 us).  At 35,937 coarse dofs (32^3 -> 16^3)
// the 1024-thread blocks were slower (14.0 -> 18.5 us).
constexpr int kRestrictWideBelow = 1 << 14;

template <typename T>
void launch_restrict(const fe_hierarchy* h, int lf, const T* bf, const T* yf, T* rc, bool zero_bd, cudaStream_t s) {
  const Level& F = h->L[lf];
  const Level& Cc = h->L[lf - 1];
  const TransferTables& t = h->tt;
  if (h->deg == 1)
    k_restrict<1, T, 4><<<ceil_div(Cc.n, 32), 32 * 4, 0, s>>>(F.num.m, Cc.num, Cc.n, t.res_margin, t.res_start,
                                                              F.rtab, tt_weights<T>(t.res_w, t.res_wf), bf,
                                                              yf, rc, zero_bd);
  else if (h->deg == 2 && Cc.n < kRestrictWideBelow)
    k_restrict<2, T, 32><<<ceil_div(Cc.n, 32), 32 * 32, 0, s>>>(F.num.m, Cc.num, Cc.n, t.res_margin, t.res_start,
                                                                F.rtab, tt_weights<T>(t.res_w, t.res_wf), bf,
                                                                yf, rc, zero_bd);
  else if (h->deg == 2)
    k_restrict<2, T, 8><<<ceil_div(Cc.n, 32), 32 * 8, 0, s>>>(F.num.m, Cc.num, Cc.n, t.res_margin, t.res_start,
                                                              F.rtab, tt_weights<T>(t.res_w, t.res_wf), bf,
                                                              yf, rc, zero_bd);
  else
    k_restrict<3, T, 8><<<ceil_div(Cc.n, 32), 32 * 8, 0, s>>>(F.num.m, Cc.num, Cc.n, t.res_margin, t.res_start,
                                                              F.rtab, tt_weights<T>(t.res_w, t.res_wf), bf,
                                                              yf, rc, zero_bd);
  LAUNCH_CHECK();
}

template void launch_prolong<double>(const fe_hierarchy*, int, const double*, double*, bool, cudaStream_t, float2*);
template void launch_prolong<float>(const fe_hierarchy*, int, const float*, float*, bool, cudaStream_t, float2*);
template void launch_restrict<double>(const fe_hierarchy*, int, const double*, const double*, double*, bool,
                                      cudaStream_t);
template void launch_restrict<float>(const fe_hierarchy*, int, const float*, const float*, float*, bool, cudaStream_t);

template <typename T>
void launch_cheb_step(int n, const T* b, const T* y, const T* dinv, T* x, T* d, double c1, double c2,
                      bool first_from_zero, cudaStream_t s, bool store_d, float2* xs) {
  if constexpr (sizeof(T) == 8) {
    auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (a16(b) && a16(y) && a16(dinv) && a16(x) && a16(d) && a16(xs)) {  // null pointers count as aligned
      k_cheb_step2<<<ceil_div(ceil_div(n, 2), kBlock), kBlock, 0, s>>>(n, (const double*)b, (const double*)y,
                                                                      (const double*)dinv, (double*)x, (double*)d, c1,
                                                                      c2, first_from_zero ? 1 : 0, store_d ? 1 : 0, xs);
      LAUNCH_CHECK();
      return;
    }
  }
  k_cheb_step<T><<<ceil_div(n, kBlock), kBlock, 0, s>>>(n, b, y, dinv, x, d, (T)c1, (T)c2, first_from_zero ? 1 : 0,
                                                        store_d ? 1 : 0, xs);
  LAUNCH_CHECK();
}
template void launch_cheb_step<double>(int, const double*, const double*, const double*, double*, double*, double,
                                       double, bool, cudaStream_t, bool, float2*);
template void launch_cheb_step<float>(int, const float*, const float*, const float*, float*, float*, double, double,
                                      bool, cudaStream_t, bool, float2*);

template <typename Ti, typename To>
void launch_convert(int n, const Ti* in, To* out, cudaStream_t s) {
  k_convert<Ti, To><<<ceil_div(n, kBlock), kBlock, 0, s>>>(n, in, out);
  LAUNCH_CHECK();
}
template void launch_convert<double, float>(int, const double*, float*, cudaStream_t);
template void launch_convert<float, double>(int, const float*, double*, cudaStream_t);

void launch_set_boundary(const Level& L, const double* src, double* dst, cudaStream_t s) {
  if (L.nb == 0) return;
  k_set_boundary<<<ceil_div(L.nb, kBlock), kBlock, 0, s>>>(L.nb, L.bnd, src, dst);
  LAUNCH_CHECK();
}

void launch_zero_boundary64(const Level& L, double* v, cudaStream_t s) { launch_set_boundary(L, nullptr, v, s); }

void launch_bc_lift(const Level& L, const double* g, double* b, cudaStream_t s) {
  by_degree(L.deg, [&](auto D) {
    k_bc_lift<D.value><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.geo64, g, b);
  });
  LAUNCH_CHECK();
  launch_set_boundary(L, g, b, s);
}

void launch_random(int n, uint64_t seed, double* v, cudaStream_t s) {
  k_random<<<ceil_div(n, kBlock), kBlock, 0, s>>>(n, seed, v);
  LAUNCH_CHECK();
}

// ------------------------------------------------------- reference tables
// (host code in fe_reftables.h)
void upload_mass_tables() {
  double m1[16], m2[100];
  fe_ref::mass_tables(m1, m2);
  CUDA_CHECK(cudaMemcpyToSymbol(c_mref1, m1, sizeof(m1)));
  CUDA_CHECK(cudaMemcpyToSymbol(c_mref2, m2, sizeof(m2)));
  static double K3[210][6], M3[400];
  fe_ref::p3_tables(K3, M3);
  CUDA_CHECK(cudaMemcpyToSymbol(c_K3, K3, sizeof(K3)));
  CUDA_CHECK(cudaMemcpyToSymbol(c_mref3, M3, sizeof(M3)));
  // the P3 mass entries are integers over 26880: exact FP32 copies for the float-pair mass kernel
  static float M3i[400];
  for (int i = 0; i < 400; ++i) {
    const double v = M3[i] * 26880.0, r = std::nearbyint(v);
    FE_REQUIRE(std::fabs(v - r) < 1e-8 && std::fabs(r) < 4096, FE_ERR_CUDA, "P3 mass entries are not k/26880");
    M3i[i] = (float)r;
  }
  upload_p3_mass_table(M3i);
  double xi[FE_QUAD_POINTS][3], w[FE_QUAD_POINTS], p1[FE_QUAD_POINTS][4], p2[FE_QUAD_POINTS][10];
  double p3[FE_QUAD_POINTS][20];
  fe_ref::quad_tables(xi, w, p1, p2, p3);
  CUDA_CHECK(cudaMemcpyToSymbol(c_qxi, xi, sizeof(xi)));
  CUDA_CHECK(cudaMemcpyToSymbol(c_qw, w, sizeof(w)));
  CUDA_CHECK(cudaMemcpyToSymbol(c_qphi1, p1, sizeof(p1)));
  CUDA_CHECK(cudaMemcpyToSymbol(c_qphi2, p2, sizeof(p2)));
  CUDA_CHECK(cudaMemcpyToSymbol(c_qphi3, p3, sizeof(p3)));
}

void launch_quad_points(const Level& L, double* xyz, cudaStream_t s) {
  k_quad_points<<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.vx, L.vy, L.vz, xyz);
  LAUNCH_CHECK();
}

void launch_load_quadrature(const Level& L, const double* fq, double* b, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(b, 0, sizeof(double) * (size_t)L.n, s));
  by_degree(L.deg, [&](auto D) {
    k_load_quad<D.value><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.detj, fq, b);
  });
  LAUNCH_CHECK();
}

namespace {
__global__ void k_fill64(size_t n, double v, double* __restrict__ p) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}
}  // namespace

void launch_fill64(size_t n, double v, double* p, cudaStream_t s) {
  k_fill64<<<1024, 256, 0, s>>>(n, v, p);
  LAUNCH_CHECK();
}
