// Vertex-star patch preconditioner for the Chebyshev smoother (the paper's
// PatchPC with star patches around vertices and exact local solves, combined
// additively; Section 3, the level-smoother options of the Poisson solver).
//
// For P2 the open star of a vertex V holds V's dof and the midpoints of the 14
// Kuhn edges at V (directions +-e_x, +-e_y, +-e_z, +-(e_x+e_y), +-(e_x+e_z),
// +-(e_y+e_z), +-(1,1,1)); Dirichlet dofs are left out.  Every patch has these
// 15 slots (a slot outside the domain or on its boundary is inactive), so the
// patch data is uniform: slot dofs [15][Pp] and the packed upper triangle of
// A_p^-1 [120][Pp], one column per vertex (a warp reads consecutive entries;
// the float-pair copy holds entries 2k and 2k+1 together in [60][Pp] float4).
// A_p is assembled from the element matrices of the 24 (fewer at the
// boundary) tets around V and inverted once per coefficient; an inactive slot
// gets an identity row so that A_p stays invertible and its r and z stay 0.
// M^-1 r = sum_p R_p^T A_p^-1 R_p r is one thread per patch (gather r = b - y,
// 120-entry symmetric product, atomic scatter); Dirichlet rows take z = r.
// The FP64 product runs in float pairs (k_patch_apply_df) unless the
// hierarchy's FP64 mode is native.  P3 stars hold 65 dofs (the vertex, the 2
// nodes of each of its 14 edges, its 36 face centroids): a block per patch
// builds A_p^-1 (k_patch_setup_p3, fe_kernels.cu) and a warp per patch applies
// it (k_patch_apply_p3).
#include "fe_df.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int NS = 15;                     // slots per P2 patch
constexpr int NP = NS * (NS + 1) / 2;      // packed upper triangle
__constant__ int c_pdir[NS][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1}, {1, 1, 0},   {-1, -1, 0}, {1, 0, 1},
                                  {-1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {1, 1, 1},   {-1, -1, -1}};

__device__ int slot_of(int dx, int dy, int dz) {
  for (int s = 0; s < NS; ++s)
    if (c_pdir[s][0] == dx && c_pdir[s][1] == dy && c_pdir[s][2] == dz) return s;
  return -1;
}

__global__ void k_patch_setup(Numbering num, int P, int Pp, int Cs, const double* __restrict__ geo64,
                              int* __restrict__ pdof, double* __restrict__ pinv, float2* __restrict__ pinvdf,
                              float* __restrict__ pinv32, int* __restrict__ flag) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= P) return;
  const int N = num.N, n1 = N + 1, m = num.m;
  const int V[3] = {v % n1, (v / n1) % n1, v / (n1 * n1)};
  int dof[NS];
  for (int s = 0; s < NS; ++s) {
    const int x = 2 * V[0] + c_pdir[s][0], y = 2 * V[1] + c_pdir[s][1], z = 2 * V[2] + c_pdir[s][2];
    const bool active = x > 0 && y > 0 && z > 0 && x < m && y < m && z < m;  // inside, not Dirichlet
    dof[s] = active ? lattice_to_dof(num, x, y, z) : -1;
    pdof[(size_t)s * Pp + v] = dof[s];
  }
  double A[NS * NS];
  for (int i = 0; i < NS * NS; ++i) A[i] = 0.0;
  for (int oz = V[2] - 1; oz <= V[2]; ++oz)
    for (int oy = V[1] - 1; oy <= V[1]; ++oy)
      for (int ox = V[0] - 1; ox <= V[0]; ++ox) {
        if (ox < 0 || oy < 0 || oz < 0 || ox >= N || oy >= N || oz >= N) continue;
        const int q = ox + N * (oy + N * oz);
        for (int t = 0; t < 6; ++t) {
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
          const int c = 6 * q + t;
          double g[6];
          for (int k = 0; k < 6; ++k) g[k] = geo64[(size_t)k * Cs + c];
          // the tet's dofs in V's open star: V itself and the midpoints of its 3 edges at V
          int loc[4], slot[4];
          loc[0] = a;
          slot[0] = 0;
          for (int b = 0, r = 1; b < 4; ++b) {
            if (b == a) continue;
            loc[r] = p2_edge(a, b);
            slot[r] = slot_of(w[b][0] - V[0], w[b][1] - V[1], w[b][2] - V[2]);
            ++r;
          }
          for (int r = 0; r < 4; ++r) {
            if (slot[r] < 0) {
              atomicOr(flag, 1);  // an edge direction outside the Kuhn set: never happens on this mesh
              continue;
            }
            double u[10], out[10];
            for (int j = 0; j < 10; ++j) u[j] = j == loc[r] ? 1.0 : 0.0;
            element_apply<2, double>(u, g, out);  // column loc[r] of the element matrix
            for (int r2 = 0; r2 < 4; ++r2)
              if (slot[r2] >= 0 && dof[slot[r2]] >= 0 && dof[slot[r]] >= 0) A[slot[r2] * NS + slot[r]] += out[loc[r2]];
          }
        }
      }
  for (int s = 0; s < NS; ++s)
    if (dof[s] < 0) A[s * NS + s] = 1.0;
  // Gauss-Jordan inverse (A is symmetric positive definite: no pivoting needed)
  double B[NS * NS];
  for (int i = 0; i < NS * NS; ++i) B[i] = (i % (NS + 1) == 0) ? 1.0 : 0.0;
  for (int k = 0; k < NS; ++k) {
    const double piv = A[k * NS + k];
    if (!(piv > 0.0)) {
      atomicOr(flag, 2);
      return;
    }
    const double ip = 1.0 / piv;
    for (int j = 0; j < NS; ++j) {
      A[k * NS + j] *= ip;
      B[k * NS + j] *= ip;
    }
    for (int i = 0; i < NS; ++i) {
      if (i == k) continue;
      const double f = A[i * NS + k];
      if (f == 0.0) continue;
      for (int j = 0; j < NS; ++j) {
        A[i * NS + j] -= f * A[k * NS + j];
        B[i * NS + j] -= f * B[k * NS + j];
      }
    }
  }
  for (int i = 0, p = 0; i < NS; ++i)
    for (int j = i; j < NS; ++j, ++p) {
      const double e = 0.5 * (B[i * NS + j] + B[j * NS + i]);  // symmetric up to rounding
      pinv[(size_t)p * Pp + v] = e;
      const float hi = (float)e;
      // float pairs of entries 2k and 2k+1 share one 16-byte slot [k][Pp] (one float4 load)
      pinvdf[((size_t)(p >> 1) * Pp + v) * 2 + (p & 1)] = make_float2(hi, (float)(e - (double)hi));
      pinv32[(size_t)p * Pp + v] = hi;
    }
}

// z += sum_p R_p^T A_p^-1 R_p (b - y) (y may be null: r = b); threads past the
// last patch set z = b - y on the Dirichlet dofs.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_patch_apply(int P, int Pp, int Ppad, const int* __restrict__ pdof,
                                                        const T* __restrict__ pinv, const T* __restrict__ b,
                                                        const T* __restrict__ y, T* __restrict__ z, int nb,
                                                        const int* __restrict__ bnd) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < P) {
    int dof[NS];
    T r[NS], zz[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      dof[s] = __ldg(pdof + (size_t)s * Pp + v);
      r[s] = dof[s] >= 0 ? __ldg(b + dof[s]) - (y ? __ldg(y + dof[s]) : T(0)) : T(0);
      zz[s] = T(0);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int j = i; j < NS; ++j) {
        const int p = NS * i - i * (i - 1) / 2 + (j - i);
        const T a = __ldg(pinv + (size_t)p * Pp + v);
        zz[i] += a * r[j];
        if (j != i) zz[j] += a * r[i];
      }
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (dof[s] >= 0) atomicAdd(z + dof[s], zz[s]);
  } else if (v >= Ppad && v - Ppad < nb) {
    const int i = bnd[v - Ppad];
    z[i] = b[i] - (y ? y[i] : T(0));
  }
}

// The FP64 product in float pairs on the FP32 pipes (as the operator): the
// residual r = b - y (FP64) is scaled by the patch's largest power of two and
// split, A_p^-1 is read as (hi, lo) pairs, and z is widened back per slot.
__global__ void __launch_bounds__(kBlock) k_patch_apply_df(int P, int Pp, int Ppad, const int* __restrict__ pdof,
                                                           const float4* __restrict__ pinv, const double* __restrict__ b,
                                                           const double* __restrict__ y, double* __restrict__ z,
                                                           int nb, const int* __restrict__ bnd) {
  using namespace fe_df;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < P) {
    int dof[NS];
    double rd[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      dof[s] = __ldg(pdof + (size_t)s * Pp + v);
      rd[s] = dof[s] >= 0 ? __ldg(b + dof[s]) - (y ? __ldg(y + dof[s]) : 0.0) : 0.0;
    }
    const int emax = block_exponent<NS>(rd);
    DF r[NS], zz[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      r[s] = split_scaled(rd[s], emax);
      zz[s] = DF(0.0f);
    }
    if (emax == 0x7FF) r[0] = DF(__int_as_float(0x7fc00000), 0.0f);  // propagate NaN/inf residuals
    float4 e;
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int j = i; j < NS; ++j) {
        const int p = NS * i - i * (i - 1) / 2 + (j - i);
        if ((p & 1) == 0) e = __ldg(pinv + (size_t)(p >> 1) * Pp + v);
        const DF a = (p & 1) ? DF(e.z, e.w) : DF(e.x, e.y);
        zz[i] = zz[i] + mul(a, r[j]);
        if (j != i) zz[j] = zz[j] + mul(a, r[i]);
      }
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (dof[s] >= 0) atomicAdd(z + dof[s], widen_scaled(zz[s].hi, emax) + widen_scaled(zz[s].lo, emax));
  } else if (v >= Ppad && v - Ppad < nb) {
    const int i = bnd[v - Ppad];
    z[i] = b[i] - (y ? y[i] : 0.0);
  }
}

// P3 (65 slots, packed inverse patch-major [P][2145]): one warp per patch.  Each
// lane owns rows lane, lane + 32 and lane + 64 (< 65); r = b - y is split into
// float pairs with the warp's largest exponent and shared through shared
// memory; z_i = sum_j (A_p^-1)_ij r_j reads the packed upper triangle, whose
// 17 KB per patch the warp streams through L1.  T = double: float-pair
// arithmetic; T = float: FP32 with the FP32 copy.
constexpr int NS3 = 65, NP3 = NS3 * (NS3 + 1) / 2, kWarpsP3 = 4;
template <typename T>
__global__ void __launch_bounds__(32 * kWarpsP3) k_patch_apply_p3(int P, const int* __restrict__ pdof,
                                                                  const float2* __restrict__ pinvdf,
                                                                  const float* __restrict__ pinv32,
                                                                  const T* __restrict__ b, const T* __restrict__ y,
                                                                  T* __restrict__ z, int nb,
                                                                  const int* __restrict__ bnd) {
  using namespace fe_df;
  __shared__ float2 rs[kWarpsP3][NS3];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int v = blockIdx.x * kWarpsP3 + wib;
  // Dirichlet rows: z = r (a grid-stride loop over all threads)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int k = bnd[i];
    z[k] = b[k] - (y ? y[k] : T(0));
  }
  if (v >= P) return;
  int dof[3];
  T rr[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int sl = lane + 32 * q;
    dof[q] = sl < NS3 ? __ldg(pdof + (size_t)v * NS3 + sl) : -1;
    rr[q] = dof[q] >= 0 ? __ldg(b + dof[q]) - (y ? __ldg(y + dof[q]) : T(0)) : T(0);
  }
  int emax = 0;
  if constexpr (sizeof(T) == 8) {
    emax = block_exponent<3>(rr);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int sl = lane + 32 * q;
    if (sl < NS3) {
      if constexpr (sizeof(T) == 8) {
        DF d = split_scaled((double)rr[q], emax);
        if (q == 0 && lane == 0 && emax == 0x7FF) d = DF(__int_as_float(0x7fc00000), 0.0f);
        rs[wib][sl] = make_float2(d.hi, d.lo);
      } else {
        rs[wib][sl] = make_float2((float)rr[q], 0.0f);
      }
    }
  }
  __syncwarp();
  const size_t base = (size_t)v * NP3;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int i = lane + 32 * q;
    if (i >= NS3) continue;
    if constexpr (sizeof(T) == 8) {
      DF acc(0.0f);
#pragma unroll 5  // loads issued ahead of the dependent float-pair chain: 3.5% faster than a rolled loop
      for (int j = 0; j < NS3; ++j) {
        const int lo = min(i, j), hi = max(i, j);
        const float2 e = __ldg(pinvdf + base + NS3 * lo - lo * (lo - 1) / 2 + (hi - lo));
        const float2 r = rs[wib][j];
        acc = acc + mul(DF(e.x, e.y), DF(r.x, r.y));
      }
      if (dof[q] >= 0) atomicAdd(z + dof[q], (T)(widen_scaled(acc.hi, emax) + widen_scaled(acc.lo, emax)));
    } else {
      float acc = 0.0f;
      for (int j = 0; j < NS3; ++j) {
        const int lo = min(i, j), hi = max(i, j);
        acc += __ldg(pinv32 + base + NS3 * lo - lo * (lo - 1) / 2 + (hi - lo)) * rs[wib][j].x;
      }
      if (dof[q] >= 0) atomicAdd(z + dof[q], (T)acc);
    }
  }
}

// Chebyshev step with a preconditioned residual z: d = c1 d + c2 z, x += d
// (first_from_zero: x = d = c2 z).
template <typename T>
__global__ void k_cheb_pc(int n, const T* __restrict__ z, T* __restrict__ x, T* __restrict__ d, T c1, T c2,
                          int first_from_zero, int store_d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T dn = (c1 != T(0) && !first_from_zero ? c1 * d[i] : T(0)) + c2 * z[i];
  if (store_d) d[i] = dn;
  x[i] = first_from_zero ? dn : x[i] + dn;
}

template <typename T>
const T* patch_inv(const Level& L);
template <>
const double* patch_inv<double>(const Level& L) { return L.pinv; }
template <>
const float* patch_inv<float>(const Level& L) { return L.pinv32; }

}  // namespace

void launch_patch_setup(Level& L, cudaStream_t s) {
  if (L.deg == 3) {
    launch_patch_setup_p3(L, s);
    return;
  }
  FE_REQUIRE(L.deg == 2, FE_ERR_UNSUPPORTED, "the GPU patch setup is for P2/P3 (P1 patches are Jacobi)");
  const int P = L.V, Pp = (P + 127) / 128 * 128;
  if (L.pdof.n != (size_t)NS * Pp) {
    L.pdof.alloc((size_t)NS * Pp);
    L.pinv.alloc((size_t)NP * Pp);
    L.pinvdf.alloc((size_t)NP * Pp);
    L.pinv32.alloc((size_t)NP * Pp);
  }
  DBuf<int> flag;
  flag.alloc(1);
  CUDA_CHECK(cudaMemsetAsync(flag, 0, sizeof(int), s));
  k_patch_setup<<<ceil_div(P, 128), 128, 0, s>>>(L.num, P, Pp, L.Cs, L.geo64, L.pdof, L.pinv, L.pinvdf, L.pinv32,
                                                  flag);
  LAUNCH_CHECK();
  int hflag = 0;
  CUDA_CHECK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  FE_REQUIRE(hflag == 0, FE_ERR_CUDA, "patch setup failed (non-positive pivot or unknown edge direction)");
}

template <typename T>
void launch_patch_apply(const Level& L, const T* b, const T* y, T* z, bool df, cudaStream_t s) {
  const int P = L.V, Pp = (P + 127) / 128 * 128, Ppad = ceil_div(P, kBlock) * kBlock;
  CUDA_CHECK(cudaMemsetAsync(z, 0, sizeof(T) * (size_t)L.n, s));
  if (L.deg == 3) {  // P3: the FP64 product always in float pairs
    (void)df;
    k_patch_apply_p3<T><<<ceil_div(P, kWarpsP3), 32 * kWarpsP3, 0, s>>>(P, L.pdof, L.pinvdf, L.pinv32, b, y, z, L.nb,
                                                                       L.bnd);
    LAUNCH_CHECK();
    return;
  }
  const int grid = ceil_div((long long)Ppad + L.nb, kBlock);
  if constexpr (sizeof(T) == 8) {
    if (df) {
      k_patch_apply_df<<<grid, kBlock, 0, s>>>(P, Pp, Ppad, L.pdof, reinterpret_cast<const float4*>(L.pinvdf.p), b,
                                               y, z, L.nb, L.bnd);
      LAUNCH_CHECK();
      return;
    }
  }
  k_patch_apply<T><<<grid, kBlock, 0, s>>>(P, Pp, Ppad, L.pdof, patch_inv<T>(L), b, y, z, L.nb, L.bnd);
  LAUNCH_CHECK();
}

template <typename T>
void launch_cheb_pc(int n, const T* z, T* x, T* d, double c1, double c2, bool first_from_zero, bool store_d,
                    cudaStream_t s) {
  k_cheb_pc<T><<<ceil_div(n, kBlock), kBlock, 0, s>>>(n, z, x, d, (T)c1, (T)c2, first_from_zero ? 1 : 0,
                                                      store_d ? 1 : 0);
  LAUNCH_CHECK();
}

template void launch_patch_apply<double>(const Level&, const double*, const double*, double*, bool, cudaStream_t);
template void launch_patch_apply<float>(const Level&, const float*, const float*, float*, bool, cudaStream_t);
template void launch_cheb_pc<double>(int, const double*, double*, double*, double, double, bool, bool, cudaStream_t);
template void launch_cheb_pc<float>(int, const float*, float*, float*, double, double, bool, bool, cudaStream_t);
