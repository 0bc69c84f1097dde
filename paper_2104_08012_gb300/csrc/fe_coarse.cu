// Device-resident FP64 coarse-grid direct solve (paper Section 3: the coarsest
// multigrid level is handled by a direct factorisation, Cholesky here).
//
// Setup (once per coefficient): the interior block of the coarse operator is
// assembled densely in the lexicographic lattice order of the interior dofs,
// which makes it banded with half-bandwidth w = k (1 + e + e^2) (e interior
// points per axis); a right-looking band Cholesky A = L L^T runs one launch
// per column, and the inverse factor L^-1 is formed column by column (one
// warp per column, forward substitution over the band).
// Solve (every V-cycle): x = L^-T (L^-1 b) as two dense triangular
// matrix-vector products, which are fully parallel instead of 2 n
// dependent substitution steps.  Unless the hierarchy runs native FP64, the
// products are evaluated in float-pair arithmetic on the FP32 pipes (L^-1 and
// L^-T stored as float pairs, the vector scaled by a power of two and split
// once per product), since FP64 fused multiply-adds bound the FP64 form.
#include "fe_df.cuh"

namespace {

constexpr int kBlock = 256;

template <int DEG>
__global__ void k_coarse_assemble(int C, int Cs, const int* __restrict__ map, const double* __restrict__ geo,
                                  const int* __restrict__ dof2int, int nci, double* __restrict__ A) {
  constexpr int ND = DEG == 1 ? 4 : 10;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int ii[ND];
  double g[6];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int m = map[(size_t)j * Cs + c];
    ii[j] = m >= 0 ? dof2int[m] : -1;
  }
#pragma unroll
  for (int a = 0; a < 6; ++a) g[a] = geo[(size_t)a * Cs + c];
  for (int j = 0; j < ND; ++j) {
    if (ii[j] < 0) continue;
    double u[ND], out[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) u[k] = (k == j) ? 1.0 : 0.0;
    element_apply<DEG, double>(u, g, out);
    for (int i = 0; i < ND; ++i)
      if (ii[i] >= 0) atomicAdd(A + (size_t)ii[i] * nci + ii[j], out[i]);
  }
}

// Right-looking step j: A[i][k] -= A[i][j] A[k][j] / A[j][j] for j < k <= i <= j + w.
__global__ void k_chol_update(int n, int w, int j, double* __restrict__ A) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x + 1;  // k - j
  const int a = blockIdx.y * blockDim.y + threadIdx.y + 1;  // i - j
  const int wl = min(w, n - 1 - j);
  if (a > wl || b > a) return;
  const int i = j + a, k = j + b;
  const double piv = A[(size_t)j * n + j];
  A[(size_t)i * n + k] -= A[(size_t)i * n + j] * A[(size_t)k * n + j] / piv;
}

// L[i][j] = A[i][j] / sqrt(A[j][j]) inside the band, 0 elsewhere; flags a non-positive pivot.
__global__ void k_chol_scale(int n, int w, double* __restrict__ A, double* __restrict__ dinv, int* __restrict__ flag) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t - (size_t)i * n);
  const double piv = A[(size_t)j * n + j];
  if (i == j && !(piv > 0.0)) atomicOr(flag, 1);
  if (i < j || i - j > w) {
    A[t] = 0.0;
    return;
  }
  // every thread of column j reads the untouched pivot before it is overwritten:
  // the diagonal is rescaled in a separate pass below
  if (i != j) A[t] = A[t] / sqrt(piv);
}

__global__ void k_chol_diag(int n, double* __restrict__ A, double* __restrict__ dinv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double l = sqrt(A[(size_t)j * n + j]);
  A[(size_t)j * n + j] = l;
  dinv[j] = 1.0 / l;
}

// X = L^-1, one warp per column j: X[i][j] = (delta_ij - sum_{k} L[i][k] X[k][j]) / L[i][i]
// for k in [max(j, i-w), i-1]; the last w+1 values of the column live in a
// shared-memory ring.
__global__ void k_tri_inverse(int n, int w, const double* __restrict__ L, const double* __restrict__ dinv,
                              double* __restrict__ Linv, double* __restrict__ LinvT) {
  extern __shared__ double ring_all[];
  const int warps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int j = blockIdx.x * warps + wib;
  if (j >= n) return;
  const int R = w + 1;
  double* ring = ring_all + (size_t)wib * R;
  for (int i = j; i < n; ++i) {
    const int kmin = max(j, i - w);
    double s = 0.0;
    for (int k = kmin + lane; k < i; k += 32) s += L[(size_t)i * n + k] * ring[k % R];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double xi = ((i == j) ? 1.0 : 0.0) - s;
      const double v = xi * dinv[i];
      ring[i % R] = v;
      Linv[(size_t)i * n + j] = v;
      LinvT[(size_t)j * n + i] = v;
    }
    __syncwarp();
  }
}

template <typename T>
__global__ void k_coarse_gather(int nci, const int* __restrict__ ci, const T* __restrict__ b, double* __restrict__ t) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nci) t[j] = (double)b[ci[j]];
}

// out_i = sum_{j<=i} M[i][j] in_j (lower) or out_i = sum_{j>=i} M[i][j] in_j (upper).
// One 256-thread block per row with two independent accumulators per thread:
// the per-row dot products are long (up to n) and FP64-FMA latency bound when
// a single warp walks them.
constexpr int kRowThreads = 256;
__global__ void __launch_bounds__(kRowThreads) k_trimv(int n, const double* __restrict__ M,
                                                       const double* __restrict__ in, double* __restrict__ out,
                                                       int upper) {
  __shared__ double sh[kRowThreads / 32];
  const int row = blockIdx.x;
  const double* Mr = M + (size_t)row * n;
  const int j0 = upper ? row : 0, j1 = upper ? n : row + 1;
  double s0 = 0.0, s1 = 0.0;
  int jj = j0 + threadIdx.x;
  for (; jj + kRowThreads < j1; jj += 2 * kRowThreads) {
    s0 += __ldg(Mr + jj) * __ldg(in + jj);
    s1 += __ldg(Mr + jj + kRowThreads) * __ldg(in + jj + kRowThreads);
  }
  if (jj < j1) s0 += __ldg(Mr + jj) * __ldg(in + jj);
  double s = s0 + s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kRowThreads / 32; ++w) t += sh[w];
    out[row] = t;
  }
}

// Row kernel of y = M v in float pairs: M row-major n x n (float pairs), v
// split by k_split_vec with exponent *ev; y in FP64.
__global__ void __launch_bounds__(kRowThreads) k_trimv_df(int n, const float2* __restrict__ M,
                                                          const float2* __restrict__ v, const int* __restrict__ ev,
                                                          double* __restrict__ out, int upper) {
  using namespace fe_df;
  __shared__ float2 sh[kRowThreads / 32];
  const int row = blockIdx.x;
  const float2* Mr = M + (size_t)row * n;
  const int j0 = upper ? row : 0, j1 = upper ? n : row + 1;
  DF s0, s1;
  int jj = j0 + threadIdx.x;
  for (; jj + kRowThreads < j1; jj += 2 * kRowThreads) {
    const float2 a = __ldg(Mr + jj), b = __ldg(v + jj), c = __ldg(Mr + jj + kRowThreads),
                 d = __ldg(v + jj + kRowThreads);
    s0 = s0 + mul(DF(a.x, a.y), DF(b.x, b.y));
    s1 = s1 + mul(DF(c.x, c.y), DF(d.x, d.y));
  }
  if (jj < j1) {
    const float2 a = __ldg(Mr + jj), b = __ldg(v + jj);
    s0 = s0 + mul(DF(a.x, a.y), DF(b.x, b.y));
  }
  DF s = s0 + s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    s = s + DF(__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_float2(s.hi, s.lo);
  __syncthreads();
  if (threadIdx.x == 0) {
    DF t;
#pragma unroll
    for (int w = 0; w < kRowThreads / 32; ++w) t = t + DF(sh[w].x, sh[w].y);
    const int e = *ev;
    out[row] = widen_scaled(t.hi, e) + widen_scaled(t.lo, e);
  }
}

// One block: v (gathered through idx when idx != null) -> float pairs scaled by
// 2^(1023 - e), e = the largest biased exponent of v (0x7FF: a non-finite
// entry, which is propagated as NaN).
template <typename T>
__global__ void k_split_vec(int n, const int* __restrict__ idx, const T* __restrict__ v, double* __restrict__ vd,
                            float2* __restrict__ vs, int* __restrict__ ev) {
  using namespace fe_df;
  __shared__ int smax;
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  int e = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = (double)v[idx ? idx[i] : i];
    if (vd) vd[i] = x;
    e = max(e, (int)(((unsigned int)__double2hiint(x) >> 20) & 0x7FFu));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&smax, e);
  __syncthreads();
  const int E = smax == 0 ? 1023 : smax;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    DF d = split_scaled((double)v[idx ? idx[i] : i], E);
    if (E == 0x7FF) d = DF(__int_as_float(0x7fc00000), 0.0f);
    vs[i] = make_float2(d.hi, d.lo);
  }
  if (threadIdx.x == 0) *ev = E;
}

__global__ void k_split_mat(size_t nn, const double* __restrict__ a, float2* __restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double x = a[i];
  const float hi = (float)x;
  b[i] = make_float2(hi, (float)(x - (double)hi));
}

template <typename T>
__global__ void k_coarse_scatter(int n, const int* __restrict__ dof2int, const double* __restrict__ t,
                                 const T* __restrict__ b, T* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = dof2int[i];
  x[i] = k >= 0 ? (T)t[k] : b[i];
}

}  // namespace

void coarse_setup(fe_hierarchy* h, cudaStream_t s) {
  Level& L0 = h->L[0];
  CoarseSolver& cs = h->cs;
  const int m = L0.num.m;
  const int e = m - 1;
  const int nci = e * e * e;
  if (nci == 0) {  // every coarse dof is a Dirichlet dof: the coarse solve is the identity
    cs.nci = 0;
    cs.band = 0;
    cs.dof2int.alloc(L0.n);
    CUDA_CHECK(cudaMemsetAsync(cs.dof2int, 0xff, sizeof(int) * L0.n, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    return;
  }
  FE_REQUIRE((double)nci * nci * 8.0 * 3 < 24e9, FE_ERR_UNSUPPORTED, "coarse level too large for the dense Cholesky");
  if (cs.nci != nci) {
    std::vector<int> ci(nci), d2i(L0.n, -1);
    int j = 0;
    for (int z = 1; z < m; ++z)
      for (int y = 1; y < m; ++y)
        for (int x = 1; x < m; ++x) {
          const int dof = lattice_to_dof(L0.num, x, y, z);
          ci[j] = dof;
          d2i[dof] = j++;
        }
    cs.nci = nci;
    cs.band = L0.deg * (1 + e + e * e);
    if (cs.band > nci - 1) cs.band = nci - 1;
    cs.ci.alloc(nci);
    cs.dof2int.alloc(L0.n);
    CUDA_CHECK(cudaMemcpy(cs.ci, ci.data(), sizeof(int) * nci, cudaMemcpyHostToDevice));
    CUDA_CHECK(cudaMemcpy(cs.dof2int, d2i.data(), sizeof(int) * L0.n, cudaMemcpyHostToDevice));
    cs.A.alloc((size_t)nci * nci);
    cs.Linv.alloc((size_t)nci * nci);
    cs.LinvT.alloc((size_t)nci * nci);
    cs.LinvDF.alloc((size_t)nci * nci);
    cs.LinvTDF.alloc((size_t)nci * nci);
    cs.t0.alloc(nci);
    cs.t1.alloc(nci);
    cs.v0.alloc(nci);
    cs.v1.alloc(nci);
    cs.ev.alloc(2);
    cs.flag.alloc(1);
  }
  const size_t nn = (size_t)nci * nci;
  CUDA_CHECK(cudaMemsetAsync(cs.A, 0, sizeof(double) * nn, s));
  if (L0.deg == 1) {
    k_coarse_assemble<1><<<ceil_div(L0.C, kBlock), kBlock, 0, s>>>(L0.C, L0.Cs, L0.map, L0.geo64, cs.dof2int, nci, cs.A);
    LAUNCH_CHECK();
  } else if (L0.deg == 2) {
    k_coarse_assemble<2><<<ceil_div(L0.C, kBlock), kBlock, 0, s>>>(L0.C, L0.Cs, L0.map, L0.geo64, cs.dof2int, nci, cs.A);
    LAUNCH_CHECK();
  } else {
    launch_coarse_assemble_p3(L0, cs.dof2int, nci, cs.A, s);
  }
  const int w = cs.band;
  for (int j = 0; j + 1 < nci; ++j) {
    const int wl = std::min(w, nci - 1 - j);
    dim3 blk(32, 8), grd(ceil_div(wl, 32), ceil_div(wl, 8));
    k_chol_update<<<grd, blk, 0, s>>>(nci, w, j, cs.A);
  }
  LAUNCH_CHECK();
  CUDA_CHECK(cudaMemsetAsync(cs.flag, 0, sizeof(int), s));
  k_chol_scale<<<ceil_div((long long)nn, kBlock), kBlock, 0, s>>>(nci, w, cs.A, cs.t0, cs.flag);
  LAUNCH_CHECK();
  k_chol_diag<<<ceil_div(nci, kBlock), kBlock, 0, s>>>(nci, cs.A, cs.t0);
  LAUNCH_CHECK();
  int hflag = 0;
  CUDA_CHECK(cudaMemcpyAsync(&hflag, cs.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  FE_REQUIRE(hflag == 0, FE_ERR_ARG, "coarse matrix is not positive definite");
  CUDA_CHECK(cudaMemsetAsync(cs.Linv, 0, sizeof(double) * nn, s));
  CUDA_CHECK(cudaMemsetAsync(cs.LinvT, 0, sizeof(double) * nn, s));
  const int warps = 4;
  const size_t shm = sizeof(double) * (size_t)(w + 1) * warps;
  FE_REQUIRE(shm <= 200 * 1024, FE_ERR_UNSUPPORTED, "coarse band too wide");
  if (shm > 48 * 1024) CUDA_CHECK(cudaFuncSetAttribute(k_tri_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  k_tri_inverse<<<ceil_div(nci, warps), warps * 32, shm, s>>>(nci, w, cs.A, cs.t0, cs.Linv, cs.LinvT);
  LAUNCH_CHECK();
  k_split_mat<<<ceil_div((long long)nn, kBlock), kBlock, 0, s>>>(nn, cs.Linv, cs.LinvDF);
  LAUNCH_CHECK();
  k_split_mat<<<ceil_div((long long)nn, kBlock), kBlock, 0, s>>>(nn, cs.LinvT, cs.LinvTDF);
  LAUNCH_CHECK();
  CUDA_CHECK(cudaStreamSynchronize(s));
}

template <typename T>
void coarse_solve(const fe_hierarchy* h, const T* b, T* x, cudaStream_t s) {
  const CoarseSolver& cs = h->cs;
  const Level& L0 = h->L[0];
  const int nci = cs.nci;
  if (nci == 0) {
    k_coarse_scatter<T><<<ceil_div(L0.n, kBlock), kBlock, 0, s>>>(L0.n, cs.dof2int, cs.t0, b, x);
    LAUNCH_CHECK();
    return;
  }
  if (h->f64_mode == FE_F64_NATIVE) {
    k_coarse_gather<T><<<ceil_div(nci, kBlock), kBlock, 0, s>>>(nci, cs.ci, b, cs.t0);
    LAUNCH_CHECK();
    k_trimv<<<nci, kRowThreads, 0, s>>>(nci, cs.Linv, cs.t0, cs.t1, 0);
    LAUNCH_CHECK();
    k_trimv<<<nci, kRowThreads, 0, s>>>(nci, cs.LinvT, cs.t1, cs.t0, 1);
    LAUNCH_CHECK();
  } else {
    k_split_vec<T><<<1, 1024, 0, s>>>(nci, cs.ci, b, nullptr, cs.v0, cs.ev);
    LAUNCH_CHECK();
    k_trimv_df<<<nci, kRowThreads, 0, s>>>(nci, cs.LinvDF, cs.v0, cs.ev, cs.t1, 0);
    LAUNCH_CHECK();
    k_split_vec<double><<<1, 1024, 0, s>>>(nci, nullptr, cs.t1, nullptr, cs.v1, cs.ev + 1);
    LAUNCH_CHECK();
    k_trimv_df<<<nci, kRowThreads, 0, s>>>(nci, cs.LinvTDF, cs.v1, cs.ev + 1, cs.t0, 1);
    LAUNCH_CHECK();
  }
  k_coarse_scatter<T><<<ceil_div(L0.n, kBlock), kBlock, 0, s>>>(L0.n, cs.dof2int, cs.t0, b, x);
  LAUNCH_CHECK();
}

template void coarse_solve<double>(const fe_hierarchy*, const double*, double*, cudaStream_t);
template void coarse_solve<float>(const fe_hierarchy*, const float*, float*, cudaStream_t);
