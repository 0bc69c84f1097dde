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
// dependent substitution steps (native FP64 hierarchies).  Otherwise the
// setup also forms A^-1 = L^-T L^-1 (FP64 sums, stored as float pairs) and a
// solve is one launch: the vector scaled by a power of two and split into
// float pairs in each block's shared memory, one dense product with A^-1 in
// float-pair arithmetic on the FP32 pipes (FP64 fused multiply-adds would
// bound it), the result written straight to the interior dofs.
//
// Blocked form (large coarse levels, where n^2 storage is out of reach): the
// band is assembled and factored in band storage (row i holds A[i][i-w..i];
// the interior unknowns are padded with identity rows to a multiple of
// B = w), then for every block I of B rows the inverse D_I of the diagonal
// block L_II and the block E_I = L_{I,I-1} (upper triangular, since B = w)
// are stored with their transposes.  A solve is the forward pass
// y_I = D_I (b_I - E_I y_{I-1}) and the backward pass
// x_I = D_I^T (y_I - E_{I+1}^T x_{I+1}): 4 nb - 2 dense block products, each
// fully parallel over its B rows, in FP64.
#include <chrono>
#include <vector>

#include "fe_df.cuh"

namespace {

constexpr int kBlock = 256;

// band < 0: dense nci x nci (both triangles); band >= 0: band storage
// [nci][band + 1] of the lower triangle.
template <int DEG>
__global__ void k_coarse_assemble(int C, int Cs, const int* __restrict__ map, const double* __restrict__ geo,
                                  const int* __restrict__ dof2int, int nci, double* __restrict__ A, int band) {
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
    for (int i = 0; i < ND; ++i) {
      if (ii[i] < 0) continue;
      if (band < 0)
        atomicAdd(A + (size_t)ii[i] * nci + ii[j], out[i]);
      else if (ii[j] <= ii[i])
        atomicAdd(A + (size_t)ii[i] * (band + 1) + (ii[j] - ii[i] + band), out[i]);
    }
  }
}

// ---- blocked band factor ----
// Right-looking band Cholesky in band storage (p = w + 1 values per row,
// A[i][k] at Ab[i p + k - i + w]) with every column scaled as soon as it is
// final, so the trailing update is a plain product (no FP64 division per
// entry).  Before step j, column j holds L[., j] below the diagonal; step j
// (i = j + a, k = j + b, 1 <= b <= a <= w):
//   b > 1:  A[i][k] -= L[i][j] L[k][j];
//   b = 1:  column j + 1 becomes final: d = A[j+1][j+1] - L[j+1][j]^2 (each
//           thread recomputes it) and L[i][j+1] = (A[i][j+1] - L[i][j] L[j+1][j]) / sqrt(d)
//           for i > j + 1; the diagonal itself is written by thread (1, 1) of
//           step j + 1 (k_bchol_diag_prev for the last two columns), after
//           every thread of step j has read it.
__global__ void k_bchol_first(int n, int w, double* __restrict__ Ab, int* __restrict__ flag) {
  const size_t p = (size_t)w + 1;
  const double d = Ab[w];
  if (!(d > 0.0)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(flag, 1);
    return;
  }
  const double s = sqrt(d);
  const int wl = min(w, n - 1);
  for (int a = blockIdx.x * blockDim.x + threadIdx.x + 1; a <= wl; a += gridDim.x * blockDim.x)
    Ab[(size_t)a * p + (w - a)] /= s;  // L[a][0]
}

__global__ void k_bchol_step(int n, int w, int j, double* __restrict__ Ab, int* __restrict__ flag) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x + 1;  // k - j
  const int a = blockIdx.y * blockDim.y + threadIdx.y + 1;  // i - j
  // rows j + 1 .. j + w + 1: the last one only to scale its entry of column j + 1 (it has no entry in column j)
  const int wl = min(w + 1, n - 1 - j);
  if (a > wl || b > a || (a > w && b > 1)) return;
  const size_t p = (size_t)w + 1;
  const int i = j + a, k = j + b;
  const double lij = a <= w ? Ab[(size_t)i * p + (w - a)] : 0.0;
  if (b > 1) {
    Ab[(size_t)i * p + (k - i + w)] -= lij * Ab[(size_t)k * p + (w - b)];
    return;
  }
  // b = 1: k = j + 1
  const double l1 = Ab[(size_t)k * p + (w - 1)];                // L[j+1][j]
  const double d = Ab[(size_t)k * p + w] - l1 * l1;              // pivot of column j + 1
  if (a == 1) {
    if (!(d > 0.0)) atomicOr(flag, 1);
    if (j >= 1) {  // the diagonal of column j - 1 (no thread of step j reads it)
      const size_t c = (size_t)(j - 1) * p + w;
      const double lc = j >= 2 ? Ab[(size_t)(j - 1) * p + (w - 1)] : 0.0;
      Ab[c] = sqrt(Ab[c] - lc * lc);
    }
    return;
  }
  if (!(d > 0.0)) return;
  const size_t at = (size_t)i * p + (k - i + w);                 // A[i][j+1]
  Ab[at] = (Ab[at] - lij * l1) / sqrt(d);
}

// Diagonal of column j - 1 (for j = n: the last column): sqrt(A[j-1][j-1] - L[j-1][j-2]^2),
// or sqrt(A[0][0]) for column 0.
__global__ void k_bchol_diag_prev(int w, int j, double* __restrict__ Ab) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const size_t p = (size_t)w + 1;
  const int c = j - 1;
  if (c < 0) return;
  const double l = c > 0 ? Ab[(size_t)c * p + (w - 1)] : 0.0;
  Ab[(size_t)c * p + w] = sqrt(Ab[(size_t)c * p + w] - l * l);
}

// D = L_II^-1 for diagonal block I (rows and columns [I B, I B + B)), one
// warp per column j: X[i][j] = (delta_ij - sum_{k = max(j, i - w)}^{i-1}
// L[i][k] X[k][j]) / L[i][i]; the last w + 1 values of the column live in a
// shared-memory ring.  D is row-major B x B (zero above the diagonal, set by
// the caller), DT its transpose.
__global__ void k_btri_inverse(int B, int w, int I, const double* __restrict__ Ab, double* __restrict__ D,
                               double* __restrict__ DT) {
  extern __shared__ double ring_all[];
  const int warps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int jl = blockIdx.x * warps + wib;
  if (jl >= B) return;
  const int R = w + 1;
  const size_t p = (size_t)w + 1;
  double* ring = ring_all + (size_t)wib * R;
  const int j = I * B + jl;
  for (int il = jl; il < B; ++il) {
    const int i = I * B + il;
    const int kmin = max(j, i - w);
    double s = 0.0;
    for (int k = kmin + lane; k < i; k += 32) s += Ab[(size_t)i * p + (k - i + w)] * ring[k % R];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double v = (((i == j) ? 1.0 : 0.0) - s) / Ab[(size_t)i * p + w];
      ring[i % R] = v;
      D[(size_t)il * B + jl] = v;
      DT[(size_t)jl * B + il] = v;
    }
    __syncwarp();
  }
}

// E_I[a][b] = L[I B + a][(I - 1) B + b] (nonzero for b >= a, since B = w) and its transpose.
__global__ void k_bextract(int B, int w, int I, const double* __restrict__ Ab, double* __restrict__ E,
                           double* __restrict__ ET) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)B * B) return;
  const int a = (int)(t / B), b = (int)(t - (size_t)a * B);
  const int i = I * B + a, j = (I - 1) * B + b;
  const double v = (i - j <= w) ? Ab[(size_t)i * ((size_t)w + 1) + (j - i + w)] : 0.0;
  E[t] = v;
  ET[(size_t)b * B + a] = v;
}

// out_r = base_r - sum_j M[r][j] v_j (base != null) or sum_j M[r][j] v_j, j
// over [0, r] (lower) or [r, B) (upper); one block per row.
constexpr int kBlkThreads = 256;
__global__ void __launch_bounds__(kBlkThreads) k_blkmv(int B, const double* __restrict__ M,
                                                       const double* __restrict__ v, const double* __restrict__ base,
                                                       double* __restrict__ out, int upper) {
  __shared__ double sh[kBlkThreads / 32];
  const int row = blockIdx.x;
  const double* Mr = M + (size_t)row * B;
  const int j0 = upper ? row : 0, j1 = upper ? B : row + 1;
  double s0 = 0.0, s1 = 0.0;
  int jj = j0 + threadIdx.x;
  for (; jj + kBlkThreads < j1; jj += 2 * kBlkThreads) {
    s0 += __ldg(Mr + jj) * __ldg(v + jj);
    s1 += __ldg(Mr + jj + kBlkThreads) * __ldg(v + jj + kBlkThreads);
  }
  if (jj < j1) s0 += __ldg(Mr + jj) * __ldg(v + jj);
  double s = s0 + s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kBlkThreads / 32; ++q) t += sh[q];
    out[row] = base ? base[row] - t : t;
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
__global__ void k_coarse_gather(int nci, int npad, const int* __restrict__ ci, const T* __restrict__ b,
                                double* __restrict__ t) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nci)
    t[j] = (double)b[ci[j]];
  else if (j < npad)
    t[j] = 0.0;  // identity padding rows
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

// The coarse inverse A^-1 = L^-T L^-1 from the inverse factor (row-major,
// lower triangular): entry (i, j) is the sum over k >= max(i, j) of
// Linv[k][i] Linv[k][j], in FP64 (n x n, row-major).  One 32 x 32 tile per
// block, tiles above the diagonal only, each mirrored.
constexpr int kGramTile = 32;
__global__ void __launch_bounds__(kGramTile * 8) k_inv_gram(int n, const double* __restrict__ Linv,
                                                            double* __restrict__ Ainv) {
  const int I = blockIdx.y, J = blockIdx.x;
  if (I > J) return;
  __shared__ double si[kGramTile][kGramTile + 1], sj[kGramTile][kGramTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int i0 = I * kGramTile, j0 = J * kGramTile;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = j0; k0 < n; k0 += kGramTile) {  // Linv[k][i] = 0 for k < i: k starts at the tile's larger index
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int k = k0 + ty + 8 * r;
      si[ty + 8 * r][tx] = k < n && i0 + tx < n ? Linv[(size_t)k * n + i0 + tx] : 0.0;
      sj[ty + 8 * r][tx] = k < n && j0 + tx < n ? Linv[(size_t)k * n + j0 + tx] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGramTile; ++kk) {
      const double b = sj[kk][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = fma(si[kk][ty + 8 * r], b, acc[r]);
    }
    __syncthreads();
  }
  const int j = j0 + tx;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 8 * r;
    if (i < n && j < n) {
      Ainv[(size_t)i * n + j] = acc[r];
      Ainv[(size_t)j * n + i] = acc[r];
    }
  }
}

// The largest biased exponent on the diagonal of A^-1 (an SPD matrix: its
// largest entry lies on the diagonal).
__global__ void k_diag_exponent(int n, const double* __restrict__ Ainv, int* __restrict__ e) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicMax(e, (int)(((unsigned int)__double2hiint(Ainv[(size_t)i * n + i]) >> 20) & 0x7FFu));
}

// A^-1 * 2^(1023 - ea) as float pairs in rows of the even length ld (every row
// starts on 16 bytes; the padding is zero).
__global__ void k_split_rows(int n, int ld, const double* __restrict__ Ainv, const int* __restrict__ ea,
                             float2* __restrict__ out) {
  const size_t nn = (size_t)n * ld;
  const double sc = __hiloint2double((2046 - *ea) << 20, 0);  // 2^(1023 - ea), ea in [1, 2045]
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / ld), j = (int)(t - (size_t)i * ld);
    const double x = j < n ? Ainv[(size_t)i * n + j] * sc : 0.0;
    const float hi = (float)x;
    out[t] = make_float2(hi, (float)(x - (double)hi));
  }
}

// The whole coarse solve x = A^-1 b in one launch (float pairs on the FP32
// pipes).  Each warp streams its rows of A^-1 2^(1023 - ea) (float pairs) in
// chunks of 128 16-byte words through a three-stage ring in shared memory,
// filled by cp.async (no registers held by the copies in flight; each lane
// contracts exactly the words it copied, so the ring needs no barrier).  The
// first two chunks go out before the block prepares v: the interior entries
// of b gathered into shared memory as float pairs scaled by 2^(1023 - e), e
// the largest biased exponent among them (0x7FF: a non-finite entry,
// propagated as NaN).  Each row is scaled back by 2^(e + ea - 2046) and
// written to its interior dof of x; the boundary dofs copy b.  The matrix is
// read once per solve (n_interior * ld * 8 bytes); b and x must not overlap.
constexpr int kInvThreads = 256;
constexpr int kInvStages = 3;
constexpr int kInvWords = 4;                      // 16-byte words per lane per chunk
constexpr int kInvChunkWords = 32 * kInvWords;    // per warp: 2 KB
__host__ __device__ constexpr size_t coarse_inv_smem(int ld) {  // ring of every warp, then v
  return sizeof(float4) * ((size_t)(kInvThreads / 32) * kInvStages * kInvChunkWords + (size_t)(ld / 2));
}

template <typename T>
__global__ void __launch_bounds__(kInvThreads, 3) k_coarse_inv_df(int n, int nci, int ld, const int* __restrict__ ci,
                                                                  const int* __restrict__ dof2int,
                                                                  const float2* __restrict__ Ainv, int ea,
                                                                  const T* __restrict__ b, T* __restrict__ x) {
  using namespace fe_df;
  extern __shared__ float4 sm4[];
  __shared__ int smax;
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  float4* ring = sm4 + (threadIdx.x >> 5) * (kInvStages * kInvChunkWords);
  float4* vs4 = sm4 + (kInvThreads / 32) * kInvStages * kInvChunkWords;  // [ld / 2]
  float2* vs = reinterpret_cast<float2*>(vs4);
  const int q1 = ld / 2;                                      // 16-byte words (two float pairs) per row
  const int nch = (q1 + kInvChunkWords - 1) / kInvChunkWords;  // chunks per row
  const int nrows = wid < nci ? (nci - wid + nw - 1) / nw : 0;  // rows wid, wid + nw, ...
  const int ctot = nrows * nch;
  // chunk c of this warp: row wid + nw (c / nch), words (c % nch) kInvChunkWords + 32 u + lane, into slot c % 3
  auto issue = [&](int c) {
    if (c < ctot) {
      const int rr = c / nch, k = c - rr * nch;
      const float4* Ar = reinterpret_cast<const float4*>(Ainv + (size_t)(wid + nw * rr) * ld);
      float4* dst = ring + (c % kInvStages) * kInvChunkWords;
#pragma unroll
      for (int u = 0; u < kInvWords; ++u) {
        const int q = k * kInvChunkWords + 32 * u + lane;
        cp_async16(dst + 32 * u + lane, Ar + min(q, q1 - 1), q < q1 ? 16 : 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int c = 0; c < kInvStages - 1; ++c) issue(c);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (dof2int[i] < 0) x[i] = b[i];
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  // b is gathered once, eight loads in flight per thread: the doubles are parked in the float-pair slots
  // (8 bytes each) until e is known
  double* vd = reinterpret_cast<double*>(vs4);
  int e = 0;
  for (int j0 = threadIdx.x; j0 < nci; j0 += 8 * kInvThreads) {
    int idx[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) idx[u] = j0 + kInvThreads * u < nci ? ci[j0 + kInvThreads * u] : -1;
    double d[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) d[u] = idx[u] >= 0 ? (double)b[idx[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (idx[u] >= 0) {
        vd[j0 + kInvThreads * u] = d[u];
        e = max(e, (int)(((unsigned int)__double2hiint(d[u]) >> 20) & 0x7FFu));
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&smax, e);
  __syncthreads();
  const int E = smax == 0 ? 1023 : smax;
  for (int j = threadIdx.x; j < ld; j += blockDim.x) {  // each thread converts the slots it filled
    DF d(0.0f, 0.0f);
    if (j < nci) d = E == 0x7FF ? DF(__int_as_float(0x7fc00000), 0.0f) : split_scaled(vd[j], E);
    vs[j] = make_float2(d.hi, d.lo);
  }
  __syncthreads();
  DF s0, s1;
  for (int c = 0; c < ctot; ++c) {
    issue(c + kInvStages - 1);
    cp_async_wait<kInvStages - 1>();  // this lane's words of chunk c have landed
    const float4* src = ring + (c % kInvStages) * kInvChunkWords;
    const int rr = c / nch, k = c - rr * nch;
#pragma unroll
    for (int u = 0; u < kInvWords; ++u) {
      const float4 a = src[32 * u + lane];  // zero past the row end
      const float4 v = vs4[min(k * kInvChunkWords + 32 * u + lane, q1 - 1)];
      s0 = s0 + mul(DF(a.x, a.y), DF(v.x, v.y));
      s1 = s1 + mul(DF(a.z, a.w), DF(v.z, v.w));
    }
    if (k == nch - 1) {  // the row is complete
      DF t = s0 + s1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        t = t + DF(__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o));
      if (lane == 0)
        x[ci[wid + nw * rr]] = (T)(widen_scaled(t.hi, E + ea - 1023) + widen_scaled(t.lo, E + ea - 1023));
      s0 = DF(0.0f, 0.0f);
      s1 = DF(0.0f, 0.0f);
    }
  }
  cp_async_wait_all();
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

// Interior coarse unknowns above which FE_COARSE_AUTO takes the blocked form
// (the dense inverse factors would need five n^2 arrays: 10.7 GB at 16384).
constexpr int kDenseMaxInterior = 16384;

static void coarse_setup_dense(fe_hierarchy* h, cudaStream_t s) {
  Level& L0 = h->L[0];
  CoarseSolver& cs = h->cs;
  const int nci = cs.nci, w = cs.band;
  FE_REQUIRE((double)nci * nci * 8.0 * 3 < 24e9, FE_ERR_UNSUPPORTED, "coarse level too large for the dense Cholesky");
  for (auto* b : {&cs.Ab, &cs.D, &cs.DT, &cs.E, &cs.ET, &cs.yb}) b->release();
  const size_t nn = (size_t)nci * nci;
  cs.A.alloc(nn);
  cs.Linv.alloc(nn);
  cs.LinvT.alloc(nn);
  cs.ld = nci + (nci & 1);
  cs.AinvDF.alloc((size_t)nci * cs.ld);
  cs.bytes = nn * 3 * sizeof(double) + (size_t)nci * cs.ld * sizeof(float2);
  CUDA_CHECK(cudaMemsetAsync(cs.A, 0, sizeof(double) * nn, s));
  if (L0.deg == 1) {
    k_coarse_assemble<1><<<ceil_div(L0.C, kBlock), kBlock, 0, s>>>(L0.C, L0.Cs, L0.map, L0.geo64, cs.dof2int, nci, cs.A,
                                                                   -1);
    LAUNCH_CHECK();
  } else if (L0.deg == 2) {
    k_coarse_assemble<2><<<ceil_div(L0.C, kBlock), kBlock, 0, s>>>(L0.C, L0.Cs, L0.map, L0.geo64, cs.dof2int, nci, cs.A,
                                                                   -1);
    LAUNCH_CHECK();
  } else {
    launch_coarse_assemble_p3(L0, cs.dof2int, nci, cs.A, -1, s);
  }
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
  // A^-1 = L^-T L^-1 in FP64 into cs.A (the factor is no longer needed), then as scaled float pairs
  const int tiles = ceil_div(nci, kGramTile);
  k_inv_gram<<<dim3(tiles, tiles), dim3(kGramTile, 8), 0, s>>>(nci, cs.Linv, cs.A);
  LAUNCH_CHECK();
  CUDA_CHECK(cudaMemsetAsync(cs.flag, 0, sizeof(int), s));
  k_diag_exponent<<<ceil_div(nci, kBlock), kBlock, 0, s>>>(nci, cs.A, cs.flag);
  LAUNCH_CHECK();
  CUDA_CHECK(cudaMemcpyAsync(&cs.ainv_exp, cs.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  FE_REQUIRE(cs.ainv_exp >= 1 && cs.ainv_exp <= 2045, FE_ERR_ARG, "coarse inverse out of the FP64 range");
  k_split_rows<<<std::min(ceil_div((long long)nci * cs.ld, kBlock), 1 << 20), kBlock, 0, s>>>(nci, cs.ld, cs.A,
                                                                                             cs.flag, cs.AinvDF);
  LAUNCH_CHECK();
  // the fused solve: v in dynamic shared memory, a persistent grid of the resident blocks (at most one warp per row)
  // The shared-memory limit is a process-wide attribute of the kernel: it is set to the cap checked here, the
  // largest size the kernel is ever launched with, not to this hierarchy's size, so that setting up a smaller coarse
  // level later cannot invalidate the launches of a larger one.
  constexpr int kInvSmemMax = 200 * 1024;
  cs.inv_smem = coarse_inv_smem(cs.ld);
  FE_REQUIRE(cs.inv_smem <= kInvSmemMax, FE_ERR_UNSUPPORTED, "coarse level too large for the fused dense solve");
  int dev = 0, sms = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  auto grid_of = [&](auto kernel) {
    CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kInvSmemMax));
    int per_sm = 0;
    CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kInvThreads, cs.inv_smem));
    return std::max(1, std::min(std::max(1, per_sm) * sms, ceil_div(nci, kInvThreads / 32)));
  };
  cs.inv_grid64 = grid_of(k_coarse_inv_df<double>);
  cs.inv_grid32 = grid_of(k_coarse_inv_df<float>);
}

static void coarse_setup_blocked(fe_hierarchy* h, cudaStream_t s) {
  Level& L0 = h->L[0];
  CoarseSolver& cs = h->cs;
  const int nci = cs.nci, w = cs.band;
  for (auto* b : {&cs.A, &cs.Linv, &cs.LinvT}) b->release();
  cs.AinvDF.release();
  const int B = std::max(w, 1);
  const int nb = ceil_div(nci, B), npad = nb * B;
  const size_t p = (size_t)w + 1, bb = (size_t)B * B;
  cs.B = B;
  cs.nb = nb;
  cs.npad = npad;
  cs.Ab.alloc((size_t)npad * p);
  cs.D.alloc(nb * bb);
  cs.DT.alloc(nb * bb);
  cs.E.alloc(nb * bb);
  cs.ET.alloc(nb * bb);
  cs.yb.alloc(npad);
  cs.t0.alloc(npad);
  cs.t1.alloc(npad);
  cs.bytes = 4 * nb * bb * sizeof(double);
  // band assembly of the interior block, identity on the padding rows
  CUDA_CHECK(cudaMemsetAsync(cs.Ab, 0, sizeof(double) * (size_t)npad * p, s));
  if (L0.deg == 1) {
    k_coarse_assemble<1><<<ceil_div(L0.C, kBlock), kBlock, 0, s>>>(L0.C, L0.Cs, L0.map, L0.geo64, cs.dof2int, nci,
                                                                   cs.Ab, w);
    LAUNCH_CHECK();
  } else if (L0.deg == 2) {
    k_coarse_assemble<2><<<ceil_div(L0.C, kBlock), kBlock, 0, s>>>(L0.C, L0.Cs, L0.map, L0.geo64, cs.dof2int, nci,
                                                                   cs.Ab, w);
    LAUNCH_CHECK();
  } else {
    launch_coarse_assemble_p3(L0, cs.dof2int, nci, cs.Ab, w, s);
  }
  if (npad > nci) {
    std::vector<double> one(1, 1.0);
    for (int i = nci; i < npad; ++i)
      CUDA_CHECK(cudaMemcpyAsync(cs.Ab.p + (size_t)i * p + w, one.data(), sizeof(double), cudaMemcpyHostToDevice, s));
  }
  // right-looking band Cholesky, one launch per column (columns scaled as they become final)
  CUDA_CHECK(cudaMemsetAsync(cs.flag, 0, sizeof(int), s));
  k_bchol_first<<<ceil_div(std::max(w, 1), kBlock), kBlock, 0, s>>>(npad, w, cs.Ab, cs.flag);
  LAUNCH_CHECK();
  for (int j = 0; j + 1 < npad; ++j) {
    const int wl = std::min(w + 1, npad - 1 - j);
    dim3 blk(32, 8), grd(ceil_div(std::min(wl, w), 32), ceil_div(wl, 8));
    k_bchol_step<<<grd, blk, 0, s>>>(npad, w, j, cs.Ab, cs.flag);
  }
  k_bchol_diag_prev<<<1, 32, 0, s>>>(w, npad - 1, cs.Ab);
  k_bchol_diag_prev<<<1, 32, 0, s>>>(w, npad, cs.Ab);
  LAUNCH_CHECK();
  int hflag = 0;
  CUDA_CHECK(cudaMemcpyAsync(&hflag, cs.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  FE_REQUIRE(hflag == 0, FE_ERR_ARG, "coarse matrix is not positive definite");
  // per block: D_I = L_II^-1 (and transpose), E_I = L_{I,I-1} (and transpose)
  CUDA_CHECK(cudaMemsetAsync(cs.D, 0, sizeof(double) * nb * bb, s));
  CUDA_CHECK(cudaMemsetAsync(cs.DT, 0, sizeof(double) * nb * bb, s));
  CUDA_CHECK(cudaMemsetAsync(cs.E, 0, sizeof(double) * nb * bb, s));
  CUDA_CHECK(cudaMemsetAsync(cs.ET, 0, sizeof(double) * nb * bb, s));
  // one shared ring of w + 1 doubles per warp: as many warps per block (up to 4) as fit in 200 KB
  const int warps = (int)std::min<size_t>(4, (200 * 1024) / (sizeof(double) * p));
  FE_REQUIRE(warps >= 1, FE_ERR_UNSUPPORTED, "coarse band too wide for the blocked factor");
  const size_t shm = sizeof(double) * p * warps;
  if (shm > 48 * 1024)
    CUDA_CHECK(cudaFuncSetAttribute(k_btri_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  for (int I = 0; I < nb; ++I) {
    k_btri_inverse<<<ceil_div(B, warps), warps * 32, shm, s>>>(B, w, I, cs.Ab, cs.D.p + I * bb, cs.DT.p + I * bb);
    LAUNCH_CHECK();
    if (I > 0) {
      k_bextract<<<ceil_div((long long)bb, kBlock), kBlock, 0, s>>>(B, w, I, cs.Ab, cs.E.p + I * bb, cs.ET.p + I * bb);
      LAUNCH_CHECK();
    }
  }
  CUDA_CHECK(cudaStreamSynchronize(s));
  cs.Ab.release();  // the blocks hold everything the solves need
}

void coarse_setup(fe_hierarchy* h, cudaStream_t s) {
  Level& L0 = h->L[0];
  CoarseSolver& cs = h->cs;
  const int m = L0.num.m;
  const int e = m - 1;
  const int nci = e * e * e;
  const auto t0 = std::chrono::steady_clock::now();
  if (nci == 0) {  // every coarse dof is a Dirichlet dof: the coarse solve is the identity
    cs.nci = 0;
    cs.band = 0;
    cs.blocked = 0;
    cs.bytes = 0;
    cs.dof2int.alloc(L0.n);
    CUDA_CHECK(cudaMemsetAsync(cs.dof2int, 0xff, sizeof(int) * L0.n, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    return;
  }
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
    cs.t0.alloc(nci);
    cs.t1.alloc(nci);
    cs.flag.alloc(1);
  }
  const bool blocked =
      h->coarse_mode == FE_COARSE_BLOCKED || (h->coarse_mode == FE_COARSE_AUTO && nci > kDenseMaxInterior);
  cs.blocked = blocked ? 1 : 0;
  if (blocked)
    coarse_setup_blocked(h, s);
  else
    coarse_setup_dense(h, s);
  CUDA_CHECK(cudaStreamSynchronize(s));
  cs.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
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
  if (cs.blocked) {
    const int B = cs.B, nb = cs.nb;
    const size_t bb = (size_t)B * B;
    k_coarse_gather<T><<<ceil_div(cs.npad, kBlock), kBlock, 0, s>>>(nci, cs.npad, cs.ci, b, cs.t0);
    LAUNCH_CHECK();
    // forward: y_I = D_I (b_I - E_I y_{I-1})
    for (int I = 0; I < nb; ++I) {
      const double* rhs = cs.t0.p + (size_t)I * B;
      if (I > 0) {
        k_blkmv<<<B, kBlkThreads, 0, s>>>(B, cs.E.p + I * bb, cs.yb.p + (size_t)(I - 1) * B, rhs,
                                          cs.t1.p + (size_t)I * B, 1);
        LAUNCH_CHECK();
        rhs = cs.t1.p + (size_t)I * B;
      }
      k_blkmv<<<B, kBlkThreads, 0, s>>>(B, cs.D.p + I * bb, rhs, nullptr, cs.yb.p + (size_t)I * B, 0);
      LAUNCH_CHECK();
    }
    // backward: x_I = D_I^T (y_I - E_{I+1}^T x_{I+1}), x in t0
    for (int I = nb - 1; I >= 0; --I) {
      const double* rhs = cs.yb.p + (size_t)I * B;
      if (I + 1 < nb) {
        k_blkmv<<<B, kBlkThreads, 0, s>>>(B, cs.ET.p + (I + 1) * bb, cs.t0.p + (size_t)(I + 1) * B, rhs,
                                          cs.t1.p + (size_t)I * B, 0);
        LAUNCH_CHECK();
        rhs = cs.t1.p + (size_t)I * B;
      }
      k_blkmv<<<B, kBlkThreads, 0, s>>>(B, cs.DT.p + I * bb, rhs, nullptr, cs.t0.p + (size_t)I * B, 1);
      LAUNCH_CHECK();
    }
  } else if (h->f64_mode == FE_F64_NATIVE) {
    k_coarse_gather<T><<<ceil_div(nci, kBlock), kBlock, 0, s>>>(nci, nci, cs.ci, b, cs.t0);
    LAUNCH_CHECK();
    k_trimv<<<nci, kRowThreads, 0, s>>>(nci, cs.Linv, cs.t0, cs.t1, 0);
    LAUNCH_CHECK();
    k_trimv<<<nci, kRowThreads, 0, s>>>(nci, cs.LinvT, cs.t1, cs.t0, 1);
    LAUNCH_CHECK();
  } else {
    constexpr bool f64 = sizeof(T) == 8;
    k_coarse_inv_df<T><<<f64 ? cs.inv_grid64 : cs.inv_grid32, kInvThreads, cs.inv_smem, s>>>(
        L0.n, nci, cs.ld, cs.ci, cs.dof2int, cs.AinvDF, cs.ainv_exp, b, x);
    LAUNCH_CHECK();
    return;
  }
  k_coarse_scatter<T><<<ceil_div(L0.n, kBlock), kBlock, 0, s>>>(L0.n, cs.dof2int, cs.t0, b, x);
  LAUNCH_CHECK();
}

template void coarse_solve<double>(const fe_hierarchy*, const double*, double*, cudaStream_t);
template void coarse_solve<float>(const fe_hierarchy*, const float*, float*, cudaStream_t);
