// BLAS-1 kernels of conjugate gradients (the Krylov solve around the
// multigrid preconditioner, paper Section 3) with deterministic grid
// reductions.
//
// Every reduction runs on a fixed grid (ReduceCtx::grid blocks): each block
// reduces its grid-stride slice with warp shuffles, writes one partial, and
// the last block to arrive (atomic ticket) sums the partials in index order
// and derives the CG scalars (alpha, beta, ...) in device memory, so the
// recurrences never wait for the host.  Sums are accumulated in FP64 for
// every vector type.
#include "fe_df.cuh"
#include "fe_internal.cuh"

namespace {

constexpr int kRedBlock = 512;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NV values; in the last block of the grid, thread 0 returns
// true with the grid totals in out[].
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double* __restrict__ partials, unsigned int* __restrict__ counter,
                            double (&out)[NV]) {
  __shared__ double sh[NV][kRedBlock / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = kRedBlock / 32;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? sh[k][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) partials[k * gridDim.x + blockIdx.x] = s;
    }
    if (lane == 0) {
      __threadfence();
      const unsigned int ticket = atomicAdd(counter, 1u);
      last = (ticket == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kRedBlock) s += __ldcg(partials + k * gridDim.x + i);
    s = warp_sum(s);
    __syncthreads();
    if (lane == 0) sh[k][warp] = s;
    __syncthreads();
    if (warp == 0) {
      double t = lane < nw ? sh[k][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) out[k] = t;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
  return threadIdx.x == 0;
}

// The reductions run on a fixed grid of ReduceCtx::grid blocks (2 per SM), so
// with one element per thread in flight they are bound by load latency, not
// by HBM: each thread walks its grid-stride slice kUnroll elements at a time,
// issuing their loads together, then the remainder one by one (a fixed order
// per thread: the sums stay deterministic).
constexpr int kUnroll = 4;

// sum over this thread's slice of a[i] b[i]
template <typename T>
__device__ __forceinline__ double slice_dot(int n, const T* __restrict__ a, const T* __restrict__ b) {
  const int G = gridDim.x * kRedBlock;
  int i = blockIdx.x * kRedBlock + threadIdx.x;
  double s = 0.0;
  for (; i + (kUnroll - 1) * G < n; i += kUnroll * G) {
    T av[kUnroll], bv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      av[u] = a[i + u * G];
      bv[u] = b[i + u * G];
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) s += (double)av[u] * (double)bv[u];
  }
  for (; i < n; i += G) s += (double)a[i] * (double)b[i];
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kRedBlock) k_dot(int n, const T* __restrict__ a, const T* __restrict__ b,
                                                   double* partials, unsigned int* counter, double* scal, int slot) {
  double v[1] = {slice_dot(n, a, b)};
  double out[1];
  if (grid_reduce<1>(v, partials, counter, out)) scal[slot] = out[0];
}

template <typename T>
__global__ void __launch_bounds__(kRedBlock) k_cg_alpha(int n, const T* __restrict__ p, const T* __restrict__ q,
                                                        double* partials, unsigned int* counter, double* scal) {
  double v[1] = {slice_dot(n, p, q)};
  double out[1];
  if (grid_reduce<1>(v, partials, counter, out)) {
    scal[S_PQ] = out[0];
    scal[S_ALPHA] = scal[S_RZ] / out[0];
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedBlock)
    k_cg_update(int n, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                const T* __restrict__ dinv, T* __restrict__ z, double* partials, unsigned int* counter, double* scal) {
  const T alpha = (T)scal[S_ALPHA];
  double v[2] = {0.0, 0.0};
  auto one = [&](int i, T xi, T pi, T ri0, T qi) {
    x[i] = xi + alpha * pi;
    const T ri = ri0 - alpha * qi;
    r[i] = ri;
    v[0] += (double)ri * (double)ri;
    if (dinv) {
      const T zi = dinv[i] * ri;
      z[i] = zi;
      v[1] += (double)ri * (double)zi;
    }
  };
  const int G = gridDim.x * kRedBlock;
  int i = blockIdx.x * kRedBlock + threadIdx.x;
  for (; i + (kUnroll - 1) * G < n; i += kUnroll * G) {
    T xv[kUnroll], pv[kUnroll], rv[kUnroll], qv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      xv[u] = x[i + u * G];
      pv[u] = p[i + u * G];
      rv[u] = r[i + u * G];
      qv[u] = q[i + u * G];
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) one(i + u * G, xv[u], pv[u], rv[u], qv[u]);
  }
  for (; i < n; i += G) one(i, x[i], p[i], r[i], q[i]);
  double out[2];
  if (grid_reduce<2>(v, partials, counter, out)) {
    scal[S_RR] = out[0];
    if (dinv) {
      scal[S_RZNEW] = out[1];
      scal[S_BETA] = out[1] / scal[S_RZ];
      scal[S_RZ] = out[1];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedBlock) k_cg_beta(int n, const T* __restrict__ r, const T* __restrict__ z,
                                                       double* partials, unsigned int* counter, double* scal) {
  double v[1] = {slice_dot(n, r, z)};
  double out[1];
  if (grid_reduce<1>(v, partials, counter, out)) {
    scal[S_RZNEW] = out[0];
    scal[S_BETA] = out[0] / scal[S_RZ];
    scal[S_RZ] = out[0];
  }
}

template <typename T>
__global__ void k_cg_update_p(int n, T* __restrict__ p, const T* __restrict__ z, const double* __restrict__ scal,
                              float2* __restrict__ ps) {
  const T beta = (T)scal[S_BETA];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const T v = z[i] + beta * p[i];
    p[i] = v;
    if constexpr (sizeof(T) == 8)
      if (ps) ps[i] = fe_df::split_pair(v);  // the operator's next input, ready as a float pair
  }
}

__global__ void k_copy_split(int n, const double* __restrict__ z, double* __restrict__ p, float2* __restrict__ ps) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = z[i];
    p[i] = v;
    ps[i] = fe_df::split_pair(v);
  }
}

__global__ void k_axpy64(int n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] += a * x[i];
}

__global__ void k_sub64(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[i] - b[i];
}

// out = in / sqrt(*slot)  (scales a residual to unit norm before a low-precision solve)
template <typename T>
__global__ void k_scale_copy(int n, const double* __restrict__ in, const double* __restrict__ slot, int inverse,
                             T* __restrict__ out) {
  const double s = sqrt(*slot);
  const double f = inverse ? (s > 0.0 ? 1.0 / s : 0.0) : s;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (T)(in[i] * f);
}

// x += sqrt(*slot) * e
template <typename T>
__global__ void k_add_scaled(int n, const T* __restrict__ e, const double* __restrict__ slot, double* __restrict__ x) {
  const double f = sqrt(*slot);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] += f * (double)e[i];
}

int vec_grid(int n, int sms) {
  const int g = ceil_div(n, 256);
  return g < 8 * sms ? (g > 0 ? g : 1) : 8 * sms;
}

}  // namespace

void red_init(ReduceCtx& R, int sms) {
  R.grid = 2 * sms;
  R.partials.alloc((size_t)R.grid * 2);
  R.counter.alloc(1);
  R.scal.alloc(S_COUNT);
  CUDA_CHECK(cudaMemset(R.counter, 0, sizeof(unsigned int)));
  CUDA_CHECK(cudaMemset(R.scal, 0, sizeof(double) * S_COUNT));
  if (!R.h_scal) CUDA_CHECK(cudaMallocHost(&R.h_scal, sizeof(double) * S_COUNT));
}

void red_free(ReduceCtx& R) {
  if (R.h_scal) cudaFreeHost(R.h_scal);
  R.h_scal = nullptr;
}

static int red_grid(const ReduceCtx& R, int n) {
  // fewer blocks for short vectors (the order stays fixed for a given n)
  const int g = ceil_div(n, kRedBlock);
  return g < R.grid ? (g > 0 ? g : 1) : R.grid;
}

template <typename T>
void launch_dot(ReduceCtx& R, int n, const T* a, const T* b, int slot, cudaStream_t s) {
  k_dot<T><<<red_grid(R, n), kRedBlock, 0, s>>>(n, a, b, R.partials, R.counter, R.scal, slot);
  LAUNCH_CHECK();
}

template <typename T>
void launch_cg_alpha(ReduceCtx& R, int n, const T* p, const T* q, cudaStream_t s) {
  k_cg_alpha<T><<<red_grid(R, n), kRedBlock, 0, s>>>(n, p, q, R.partials, R.counter, R.scal);
  LAUNCH_CHECK();
}

template <typename T>
void launch_cg_update(ReduceCtx& R, int n, T* x, T* r, const T* p, const T* q, const T* dinv, T* z, cudaStream_t s) {
  k_cg_update<T><<<red_grid(R, n), kRedBlock, 0, s>>>(n, x, r, p, q, dinv, z, R.partials, R.counter, R.scal);
  LAUNCH_CHECK();
}

template <typename T>
void launch_cg_beta(ReduceCtx& R, int n, const T* r, const T* z, cudaStream_t s) {
  k_cg_beta<T><<<red_grid(R, n), kRedBlock, 0, s>>>(n, r, z, R.partials, R.counter, R.scal);
  LAUNCH_CHECK();
}

template <typename T>
void launch_cg_update_p(ReduceCtx& R, int n, T* p, const T* z, cudaStream_t s, float2* ps) {
  k_cg_update_p<T><<<vec_grid(n, R.grid / 2), 256, 0, s>>>(n, p, z, R.scal, ps);
  LAUNCH_CHECK();
}

void launch_copy_split(int n, const double* z, double* p, float2* ps, cudaStream_t s) {
  const int g = ceil_div(n, 256);
  k_copy_split<<<g < 8192 ? (g > 0 ? g : 1) : 8192, 256, 0, s>>>(n, z, p, ps);
  LAUNCH_CHECK();
}

namespace {
// Loop test of the device-side CG loop: ctl = {completed iterations, limit},
// cgp[0] = the squared residual target.  Continue while the residual is finite,
// above the target and the limit is not reached.
__global__ void k_cg_cond(cudaGraphConditionalHandle hnd, const double* __restrict__ scal,
                          const double* __restrict__ cgp, int* __restrict__ ctl, int inc) {
  const int it = ctl[0] + inc;
  ctl[0] = it;
  const double rr = scal[S_RR];
  cudaGraphSetConditional(hnd, (isfinite(rr) && rr > cgp[0] && it < ctl[1]) ? 1u : 0u);
}
__global__ void k_cg_set(double* __restrict__ cgp, int* __restrict__ ctl, double tol2, int it0, int max_it) {
  cgp[0] = tol2;
  ctl[0] = it0;
  ctl[1] = max_it;
}
}  // namespace

void launch_cg_cond(cudaGraphConditionalHandle hnd, const double* scal, const double* cgp, int* ctl, int inc,
                    cudaStream_t s) {
  k_cg_cond<<<1, 1, 0, s>>>(hnd, scal, cgp, ctl, inc);
  LAUNCH_CHECK();
}

void launch_cg_set(double* cgp, int* ctl, double tol2, int it0, int max_it, cudaStream_t s) {
  k_cg_set<<<1, 1, 0, s>>>(cgp, ctl, tol2, it0, max_it);
  LAUNCH_CHECK();
}

void launch_axpy64(int n, double a, const double* x, double* y, cudaStream_t s) {
  k_axpy64<<<vec_grid(n, 152), 256, 0, s>>>(n, a, x, y);
  LAUNCH_CHECK();
}

void launch_sub64(int n, const double* a, const double* b, double* out, cudaStream_t s) {
  k_sub64<<<vec_grid(n, 152), 256, 0, s>>>(n, a, b, out);
  LAUNCH_CHECK();
}

template <typename T>
void launch_scale_copy(int n, const double* in, const double* slot, bool inverse, T* out, cudaStream_t s) {
  k_scale_copy<T><<<vec_grid(n, 152), 256, 0, s>>>(n, in, slot, inverse ? 1 : 0, out);
  LAUNCH_CHECK();
}

template <typename T>
void launch_add_scaled(int n, const T* e, const double* slot, double* x, cudaStream_t s) {
  k_add_scaled<T><<<vec_grid(n, 152), 256, 0, s>>>(n, e, slot, x);
  LAUNCH_CHECK();
}

#define FE_INST(T)                                                                                      \
  template void launch_dot<T>(ReduceCtx&, int, const T*, const T*, int, cudaStream_t);                 \
  template void launch_cg_alpha<T>(ReduceCtx&, int, const T*, const T*, cudaStream_t);                  \
  template void launch_cg_update<T>(ReduceCtx&, int, T*, T*, const T*, const T*, const T*, T*,          \
                                    cudaStream_t);                                                      \
  template void launch_cg_beta<T>(ReduceCtx&, int, const T*, const T*, cudaStream_t);                   \
  template void launch_cg_update_p<T>(ReduceCtx&, int, T*, const T*, cudaStream_t, float2*);            \
  template void launch_scale_copy<T>(int, const double*, const double*, bool, T*, cudaStream_t);        \
  template void launch_add_scaled<T>(int, const T*, const double*, double*, cudaStream_t);
FE_INST(double)
FE_INST(float)
#undef FE_INST
