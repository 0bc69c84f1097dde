// Allocation-free variant of the library's deterministic grid reduction.
//
// The dot products inside the solvers use per-block partial sums in device
// scratch that a hierarchy allocates with cudaMalloc.  fe_dot_noalloc() is the
// same two-level reduction for callers that may not allocate device memory at
// all: a host application that owns the whole device memory budget through its
// own pool, or a latency-critical loop in which cudaMalloc/cudaFree (which can
// synchronise the device) are not allowed.  Its scratch is the static array
// below, which is part of the library's device image: every GPU that loads the
// library holds it until the process exits.
#include <mutex>

#include "fe_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerBlock = 4096;   // elements reduced by one block
constexpr int kNaMaxBlocks = 16384; // partial sums the scratch holds
constexpr long long kNaMaxN = (long long)kNaPerBlock * kNaMaxBlocks;  // 67,108,864 elements

// Scratch: kNaMaxBlocks partial sums, then one slot holding the last-block
// ticket (as unsigned int), then one slot holding the result for host outputs.
// 128 KiB + 512 B.
constexpr int kNaTicketSlot = kNaMaxBlocks;
constexpr int kNaResultSlot = kNaMaxBlocks + 32;
constexpr int kNaSlots = kNaMaxBlocks + 64;
static __device__ __align__(256) double g_noalloc_scratch[kNaSlots];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block b sums x[i] y[i] for i in [b*kNaPerBlock, (b+1)*kNaPerBlock) in a
// fixed order; the last block to finish adds the partials in block order, so
// the result does not depend on scheduling.  `scratch` is the device address
// of g_noalloc_scratch (looked up on the host, see below).
__global__ void __launch_bounds__(kNaThreads) k_dot_noalloc(const double* __restrict__ x, const double* __restrict__ y,
                                                            long long n, double* scratch, double* out) {
  __shared__ double sh[kNaThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long base = (long long)blockIdx.x * kNaPerBlock;
  double v = 0.0;
#pragma unroll 4
  for (int k = 0; k < kNaPerBlock / kNaThreads; ++k) {
    const long long i = base + (long long)k * kNaThreads + threadIdx.x;
    if (i < n) v += x[i] * y[i];
  }
  v = na_warp_sum(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kNaTicketSlot);
  if (warp == 0) {
    double s = lane < kNaThreads / 32 ? sh[lane] : 0.0;
    s = na_warp_sum(s);
    if (lane == 0) {
      scratch[blockIdx.x] = s;
      __threadfence();
      last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kNaThreads) s += __ldcg(scratch + b);
  s = na_warp_sum(s);
  __syncthreads();
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double t = lane < kNaThreads / 32 ? sh[lane] : 0.0;
    t = na_warp_sum(t);
    if (lane == 0) {
      *out = t;
      *ticket = 0u;
    }
  }
}

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current) and cached.  Host code must not pass the symbol itself to a
// kernel: on the host it names a stand-in, not device memory.
std::mutex g_na_mu;
double* g_na_ptr[64] = {};

double* noalloc_scratch() {
  int dev = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  FE_REQUIRE(dev >= 0 && dev < 64, FE_ERR_UNSUPPORTED, "device ordinal out of range for the no-alloc scratch table");
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      FE_FAIL(FE_ERR_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch) failed: ") + cudaGetErrorString(e));
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  return g_na_ptr[dev];
}

// Where a pointer lives: 1 = device (or managed) memory of the current
// device, 0 = host memory (pageable, pinned or unregistered), -1 = device
// memory of another device (the kernel would fault or read the wrong GPU).
int na_where(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == dev ? 1 : -1;
  if (a.type == cudaMemoryTypeManaged) return 1;
  return 0;
}

}  // namespace

extern "C" int fe_dot_noalloc(const double* x, const double* y, long long n, double* out, void* stream) {
  try {
    FE_REQUIRE(x && y && out, FE_ERR_ARG, "null argument");
    FE_REQUIRE(n >= 0, FE_ERR_ARG, "n must be >= 0");
    FE_REQUIRE(n <= kNaMaxN, FE_ERR_ARG,
               "n exceeds the no-alloc scratch capacity of " + std::to_string(kNaMaxN) + " elements");
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    const int wx = na_where(x, dev), wy = na_where(y, dev), wo = na_where(out, dev);
    FE_REQUIRE(wx >= 0 && wy >= 0 && wo >= 0, FE_ERR_ARG,
               "x, y and out must be memory of the current device (or host memory for out)");
    FE_REQUIRE(wx == 1 && wy == 1, FE_ERR_ARG,
               "x and y must be device pointers: the no-alloc entry point cannot stage host data");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = noalloc_scratch();
    const bool dev_out = wo == 1;
    double* dst = dev_out ? out : scratch + kNaResultSlot;
    if (n == 0) {
      CUDA_CHECK(cudaMemsetAsync(dst, 0, sizeof(double), s));
    } else {
      // the ticket must start at zero (a previous call leaves it at zero, a failed one may not)
      CUDA_CHECK(cudaMemsetAsync(scratch + kNaTicketSlot, 0, sizeof(double), s));
      const int grid = (int)((n + kNaPerBlock - 1) / kNaPerBlock);
      k_dot_noalloc<<<grid, kNaThreads, 0, s>>>(x, y, n, scratch, dst);
      LAUNCH_CHECK();
    }
    if (!dev_out) {
      CUDA_CHECK(cudaMemcpyAsync(out, dst, sizeof(double), cudaMemcpyDeviceToHost, s));
      CUDA_CHECK(cudaStreamSynchronize(s));
    }
  } catch (const FeError& e) {
    fe_set_error(e.msg);
    return e.code;
  } catch (...) {
    fe_set_error("unexpected C++ exception");
    return FE_ERR_CUDA;
  }
  return FE_OK;
}
