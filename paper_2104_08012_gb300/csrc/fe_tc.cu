// bf16 tensor-core operator apply (5th-generation tensor cores: tcgen05 + TMA)
// of the bilinear form of the paper's Section 2, Eq. 4.
//
// The element contraction y_K = sum_p G_p S_p x_K (p over the 6 entries of the
// symmetric metric G, S_p the reference stiffness tensors, symmetric) is recast
// as one dense GEMM per tile of 128 cells:
//     W (128 x 6*nd) = X (128 x nd) . [S_0 | ... | S_5]^T     (bf16 in, FP32 accumulate)
// followed by the G-weighted reduction y_K[i] = sum_p G_p W[p*nd + i] and an
// atomic scatter.  With the scaled tables (120 S for P2, 6 S for P1, whose
// 1/120 and 1/6 are folded into the per-cell geometric factors) every table
// entry is a small integer, exact in bf16.  Each FP32 dof is split into two
// bf16 terms, x = x_hi + x_lo + O(2^-17 |x|) (x_hi = bf16(x), x_lo =
// bf16(x - x_hi)), and W = X_hi S + X_lo S accumulates both products in the
// same TMEM tile (two MMAs), so the apply carries 16 significant bits of the
// dofs instead of bf16's 8 at no cost in tensor time (the tensor pipe is idle
// most of the kernel).
//
// Per CTA (persistent, 128 threads = one cell per thread, up to 4 CTAs/SM):
//   * TMA (cp.async.bulk.tensor.2d) stages the tile's rows of the cell->dof
//     map and of the FP32 geometric factors into shared memory (double
//     buffered, mbarrier completion);
//   * each thread gathers its cell's dofs from x (FP32), splits them into two
//     bf16 terms and writes its rows of the two A tiles (canonical K-major
//     layout, no swizzle);
//   * one thread issues two tcgen05.mma (M=128, N=64 or 32, K=16; the second
//     accumulates) into a TMEM accumulator and commits to an mbarrier;
//   * each warp reads its 32 TMEM lanes with tcgen05.ld, applies G and scatters.
// Every mbarrier wait is bounded in time; on expiry the kernel raises an error
// flag, waits (bounded) for its own copies/MMA in flight, frees its TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "fe_internal.cuh"

namespace {

constexpr int kTile = 128;
constexpr int kThreads = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

template <int DEG>
struct TcShape;
template <>
struct TcShape<1> {
  static constexpr int ND = 4, N = 32;  // 6*4 = 24 columns used
};
template <>
struct TcShape<2> {
  static constexpr int ND = 10, N = 64;  // 6*10 = 60 columns used
};

// Shared-memory layout (bytes); the A and B tiles start 1024-aligned.
template <int DEG>
struct Smem {
  static constexpr int ND = TcShape<DEG>::ND, N = TcShape<DEG>::N;
  static constexpr int A = 0;                         // 128 x 16 bf16 (leading terms)
  static constexpr int B = A + kTile * 16 * 2;        // N x 16 bf16
  static constexpr int A2 = B + N * 16 * 2;           // 128 x 16 bf16 (trailing terms), 1024-aligned
  static constexpr int MAP = A2 + kTile * 16 * 2;     // 2 stages x ND x 128 int32
  static constexpr int MAP_STAGE = ND * kTile * 4;
  static constexpr int GEO = MAP + 2 * MAP_STAGE;     // 2 stages x 6 x 128 float
  static constexpr int GEO_STAGE = 6 * kTile * 4;
  static constexpr int BAR = GEO + 2 * GEO_STAGE;     // tma[2], mma
  static constexpr int TADDR = BAR + 3 * 8;
  static constexpr int END = TADDR + 16;
  // Requested size: caps residency at 4 CTAs/SM so that at most 4 x 64 TMEM
  // columns (of 512) are ever requested per SM.
  static constexpr int REQUEST = 56 * 1024;
  static_assert(END <= REQUEST, "shared layout overflow");
};

// Canonical no-swizzle K-major layout of a (rows x 16) bf16 tile: 8x16-byte
// core matrices; core (row/8, k/8) at (row/8)*SBO + (k/8)*LBO.
constexpr int kLBO = 128;  // next core matrix along K
constexpr int kSBO = 256;  // next group of 8 rows

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
         ((uint64_t)1 << 46);  // sm_100 descriptor version; base offset 0; no swizzle
}

// kind::f16 instruction descriptor: D F32, A/B bf16, both K-major, M = 128.
template <int N>
__device__ __forceinline__ uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true if the phase completed within kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = now_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (now_ns() - t0 > kWaitNs) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int NCOL>
__device__ __forceinline__ void tmem_alloc(uint32_t slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "n"(NCOL) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

template <int NCOL>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOL) : "memory");
}

// D = A B (accumulate == 0) or D += A B.
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

#define FE_R8(i) "=r"(r[i]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), "=r"(r[i + 4]), "=r"(r[i + 5]), "=r"(r[i + 6]), "=r"(r[i + 7])

// 32 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : FE_R8(0), FE_R8(8), FE_R8(16), FE_R8(24)
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int DEG>
__global__ void __launch_bounds__(kThreads) k_apply_tc(const __grid_constant__ CUtensorMap tm_map,
                                                       const __grid_constant__ CUtensorMap tm_geo, int C, int ntiles,
                                                       const uint4* __restrict__ btile, const float* __restrict__ x,
                                                       float* __restrict__ y, int* __restrict__ err) {
  using S = Smem<DEG>;
  constexpr int ND = S::ND, N = S::N;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* sA = smem + S::A;
  unsigned char* sA2 = smem + S::A2;
  const uint32_t bar_tma0 = smem_u32(smem + S::BAR), bar_mma = smem_u32(smem + S::BAR + 16);
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(smem + S::TADDR);
  constexpr uint32_t tx_bytes = S::MAP_STAGE + S::GEO_STAGE;

  // B tile (scaled reference tables), already in the canonical layout
  for (int i = tid; i < N * 16 * 2 / 16; i += kThreads) reinterpret_cast<uint4*>(smem + S::B)[i] = btile[i];
  if (tid == 0) {
    mbar_init(bar_tma0, 1);
    mbar_init(bar_tma0 + 8, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc<N>(smem_u32(taddr_slot));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *taddr_slot;
  const uint64_t adesc = smem_desc(smem_u32(sA)), adesc2 = smem_desc(smem_u32(sA2));
  const uint64_t bdesc = smem_desc(smem_u32(smem + S::B));
  const uint32_t idesc = instr_desc<N>();

  int it = 0;
  bool failed = false;
  int tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) {
    mbar_expect_tx(bar_tma0, tx_bytes);
    tma_load_2d(smem_u32(smem + S::MAP), &tm_map, tile * kTile, 0, bar_tma0);
    tma_load_2d(smem_u32(smem + S::GEO), &tm_geo, tile * kTile, 0, bar_tma0);
  }
  for (; tile < ntiles; tile += gridDim.x, ++it) {
    const int stage = it & 1;
    const uint32_t bar_tma = bar_tma0 + 8 * stage;
    // prefetch the next tile into the other stage (read by everyone before the last __syncthreads)
    const int next = tile + gridDim.x;
    if (tid == 0 && next < ntiles) {
      const uint32_t nb = bar_tma0 + 8 * (stage ^ 1);
      mbar_expect_tx(nb, tx_bytes);
      tma_load_2d(smem_u32(smem + S::MAP + (stage ^ 1) * S::MAP_STAGE), &tm_map, next * kTile, 0, nb);
      tma_load_2d(smem_u32(smem + S::GEO + (stage ^ 1) * S::GEO_STAGE), &tm_geo, next * kTile, 0, nb);
    }
    const bool ok_tma = mbar_wait(bar_tma, (it >> 1) & 1);
    if (__syncthreads_or(!ok_tma)) {
      failed = true;
      break;
    }
    // gather: one cell per thread
    const int c = tile * kTile + tid;
    const int* ms = reinterpret_cast<const int*>(smem + S::MAP + stage * S::MAP_STAGE);
    const float* gs = reinterpret_cast<const float*>(smem + S::GEO + stage * S::GEO_STAGE);
    int idx[ND];
    float g[6];
    __nv_bfloat16 a[16], a2[16];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      idx[j] = ms[j * kTile + tid];
      const float v = (c < C && idx[j] >= 0) ? __ldg(x + idx[j]) : 0.0f;
      a[j] = __float2bfloat16_rn(v);
      a2[j] = __float2bfloat16_rn(v - __bfloat162float(a[j]));
    }
#pragma unroll
    for (int j = ND; j < 16; ++j) a[j] = a2[j] = __float2bfloat16_rn(0.0f);
#pragma unroll
    for (int p = 0; p < 6; ++p) g[p] = gs[p * kTile + tid];
    {
      const int row_off = (tid >> 3) * kSBO + (tid & 7) * 16;
      uint4 lo, hi;
      memcpy(&lo, &a[0], 16);
      memcpy(&hi, &a[8], 16);
      *reinterpret_cast<uint4*>(sA + row_off) = lo;
      *reinterpret_cast<uint4*>(sA + row_off + kLBO) = hi;
      memcpy(&lo, &a2[0], 16);
      memcpy(&hi, &a2[8], 16);
      *reinterpret_cast<uint4*>(sA2 + row_off) = lo;
      *reinterpret_cast<uint4*>(sA2 + row_off + kLBO) = hi;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      mma_bf16(tbase, adesc, bdesc, idesc, 0u);
      mma_bf16(tbase, adesc2, bdesc, idesc, 1u);
      mma_commit(bar_mma);
    }
    const bool ok_mma = mbar_wait(bar_mma, it & 1);
    if (__syncthreads_or(!ok_mma)) {
      failed = true;
      break;
    }
    tc_fence_after();
    float w[N];
    {
      uint32_t r[32];
#pragma unroll
      for (int h = 0; h < N / 32; ++h) {
        tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + h * 32, r);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 32; ++q) w[h * 32 + q] = __uint_as_float(r[q]);
      }
    }
    tc_fence_before();
    __syncthreads();  // TMEM and the A tile may now be overwritten by the next tile
    if (c < C) {
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        float s = 0.0f;
#pragma unroll
        for (int p = 0; p < 6; ++p) s = fmaf(g[p], w[p * ND + i], s);
        if (idx[i] >= 0) atomicAdd(y + idx[i], s);
      }
    }
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(err, 1);
      // let the copies and the MMA this CTA may still have in flight land (bounded)
      mbar_wait(bar_tma0 + 8 * (it & 1), (it >> 1) & 1);
      mbar_wait(bar_tma0 + 8 * ((it + 1) & 1), ((it + 1) >> 1) & 1);
      mbar_wait(bar_mma, it & 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc<N>(tbase);
}

__global__ void k_bnd_copy32(int nb, const int* __restrict__ bnd, const float* __restrict__ x, float* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nb) y[bnd[t]] = x[bnd[t]];
}

// ------------------------------------------------------------ host tables
// Reference tensors S^{ab}_{ij} = int_ref d_a(phi_i) d_b(phi_j).  Every
// reference gradient component is a linear form sum_m C[i][a][m] lambda_m in
// the barycentrics, and int_ref lambda_m lambda_n = (1 + delta_mn)/120, so
// 120 S^{ab}_{ij} = sum_mn C_iam C_jbn (1 + delta_mn) is an integer (P2); for
// P1 the gradients are constant and 6 S^{ab}_{ij} = dlambda_i[a] dlambda_j[b].
void scaled_tables(int deg, std::vector<double>& Sp) {
  const int nd = deg == 1 ? 4 : 10;
  const int dl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  std::vector<double> S(3 * 3 * nd * nd, 0.0);  // S[a][b][i][j], scaled
  if (deg == 1) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) S[((a * 3 + b) * nd + i) * nd + j] = dl[i][a] * dl[j][b];
  } else {
    double Cf[10][3][4] = {};  // gradient component a of phi_i as a linear form in lambda
    for (int v = 0; v < 4; ++v)
      for (int a = 0; a < 3; ++a)
        for (int m = 0; m < 4; ++m) Cf[v][a][m] = dl[v][a] * ((m == v) ? 3.0 : -1.0);  // (4 lam_v - 1) dlam_v
    for (int v = 0; v < 4; ++v)
      for (int w = v + 1; w < 4; ++w) {
        const int e = p2_edge(v, w);
        for (int a = 0; a < 3; ++a) {
          Cf[e][a][v] += 4.0 * dl[w][a];  // 4 (lam_v dlam_w + lam_w dlam_v)
          Cf[e][a][w] += 4.0 * dl[v][a];
        }
      }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 10; ++i)
          for (int j = 0; j < 10; ++j) {
            double s = 0.0;
            for (int m = 0; m < 4; ++m)
              for (int n = 0; n < 4; ++n) s += Cf[i][a][m] * Cf[j][b][n] * (m == n ? 2.0 : 1.0);
            S[((a * 3 + b) * nd + i) * nd + j] = s;
          }
  }
  // combined symmetric tables in the order of the geometric factors: 00, 01, 02, 11, 12, 22
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
  Sp.assign(6 * nd * nd, 0.0);
  for (int p = 0; p < 6; ++p)
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) {
        const int a = pa[p], b = pb[p];
        double v = S[((a * 3 + b) * nd + i) * nd + j];
        if (a != b) v += S[((b * 3 + a) * nd + i) * nd + j];
        Sp[(p * nd + i) * nd + j] = v;
      }
}

// B tile in the canonical K-major no-swizzle layout: B[n][k] = S_p[i][k], n = p*nd + i.
std::vector<uint16_t> build_btile(int deg) {
  const int nd = deg == 1 ? 4 : 10, N = deg == 1 ? 32 : 64;
  std::vector<double> Sp;
  scaled_tables(deg, Sp);
  std::vector<uint16_t> t(N * 16, 0);
  for (int n = 0; n < 6 * nd; ++n)
    for (int k = 0; k < nd; ++k) {
      const double v = Sp[n * nd + k];
      const __nv_bfloat16 b = __float2bfloat16_rn((float)v);
      FE_REQUIRE((double)__bfloat162float(b) == v, FE_ERR_CUDA, "reference table entry not exact in bf16");
      uint16_t bits;
      memcpy(&bits, &b, 2);
      const int off = (n >> 3) * kSBO + (k >> 3) * kLBO + (n & 7) * 16 + (k & 7) * 2;
      t[off / 2] = bits;
    }
  return t;
}

struct TcLevelData {
  const Level* L = nullptr;
  CUtensorMap tm_map, tm_geo;
};

std::mutex g_tc_mu;
DBuf<uint16_t> g_btile[2];
DBuf<int> g_err;
std::vector<TcLevelData> g_levels;

// cuTensorMapEncodeTiled is fetched from the driver at run time, so the
// library loads (and reports FE_ERR_CUDA) on hosts without a CUDA driver.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    CUDA_CHECK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    FE_REQUIRE(q == cudaDriverEntryPointSuccess && p, FE_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

void make_map_2d(CUtensorMap* tm, CUtensorMapDataType ty, void* base, int inner, int outer, int box_outer) {
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)inner * 4};
  cuuint32_t box[2] = {(cuuint32_t)kTile, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(tm, ty, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  FE_REQUIRE(r == CUDA_SUCCESS, FE_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}

const TcLevelData& level_data(const Level& L) {
  std::lock_guard<std::mutex> lock(g_tc_mu);
  for (auto& d : g_levels)
    if (d.L == &L) return d;
  FE_REQUIRE(L.Cs % kTile == 0 && (reinterpret_cast<uintptr_t>(L.map.p) & 15) == 0 &&
                 (reinterpret_cast<uintptr_t>(L.geo32.p) & 15) == 0,
             FE_ERR_CUDA, "tensor-core apply needs 16-byte aligned rows of 128-cell tiles");
  TcLevelData d;
  d.L = &L;
  make_map_2d(&d.tm_map, CU_TENSOR_MAP_DATA_TYPE_INT32, L.map.p, L.Cs, L.nd, L.nd);
  make_map_2d(&d.tm_geo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, L.geo32.p, L.Cs, 6, 6);
  if (!g_btile[L.deg - 1].p) {
    std::vector<uint16_t> t = build_btile(L.deg);
    g_btile[L.deg - 1].alloc(t.size());
    CUDA_CHECK(cudaMemcpy(g_btile[L.deg - 1].p, t.data(), t.size() * 2, cudaMemcpyHostToDevice));
  }
  if (!g_err.p) {
    g_err.alloc(1);
    CUDA_CHECK(cudaMemset(g_err.p, 0, sizeof(int)));
    CUDA_CHECK(cudaFuncSetAttribute(k_apply_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<1>::REQUEST));
    CUDA_CHECK(cudaFuncSetAttribute(k_apply_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<2>::REQUEST));
  }
  g_levels.push_back(d);
  return g_levels.back();
}

template <int DEG>
void launch_tc(const Level& L, const TcLevelData& d, const float* x, float* y, cudaStream_t s, int sms) {
  using S = Smem<DEG>;
  const int ntiles = L.Cs / kTile;
  int grid = 4 * sms;
  if (grid > ntiles) grid = ntiles;
  k_apply_tc<DEG><<<grid, kThreads, S::REQUEST, s>>>(d.tm_map, d.tm_geo, L.C, ntiles,
                                                      reinterpret_cast<const uint4*>(g_btile[DEG - 1].p), x, y, g_err.p);
  LAUNCH_CHECK();
}

}  // namespace

bool bf16_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;  // the library carries sm_103a code only
}

void apply_bf16_enqueue(const Level& L, const float* x, float* y, cudaStream_t s) {
  FE_REQUIRE(bf16_supported(), FE_ERR_UNSUPPORTED, "bf16 tensor-core apply needs an sm_103 device");
  const TcLevelData& d = level_data(L);
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(float) * (size_t)L.n, s));
  if (L.deg == 1)
    launch_tc<1>(L, d, x, y, s, sms);
  else
    launch_tc<2>(L, d, x, y, s, sms);
  if (L.nb > 0) {
    k_bnd_copy32<<<ceil_div(L.nb, 256), 256, 0, s>>>(L.nb, L.bnd, x, y);
    LAUNCH_CHECK();
  }
}

void bf16_prepare(const Level& L) {
  FE_REQUIRE(bf16_supported(), FE_ERR_UNSUPPORTED, "bf16 tensor-core apply needs an sm_103 device");
  level_data(L);
}

// Raised by k_apply_tc when a bounded wait expired; read and cleared by the host.
int bf16_take_error(cudaStream_t s) {
  if (!g_err.p) return 0;
  int h = 0;
  CUDA_CHECK(cudaMemcpyAsync(&h, g_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  if (h) CUDA_CHECK(cudaMemsetAsync(g_err.p, 0, sizeof(int), s));
  return h;
}

void bf16_forget_level(const Level* L) {
  std::lock_guard<std::mutex> lock(g_tc_mu);
  for (size_t i = 0; i < g_levels.size(); ++i)
    if (g_levels[i].L == L) {
      g_levels.erase(g_levels.begin() + i);
      return;
    }
}
