// bf16 tensor-core operator apply (5th-generation tensor cores: tcgen05 + TMA)
// of the bilinear form of the paper's Section 2, Eq. 4, for P1, P2 and P3.
//
// The element contraction y_K = sum_p G_p S_p x_K (p over the 6 entries of the
// symmetric metric G, S_p the reference stiffness tensors, symmetric) is recast
// as one dense GEMM per tile of 128 cells:
//     W (128 x N) = X (128 x K) . B^T     (bf16 in, FP32 accumulate in TMEM)
// with K = nd padded to 16 (P1, P2) or 32 (P3) and either
//   * the six tables, B = [S_0 | ... | S_5], N = 6 nd padded (32, 64, 128), and
//     the epilogue y_K[i] = sum_p G_p W[p nd + i]; or
//   * when every cell has G = c M (the Kuhn tets of UnitCubeMesh share
//     M = [[2,-1,0],[-1,2,-1],[0,-1,1]]), the one table K_M = sum_p M_p S_p,
//     N = nd padded (16, 16, 32), and the epilogue y_K[i] = c W[i].
// The tables are scaled to integers (6 S for P1, 120 S for P2, 10080 S for P3;
// the geometric factors carry kappa G / 6, / 120 and / 161280 = / (16 x 10080),
// hence the epilogue factor 16 for P3).  Integers up to 2^16 are exact as the
// sum of two bf16 terms, so B = B_hi + B_lo, and every FP32 dof enters as two
// bf16 terms x = x_hi + x_lo + O(2^-17 |x|); W accumulates x_hi B_hi +
// x_lo B_hi + x_hi B_lo (the last only when B_lo is not zero) in one TMEM tile.
//
// Per CTA (persistent, 128 threads = one cell per thread), software-pipelined
// over its tiles k = 0, 1, ...:
//   * TMA (cp.async.bulk.tensor.2d) stages the map rows and geometric values
//     of tile k + 2 into a three-stage ring (mbarrier completion);
//   * the threads gather tile k + 1 from x (FP32) into the other A buffer
//     while the MMAs of tile k run;
//   * one thread issues the MMAs of tile k + 1 into the other TMEM
//     accumulator, which then run while the threads read tile k's accumulator
//     (tcgen05.ld), apply the geometric factors and scatter atomically.
// Every mbarrier wait is bounded in time; on expiry the kernel raises an error
// flag, waits (bounded) for its own copies/MMA in flight, frees its TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "fe_internal.cuh"
#include "fe_reftables.h"

namespace {

constexpr int kTile = 128;
constexpr int kThreads = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait
constexpr int kStages = 3;                              // TMA ring of map / geometry rows

__host__ __device__ constexpr int tc_nd(int deg) { return deg == 1 ? 4 : deg == 2 ? 10 : 20; }
__host__ __device__ constexpr int tc_k(int deg) { return deg == 3 ? 32 : 16; }
__host__ __device__ constexpr int round16(int v) { return (v + 15) / 16 * 16; }
__host__ __device__ constexpr int tc_n(int deg, bool uni) { return uni ? round16(tc_nd(deg)) : round16(6 * tc_nd(deg)); }
__host__ __device__ constexpr int pow2_at_least(int v, int p = 32) { return p >= v ? p : pow2_at_least(v, 2 * p); }

// Shared-memory layout (bytes); the A and B tiles start 1024-aligned.
template <int DEG, bool UNI>
struct Smem {
  static constexpr int ND = tc_nd(DEG), K = tc_k(DEG), N = tc_n(DEG, UNI), NG = UNI ? 1 : 6;
  static constexpr int A_TILE = kTile * K * 2;        // 128 x K bf16
  static constexpr int A = 0;                         // [2 buffers][hi, lo] A tiles
  static constexpr int B = A + 4 * A_TILE;            // [hi, lo] N x K bf16
  static constexpr int B_TILE = N * K * 2;
  static constexpr int MAP = B + 2 * B_TILE;          // kStages x ND x 128 int32
  static constexpr int MAP_STAGE = ND * kTile * 4;
  static constexpr int GEO = MAP + kStages * MAP_STAGE;  // kStages x NG x 128 float
  static constexpr int GEO_STAGE = NG * kTile * 4;
  static constexpr int BAR = GEO + kStages * GEO_STAGE;  // tma[kStages], mma[2]
  static constexpr int TADDR = BAR + (kStages + 2) * 8;
  static constexpr int END = TADDR + 16;
  static constexpr int NCOL = pow2_at_least(2 * N);    // two accumulators
  // Requested size: any request above FLOOR admits at most MAXC CTAs per SM,
  // whose accumulators then fit in the SM's 512 TMEM columns.
  static constexpr int MAXC = 512 / NCOL;
  static constexpr int FLOOR = (227 * 1024) / (MAXC + 1) + 1024;
  static constexpr int REQUEST = ((END > FLOOR ? END : FLOOR) + 1023) / 1024 * 1024;
  static_assert(REQUEST <= 227 * 1024 && (227 * 1024) / REQUEST <= MAXC, "shared layout does not bound the CTAs");
};

// Canonical no-swizzle K-major layout of a (rows x K) bf16 tile: 8 x 16-byte
// core matrices; core (row/8, k/8) at (row/8)*SBO + (k/8)*LBO, SBO = K/8 * LBO.
constexpr int kLBO = 128;  // next core matrix along K

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major no-swizzle tile with 8-row group stride sbo.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
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

// 16 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : FE_R8(0), FE_R8(8)
      : "r"(taddr)
      : "memory");
}

template <int DEG, bool UNI>
__global__ void __launch_bounds__(kThreads) k_apply_tc(const __grid_constant__ CUtensorMap tm_map,
                                                       const __grid_constant__ CUtensorMap tm_geo, int C, int ntiles,
                                                       const uint4* __restrict__ btile, int has_lo, float escale,
                                                       const float* __restrict__ x, float* __restrict__ y,
                                                       int* __restrict__ err) {
  using S = Smem<DEG, UNI>;
  constexpr int ND = S::ND, K = S::K, N = S::N, NG = S::NG, SBO = K * 16;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t bar0 = smem_u32(smem + S::BAR);  // tma[s] at bar0 + 8 s, mma[a] at bar0 + 8 (kStages + a)
  auto bar_tma = [&](int st) { return bar0 + 8u * (uint32_t)st; };
  auto bar_mma = [&](int a) { return bar0 + 8u * (uint32_t)(kStages + a); };
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(smem + S::TADDR);
  constexpr uint32_t tx_bytes = S::MAP_STAGE + S::GEO_STAGE;

  // B tiles (scaled reference tables, hi then lo), already in the canonical layout
  for (int i = tid; i < 2 * S::B_TILE / 16; i += kThreads) reinterpret_cast<uint4*>(smem + S::B)[i] = btile[i];
  if (tid == 0) {
    for (int b = 0; b < kStages + 2; ++b) mbar_init(bar0 + 8u * b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc<S::NCOL>(smem_u32(taddr_slot));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *taddr_slot;
  const uint32_t idesc = instr_desc<N>();
  const int T = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // tiles of this CTA (>= 1)
  auto tile_of = [&](int k) { return (int)blockIdx.x + k * (int)gridDim.x; };
  int tma_issued = 0, tma_done = 0, mma_issued = 0, mma_done = 0;  // issue counts kept by thread 0

  auto issue_tma = [&](int k) {  // thread 0
    const int st = k % kStages;
    mbar_expect_tx(bar_tma(st), tx_bytes);
    tma_load_2d(smem_u32(smem + S::MAP + st * S::MAP_STAGE), &tm_map, tile_of(k) * kTile, 0, bar_tma(st));
    tma_load_2d(smem_u32(smem + S::GEO + st * S::GEO_STAGE), &tm_geo, tile_of(k) * kTile, 0, bar_tma(st));
    ++tma_issued;
  };
  auto issue_mma = [&](int k) {  // thread 0: W(acc k&1) = A_hi B_hi + A_lo B_hi (+ A_hi B_lo)
    const int b = k & 1;
    const uint32_t acc = tbase + (uint32_t)(b * N);
    const uint32_t a_hi = smem_u32(smem + S::A + (2 * b) * S::A_TILE), a_lo = a_hi + S::A_TILE;
    const uint32_t b_hi = smem_u32(smem + S::B), b_lo = b_hi + S::B_TILE;
    uint32_t accumulate = 0u;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
      mma_bf16(acc, smem_desc(a_hi + ks * 2 * kLBO, SBO), smem_desc(b_hi + ks * 2 * kLBO, SBO), idesc, accumulate);
      accumulate = 1u;
    }
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks)
      mma_bf16(acc, smem_desc(a_lo + ks * 2 * kLBO, SBO), smem_desc(b_hi + ks * 2 * kLBO, SBO), idesc, 1u);
    if (has_lo) {
#pragma unroll
      for (int ks = 0; ks < K / 16; ++ks)
        mma_bf16(acc, smem_desc(a_hi + ks * 2 * kLBO, SBO), smem_desc(b_lo + ks * 2 * kLBO, SBO), idesc, 1u);
    }
    mma_commit(bar_mma(b));
    ++mma_issued;
  };
  // this thread's cell of tile k: dofs from x split into two bf16 terms, written as its row of A buffer k&1
  auto gather = [&](int k) {
    const int st = k % kStages, b = k & 1;
    const int c = tile_of(k) * kTile + tid;
    const int* ms = reinterpret_cast<const int*>(smem + S::MAP + st * S::MAP_STAGE);
    __nv_bfloat16 a[K], a2[K];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int m = ms[j * kTile + tid];
      const float v = (c < C && m >= 0) ? __ldg(x + m) : 0.0f;
      a[j] = __float2bfloat16_rn(v);
      a2[j] = __float2bfloat16_rn(v - __bfloat162float(a[j]));
    }
#pragma unroll
    for (int j = ND; j < K; ++j) a[j] = a2[j] = __float2bfloat16_rn(0.0f);
    unsigned char* rhi = smem + S::A + (2 * b) * S::A_TILE + (tid >> 3) * SBO + (tid & 7) * 16;
    unsigned char* rlo = rhi + S::A_TILE;
#pragma unroll
    for (int q = 0; q < K / 8; ++q) {
      uint4 v;
      memcpy(&v, &a[8 * q], 16);
      *reinterpret_cast<uint4*>(rhi + q * kLBO) = v;
      memcpy(&v, &a2[8 * q], 16);
      *reinterpret_cast<uint4*>(rlo + q * kLBO) = v;
    }
  };

  bool failed = false;
  if (tid == 0)
    for (int k = 0; k < 2 && k < T; ++k) issue_tma(k);
  // tile 0: gather, then its MMAs
  {
    const bool ok = mbar_wait(bar_tma(0), 0);
    failed = __syncthreads_or(!ok);
    if (!failed) {
      ++tma_done;
      gather(0);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) issue_mma(0);
    }
  }
  for (int k = 0; k < T && !failed; ++k) {
    const int b = k & 1;
    // (a) tile k + 1 into the other A buffer while the MMAs of tile k run
    if (k + 1 < T) {
      const bool ok = mbar_wait(bar_tma((k + 1) % kStages), ((k + 1) / kStages) & 1);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      ++tma_done;
      gather(k + 1);
    }
    // (b) tile k's accumulator is complete
    {
      const bool ok = mbar_wait(bar_mma(b), (k >> 1) & 1);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      ++mma_done;
    }
    // (c) everyone is past tile k - 1's epilogue and tile k + 1's gather: launch tile k + 1's MMAs and the copy of
    // tile k + 2 (into the stage of tile k - 1)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      if (k + 1 < T) issue_mma(k + 1);
      if (k + 2 < T) issue_tma(k + 2);
    }
    // (d) epilogue of tile k: accumulator k&1, map and geometric values of stage k % kStages
    const int st = k % kStages;
    const int c = tile_of(k) * kTile + tid;
    const int* ms = reinterpret_cast<const int*>(smem + S::MAP + st * S::MAP_STAGE);
    const float* gs = reinterpret_cast<const float*>(smem + S::GEO + st * S::GEO_STAGE);
    float yv[ND];
    const uint32_t acc = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * N);
    if constexpr (UNI) {
      const float cf = escale * gs[tid];
      if constexpr (N == 16) {
        uint32_t r[16];
        tmem_ld16(acc, r);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < ND; ++i) yv[i] = cf * __uint_as_float(r[i]);
      } else {
        uint32_t r[32];
        tmem_ld32(acc, r);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < ND; ++i) yv[i] = cf * __uint_as_float(r[i]);
      }
    } else {
      float g[NG];
#pragma unroll
      for (int q = 0; q < NG; ++q) g[q] = escale * gs[q * kTile + tid];
#pragma unroll
      for (int i = 0; i < ND; ++i) yv[i] = 0.0f;
#pragma unroll
      for (int h = 0; h < N / 32; ++h) {
        uint32_t r[32];
        tmem_ld32(acc + h * 32, r);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int n = h * 32 + q;
          if (n < 6 * ND) yv[n % ND] = fmaf(g[n / ND], __uint_as_float(r[q]), yv[n % ND]);
        }
      }
    }
    if (c < C) {
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        const int m = ms[i * kTile + tid];
        if (m >= 0) atomicAdd(y + m, yv[i]);
      }
    }
  }
  if (failed && tid == 0) {
    atomicOr(err, 1);
    // let the copies and MMAs this CTA still has in flight land (bounded)
    for (int k = tma_done; k < tma_issued; ++k) mbar_wait(bar_tma(k % kStages), (k / kStages) & 1);
    for (int k = mma_done; k < mma_issued; ++k) mbar_wait(bar_mma(k & 1), (k >> 1) & 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc<S::NCOL>(tbase);
}

__global__ void k_bnd_copy32(int nb, const int* __restrict__ bnd, const float* __restrict__ x, float* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nb) y[bnd[t]] = x[bnd[t]];
}

// ------------------------------------------------------------ host tables
// Reference tensors S^{ab}_{ij} = int_ref d_a(phi_i) d_b(phi_j), combined per
// entry p of the symmetric metric (00, 01, 02, 11, 12, 22; an off-diagonal
// entry takes both (a, b) and (b, a)) and scaled to integers:
//   P1: the gradients are constant, 6 S^{ab}_{ij} = dlambda_i[a] dlambda_j[b];
//   P2: every gradient component is a linear form sum_m C[i][a][m] lambda_m and
//       int_ref lambda_m lambda_n = (1 + delta_mn) / 120, so
//       120 S^{ab}_{ij} = sum_mn C_iam C_jbn (1 + delta_mn);
//   P3: 10080 times the reference stiffness coefficients of fe_reftables.h
//       (exact integers, checked).
// escale: the factor between the stored geometric values (kappa G / 6, / 120,
// / 161280) and the tables' scale.
void scaled_tables(int deg, std::vector<double>& Sp, float& escale) {
  const int nd = tc_nd(deg);
  Sp.assign(6 * nd * nd, 0.0);
  escale = 1.0f;
  if (deg == 3) {
    static double K3[210][6], M3[400];
    fe_ref::p3_tables(K3, M3);
    for (int i = 0; i < 20; ++i)
      for (int j = 0; j < 20; ++j) {
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        const int pk = 20 * lo - lo * (lo - 1) / 2 + (hi - lo);
        for (int p = 0; p < 6; ++p) {
          const double v = 10080.0 * K3[pk][p], r = std::nearbyint(v);
          FE_REQUIRE(std::fabs(v - r) < 1e-6, FE_ERR_CUDA, "P3 reference stiffness is not k/10080");
          Sp[(p * nd + i) * nd + j] = r;
        }
      }
    escale = 16.0f;  // 161280 / 10080
    return;
  }
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
            double sum = 0.0;
            for (int m = 0; m < 4; ++m)
              for (int n = 0; n < 4; ++n) sum += Cf[i][a][m] * Cf[j][b][n] * (m == n ? 2.0 : 1.0);
            S[((a * 3 + b) * nd + i) * nd + j] = sum;
          }
  }
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
  for (int p = 0; p < 6; ++p)
    for (int i = 0; i < nd; ++i)
      for (int j = 0; j < nd; ++j) {
        const int a = pa[p], b = pb[p];
        double v = S[((a * 3 + b) * nd + i) * nd + j];
        if (a != b) v += S[((b * 3 + a) * nd + i) * nd + j];
        Sp[(p * nd + i) * nd + j] = v;
      }
}

// B tiles [hi][lo] in the canonical K-major no-swizzle layout: row n of B is
// S_p[i][.] (n = p nd + i, six tables) or K_M[i][.] = sum_p M_p S_p[i][.]
// (n = i, uniform geometry); every value v = hi + lo exactly with two bf16.
struct BTile {
  std::vector<uint16_t> t;
  int has_lo = 0;
  float escale = 1.0f;
};

BTile build_btile(int deg, bool uni) {
  const int nd = tc_nd(deg), K = tc_k(deg), N = tc_n(deg, uni), sbo = K * 16;
  std::vector<double> Sp;
  BTile bt;
  scaled_tables(deg, Sp, bt.escale);
  const double Mv[6] = {2.0, -1.0, 0.0, 2.0, -1.0, 1.0};
  bt.t.assign(2 * N * K, 0);
  const int rows = uni ? nd : 6 * nd;
  for (int n = 0; n < rows; ++n)
    for (int k = 0; k < nd; ++k) {
      double v = 0.0;
      if (uni)
        for (int p = 0; p < 6; ++p) v += Mv[p] * Sp[(p * nd + n) * nd + k];
      else
        v = Sp[n * nd + k];
      const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
      const __nv_bfloat16 lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
      FE_REQUIRE((double)__bfloat162float(hi) + (double)__bfloat162float(lo) == v, FE_ERR_CUDA,
                 "reference table entry not exact as two bf16 terms");
      if (__bfloat162float(lo) != 0.0f) bt.has_lo = 1;
      uint16_t bh, bl;
      memcpy(&bh, &hi, 2);
      memcpy(&bl, &lo, 2);
      const int off = (n >> 3) * sbo + (k >> 3) * kLBO + (n & 7) * 16 + (k & 7) * 2;
      bt.t[off / 2] = bh;
      bt.t[N * K + off / 2] = bl;
    }
  return bt;
}

struct TcLevelData {
  const Level* L = nullptr;
  bool uni = false;
  CUtensorMap tm_map, tm_geo;
};

std::mutex g_tc_mu;
DBuf<uint16_t> g_btile[3][2];
int g_has_lo[3][2] = {};
float g_escale[3] = {1.0f, 1.0f, 1.0f};
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

template <int DEG, bool UNI>
void set_smem_attr() {
  CUDA_CHECK(cudaFuncSetAttribute(k_apply_tc<DEG, UNI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  Smem<DEG, UNI>::REQUEST));
}

const TcLevelData& level_data(const Level& L) {
  std::lock_guard<std::mutex> lock(g_tc_mu);
  const bool uni = L.uniform != 0;
  for (auto& d : g_levels)
    if (d.L == &L && d.uni == uni) return d;
  const float* geo = uni ? L.c32.p : L.geo32.p;
  FE_REQUIRE(L.Cs % kTile == 0 && (reinterpret_cast<uintptr_t>(L.map.p) & 15) == 0 &&
                 (reinterpret_cast<uintptr_t>(geo) & 15) == 0 && (!uni || L.c32.n >= (size_t)L.Cs),
             FE_ERR_CUDA, "tensor-core apply needs 16-byte aligned rows of 128-cell tiles");
  TcLevelData d;
  d.L = &L;
  d.uni = uni;
  make_map_2d(&d.tm_map, CU_TENSOR_MAP_DATA_TYPE_INT32, L.map.p, L.Cs, L.nd, L.nd);
  make_map_2d(&d.tm_geo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, const_cast<float*>(geo), L.Cs, uni ? 1 : 6, uni ? 1 : 6);
  if (!g_btile[L.deg - 1][uni].p) {
    BTile bt = build_btile(L.deg, uni);
    g_btile[L.deg - 1][uni].alloc(bt.t.size());
    CUDA_CHECK(cudaMemcpy(g_btile[L.deg - 1][uni].p, bt.t.data(), bt.t.size() * 2, cudaMemcpyHostToDevice));
    g_has_lo[L.deg - 1][uni] = bt.has_lo;
    g_escale[L.deg - 1] = bt.escale;
  }
  if (!g_err.p) {
    g_err.alloc(1);
    CUDA_CHECK(cudaMemset(g_err.p, 0, sizeof(int)));
    set_smem_attr<1, false>();
    set_smem_attr<1, true>();
    set_smem_attr<2, false>();
    set_smem_attr<2, true>();
    set_smem_attr<3, false>();
    set_smem_attr<3, true>();
  }
  g_levels.push_back(d);
  return g_levels.back();
}

template <int DEG, bool UNI>
void launch_tc(const Level& L, const TcLevelData& d, const float* x, float* y, cudaStream_t s, int sms) {
  using S = Smem<DEG, UNI>;
  const int ntiles = L.Cs / kTile;
  int per_sm = (227 * 1024) / S::REQUEST;
  if (per_sm > S::MAXC) per_sm = S::MAXC;
  if (per_sm > 16) per_sm = 16;
  int grid = per_sm * sms;
  if (grid > ntiles) grid = ntiles;
  k_apply_tc<DEG, UNI><<<grid, kThreads, S::REQUEST, s>>>(
      d.tm_map, d.tm_geo, L.C, ntiles, reinterpret_cast<const uint4*>(g_btile[DEG - 1][UNI].p),
      g_has_lo[DEG - 1][UNI], g_escale[DEG - 1], x, y, g_err.p);
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
    d.uni ? launch_tc<1, true>(L, d, x, y, s, sms) : launch_tc<1, false>(L, d, x, y, s, sms);
  else if (L.deg == 2)
    d.uni ? launch_tc<2, true>(L, d, x, y, s, sms) : launch_tc<2, false>(L, d, x, y, s, sms);
  else
    d.uni ? launch_tc<3, true>(L, d, x, y, s, sms) : launch_tc<3, false>(L, d, x, y, s, sms);
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
