// FP64-accurate operator application (the bilinear form of the paper's
// Section 2, Eq. 4) computed on the FP32 pipes.
//
// GB300 issues about 2 FP64 FMAs per clock per SM against 128 FP32 operations,
// so the FP64 element contraction (124 FP64 instructions per P2 tet) is bound
// by the FP64 pipe.  This variant evaluates the same element formula in
// double-float arithmetic: every value is an unevaluated sum hi + lo of two
// floats, additions use Knuth's TwoSum and products Dekker/Kahan's FMA-based
// TwoProd (Dekker 1971; Hida, Li & Bailey's "double-double" algorithms
// restated for float pairs), giving about 48 significant bits.  The dofs are
// split into float pairs and the contributions joined back to FP64 by integer
// bit manipulation, so the FP64 pipe only performs one addition per scattered
// contribution; vectors, reductions, transfers, smoother updates and the
// coarse solve stay in FP64.  Each tet's dofs are scaled by a power of two
// (their largest exponent) before the split, so the float pairs never leave
// the FP32 exponent range whatever the magnitude of the vector.
#include <algorithm>
#include <type_traits>

#include "fe_df.cuh"
#include "fe_df2.cuh"
#include "fe_p3.cuh"

// P3 reference mass matrix times 26880 (exact integers, |k| <= 432, so exact in
// FP32); the 1/26880 is folded into the float-pair |det J| factor.
__constant__ float c_M3i[400];

namespace {

using namespace fe_df;
constexpr int kBlock = 256;
constexpr int kBlockP3 = 128;
// Block shape of the pre-split, one-value-per-cell variants of k_apply_df
// (the P2 solver path has moved to k_apply_lp): 128 threads, compiled for 5
// resident blocks (96 registers, no spills).  With the fixed-point limb element, full P2 64^3
// solves measured 6.46 / 6.63 / 6.60 ms for (threads, blocks) = (128, 5) /
// (128, 4) / (256, 2); gathering the next tet's dofs after the limb split
// instead of at the top of the iteration (so its map rows have arrived)
// measured 6.53 ms at (128, 4) and spilled at (128, 5).
constexpr int kBlockDfU = 128;
constexpr int kMinBlocksDfU = 5;


// The dofs whose countdown this thread ended (count returned 1): every other
// contribution was fenced before its countdown, so after an acquiring fence
// y_i in L2 is complete.
template <int ND>
__device__ __forceinline__ void finish_dofs(const int* pidx, const unsigned* prev, const double* y,
                                            const ChebFuse<double>& cf) {
#pragma unroll
  for (int j = 0; j < ND; ++j)
    if (prev[j] == 1u) {
      fence_acq_rel_gpu();
      const int i = pidx[j];
      cf.cnt[i] = __ldg(cf.val + i);
      cheb_update(i, __ldcg(y + i), cf.b, cf.dinv, cf.x, cf.d, cf.c1, cf.c2, cf.store_d);
    }
}

// Persistent grid-stride loop over tets: while one tet is contracted, the
// map rows, dofs and geometric factors of the thread's next tet are already
// in flight (the kernel is otherwise bound by the latency of its gathers).
//
// PRE: the dofs are gathered from xs, the input vector already split into
// unscaled float pairs by the kernel that produced it (split_pair), so a tet
// only finds its largest exponent and scales its ten pairs by a power of two
// (exact) instead of splitting ten FP64 values.  A tet that gathers a marker
// (a dof outside [2^-64, 2^64) or not finite) splits its FP64 dofs from x with
// its own scaling, as without PRE; both paths feed the same element code.
//
// With FUSE the launch also performs the Chebyshev smoother step on its
// input: each interior dof's countdown (its number of tets) is decremented
// after the tet's contributions are issued and fenced; the thread that ends
// it (it looks at the returned counts one tet later, so the atomics' latency
// overlaps the next tet's arithmetic) reads the complete y_i from L2 and
// updates d_i and x_i in place.  Every tet
// gathers x before it scatters, so x_i only changes once all its readers are
// done.  Dirichlet rows (y = x) are updated by the threads that write them.
//
// UNI: geo is L.cdf, one float pair c per cell with G = c M (see Level), and
// the element uses the fixed matrix M instead of six loaded factors.  For P2
// the element matrix is then c times one integer matrix, applied by exact
// fixed-point limbs (p2_kuhn_limbs); the tet's power-of-two scaling goes into
// c, so a pre-split tet uses its gathered pairs as they are, and a tet whose
// dofs are all zero contributes nothing and is skipped.
template <int DEG, bool FUSE, bool PRE, bool UNI>
__global__ void __launch_bounds__(UNI && PRE ? kBlockDfU : kBlock, UNI && PRE ? kMinBlocksDfU : 2) k_apply_df(int C, int Cs, const int* __restrict__ map,
                                                        const float2* __restrict__ geo, const double* x,
                                                        const float2* __restrict__ xs, double* __restrict__ y, int nb,
                                                        const int* __restrict__ bnd, ChebFuse<double> cf) {
  static_assert(!(FUSE && PRE), "the fused smoother changes x during the launch");
  constexpr int ND = DEG == 1 ? 4 : 10;
  constexpr bool LIMBS = DEG == 2 && UNI;  // P2 on Kuhn tets: fixed-point limbs (p2_kuhn_limbs)
  constexpr int NG = UNI ? 1 : 6;  // geometric values per cell
  using XV = typename std::conditional<PRE, float2, double>::type;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < nb; i += stride) {  // Dirichlet rows: identity
    const int k = bnd[i];
    const double xk = x[k];
    y[k] = xk;
    if constexpr (FUSE) cheb_update(k, xk, cf.b, cf.dinv, cf.x, cf.d, cf.c1, cf.c2, cf.store_d);
  }
  // with FUSE, x changes during the launch: plain loads instead of the read-only path
  auto ldx = [&](int i) -> XV {
    if constexpr (PRE)
      return i >= 0 ? __ldg(xs + i) : make_float2(0.0f, 0.0f);
    else
      return i >= 0 ? (FUSE ? x[i] : __ldg(x + i)) : 0.0;
  };
  int pidx[FUSE ? ND : 1];
  unsigned prev[FUSE ? ND : 1];
  bool have_prev = false;
  int c = tid;
  if (c >= C) return;
  int idx[ND];
  XV xv[ND];
  float2 gv[NG];
#pragma unroll
  for (int j = 0; j < ND; ++j) idx[j] = __ldg(map + (size_t)j * Cs + c);
#pragma unroll
  for (int j = 0; j < ND; ++j) xv[j] = ldx(idx[j]);
#pragma unroll
  for (int a = 0; a < NG; ++a) gv[a] = __ldg(geo + (size_t)a * Cs + c);
  while (true) {
    const int cn = c + stride;
    const bool more = cn < C;
    int idn[ND];
    XV xn[ND];
    float2 gn[NG];
    if (more) {
#pragma unroll
      for (int j = 0; j < ND; ++j) idn[j] = __ldg(map + (size_t)j * Cs + cn);
#pragma unroll
      for (int j = 0; j < ND; ++j) xn[j] = ldx(idn[j]);
#pragma unroll
      for (int a = 0; a < NG; ++a) gn[a] = __ldg(geo + (size_t)a * Cs + cn);
    }
    DF u[ND], out[ND];
    int emax;  // the element map is linear: scale by 2^(1023 - emax), contract, unscale
    bool split_here = !PRE;
    float fsc = 1.0f;        // LIMBS: the tet's power-of-two scaling, applied to c instead of the dofs
    bool zero_tet = false;   // LIMBS: every gathered dof is zero (no contribution)
    if constexpr (PRE) {
      unsigned int mb = 0u;  // largest magnitude bits of the leading floats (a marker NaN exceeds every finite one)
#pragma unroll
      for (int j = 0; j < ND; ++j) mb = max(mb, __float_as_uint(xv[j].x) & 0x7FFFFFFFu);
      const int ef = (int)(mb >> 23);  // its exponent field (0xFF: a marker)
      if (ef != 0xFF) {
        const float f = __uint_as_float((unsigned int)(254 - ef) << 23);  // 2^(127 - ef)
        if constexpr (LIMBS) {
#pragma unroll
          for (int j = 0; j < ND; ++j) u[j] = DF(xv[j].x, xv[j].y);
          fsc = f;
          zero_tet = mb == 0u;
        } else {
#pragma unroll
          for (int j = 0; j < ND; ++j) u[j] = DF(__fmul_rn(xv[j].x, f), __fmul_rn(xv[j].y, f));
        }
        emax = ef + 896;
      } else {
        split_here = true;
      }
    }
    if (split_here) {
      double xd[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        if constexpr (PRE)
          xd[j] = idx[j] >= 0 ? __ldg(x + idx[j]) : 0.0;
        else
          xd[j] = xv[j];
      }
      emax = block_exponent<ND>(xd);
#pragma unroll
      for (int j = 0; j < ND; ++j) u[j] = split_scaled(xd[j], emax);
      if (emax == 0x7FF) u[0] = DF(__int_as_float(0x7fc00000), 0.0f);  // propagate NaN/inf dofs
    }
    if constexpr (LIMBS) {
      float A[ND], B[ND], Cl[ND];
      int w = 0;
      if (!zero_tet) {
        // x' = c 2^(126 - ec) x 2^(1023 - emax) stays below 2 (c.hi normalised to [0.5, 1)); the
        // element matrix is 4 c K, so y = K x' 2^(ec + emax - 1147), widened with exponent w
        const unsigned int cb = __float_as_uint(gv[0].x);
        const int ec = (int)((cb >> 23) & 0xFFu);  // c in [2^-100, 2^100]: a normal float
        const float chs = __uint_as_float((cb & 0x807FFFFFu) | (126u << 23));
        const float cls = __fmul_rn(gv[0].y, __uint_as_float((unsigned int)(253 - ec) << 23));
        p2_kuhn_split(u, DF(__fmul_rn(chs, fsc), __fmul_rn(cls, fsc)), A, B, Cl);
        w = ec + emax - 124;
      }
      if (!zero_tet) {
        if (w >= 127 && w <= 1918) {  // every contribution widens without range checks
          const unsigned int kexp = (unsigned int)(w - 127) << 20;
          p2_kuhn_apply(A, B, Cl, [&](int j, DF v) {
            if (idx[j] >= 0) atomicAdd(y + idx[j], widen_in_range(v.hi, kexp) + widen_in_range(v.lo, kexp));
          });
        } else {
          p2_kuhn_apply(A, B, Cl, [&](int j, DF v) {
            if (idx[j] >= 0) atomicAdd(y + idx[j], widen_scaled(v.hi, w) + widen_scaled(v.lo, w));
          });
        }
      }
    } else {
      if constexpr (UNI) {
        element_df_m<DEG>(u, DF(gv[0].x, gv[0].y), out);
      } else {
        DF g[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) g[a] = DF(gv[a].x, gv[a].y);
        element_df<DEG>(u, g, out);
      }
      if (emax >= 127 && emax <= 1918) {  // every contribution widens without range checks
        const unsigned int kexp = (unsigned int)(emax - 127) << 20;
#pragma unroll
        for (int j = 0; j < ND; ++j)
          if (idx[j] >= 0) atomicAdd(y + idx[j], widen_in_range(out[j].hi, kexp) + widen_in_range(out[j].lo, kexp));
      } else {
#pragma unroll
        for (int j = 0; j < ND; ++j)
          if (idx[j] >= 0) atomicAdd(y + idx[j], widen_scaled(out[j].hi, emax) + widen_scaled(out[j].lo, emax));
      }
    }
    if constexpr (FUSE) {
      // the previous tet's countdowns have returned by now: finish its dofs
      if (have_prev) finish_dofs<ND>(pidx, prev, y, cf);
      fence_acq_rel_gpu();  // this tet's contributions before its countdowns
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        pidx[j] = idx[j];
        prev[j] = idx[j] >= 0 ? atomicSub(cf.cnt + idx[j], 1u) : 0u;
      }
      have_prev = true;
    }
    if (!more) break;
    c = cn;
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      idx[j] = idn[j];
      xv[j] = xn[j];
    }
#pragma unroll
    for (int a = 0; a < NG; ++a) gv[a] = gn[a];
  }
  if constexpr (FUSE)
    if (have_prev) finish_dofs<ND>(pidx, prev, y, cf);
}

// The default FP64 operator of the solver (P2, pre-split input, one c per
// Kuhn tet, fixed-point limbs) with its map rows staged in shared memory by
// asynchronous copies (cp.async): a thread's unit two iterations ahead has its
// map entries copied while the current unit is contracted, so the gathers
// of the next unit's dofs only wait for a shared-memory read, and the map
// entries of the current unit are re-read from shared memory for the scatter
// instead of occupying registers.  Three buffers per thread ([buffer][dof]
// [thread]): the current unit (scatter), the next (gathers issued this
// iteration) and the one after (copies in flight).
// A unit (Km) is one tet (KuhnTet) or, on a level where the two tets of every
// pair with the same first axis have the same c, such a pair (KuhnPair): the
// tets 2p and 2p + 1 share a face, so the pair's 14 dofs are gathered, split
// and scattered once (14 gathers and 14 FP64 atomics for two tets instead of
// 20) and the pair stiffness (136 nonzero integers against 2 x 82) is applied
// by the same exact limbs.
// 128 threads.  One tet: 6 resident blocks per SM (79 registers, no spills; the
// staged map frees the registers that held map entries); full P2 64^3 solves
// measured 6.34 / 6.30 / 6.33 / 6.72 ms at 5 / 6 / 7 (spills) / 8 blocks per
// SM, against 6.40 ms for the same element with register-held map rows
// (k_apply_df).
constexpr int kBlockLp = 128;
template <typename Km>
constexpr int lp_min_blocks() {
  return Km::cells == 1 ? 6 : 5;
}

template <typename Km>
__global__ void __launch_bounds__(kBlockLp, lp_min_blocks<Km>())
    k_apply_lp(int U, int Cs, const int* __restrict__ map, const float2* __restrict__ cdf,
               const double* __restrict__ x, const float2* __restrict__ xs, double* __restrict__ y, int nb,
               const int* __restrict__ bnd) {
  constexpr int ND = Km::nd;
  __shared__ int smap[3][ND][kBlockLp];
  const int tx = threadIdx.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < nb; i += stride) y[bnd[i]] = x[bnd[i]];  // Dirichlet rows: identity
  int c = tid;  // the current unit
  if (c >= U) return;
  auto copy_map = [&](int u, int buf) {
    if (u < U) {
#pragma unroll
      for (int j = 0; j < ND; ++j)
        cp_async4(&smap[buf][j][tx], map + (size_t)Km::local(j) * Cs + (size_t)Km::cells * u + Km::cell(j));
    }
    cp_async_commit();
  };
  copy_map(c, 0);
  copy_map(c + stride, 1);
  cp_async_wait_all();
  float2 xv[ND], gv;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int i = smap[0][j][tx];
    xv[j] = i >= 0 ? __ldg(xs + i) : make_float2(0.0f, 0.0f);
  }
  gv = __ldg(cdf + (size_t)Km::cells * c);
  int b = 0;  // buffer of the current unit
  while (true) {
    const int cn = c + stride;
    const bool more = cn < U;
    const int bn = b == 2 ? 0 : b + 1, bnn = bn == 2 ? 0 : bn + 1;
    float2 xn[ND], gn = make_float2(0.0f, 0.0f);
    if (more) {
      cp_async_wait_all();  // the next unit's map entries (copied one iteration ago)
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int i = smap[bn][j][tx];
        xn[j] = i >= 0 ? __ldg(xs + i) : make_float2(0.0f, 0.0f);
      }
      gn = __ldg(cdf + (size_t)Km::cells * cn);
      copy_map(cn + stride, bnn);
    }
    unsigned int mb = 0u;  // largest magnitude bits of the leading floats (a marker NaN exceeds every finite one)
#pragma unroll
    for (int j = 0; j < ND; ++j) mb = max(mb, __float_as_uint(xv[j].x) & 0x7FFFFFFFu);
    const int ef = (int)(mb >> 23);
    if (mb != 0u) {  // a unit whose dofs are all zero contributes nothing
      DF u[ND];
      int emax;
      float fsc = 1.0f;
      if (ef != 0xFF) {
#pragma unroll
        for (int j = 0; j < ND; ++j) u[j] = DF(xv[j].x, xv[j].y);
        fsc = __uint_as_float((unsigned int)(254 - ef) << 23);  // 2^(127 - ef), applied to c
        emax = ef + 896;
      } else {  // a marker: the unit's FP64 dofs split with their own scaling
        double xd[ND];
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          const int i = smap[b][j][tx];
          xd[j] = i >= 0 ? __ldg(x + i) : 0.0;
        }
        emax = block_exponent<ND>(xd);
#pragma unroll
        for (int j = 0; j < ND; ++j) u[j] = split_scaled(xd[j], emax);
        if (emax == 0x7FF) u[0] = DF(__int_as_float(0x7fc00000), 0.0f);  // propagate NaN/inf dofs
      }
      const unsigned int cb = __float_as_uint(gv.x);
      const int ec = (int)((cb >> 23) & 0xFFu);  // c in [2^-100, 2^100]: a normal float
      const float chs = __uint_as_float((cb & 0x807FFFFFu) | (126u << 23));
      const float cls = __fmul_rn(gv.y, __uint_as_float((unsigned int)(253 - ec) << 23));
      float A[ND], B[ND], Cl[ND];
      p2_kuhn_split(u, DF(__fmul_rn(chs, fsc), __fmul_rn(cls, fsc)), A, B, Cl);
      const int w = ec + emax - 124;
      if (w >= 127 && w <= 1918) {  // every contribution widens without range checks
        const unsigned int kexp = (unsigned int)(w - 127) << 20;
        p2_kuhn_apply<Km>(A, B, Cl, [&](int j, DF v) {
          const int i = smap[b][j][tx];
          if (i >= 0) atomicAdd(y + i, widen_in_range(v.hi, kexp) + widen_in_range(v.lo, kexp));
        });
      } else {
        p2_kuhn_apply<Km>(A, B, Cl, [&](int j, DF v) {
          const int i = smap[b][j][tx];
          if (i >= 0) atomicAdd(y + i, widen_scaled(v.hi, w) + widen_scaled(v.lo, w));
        });
      }
    }
    if (!more) break;
    c = cn;
    b = bn;
#pragma unroll
    for (int j = 0; j < ND; ++j) xv[j] = xn[j];
    gv = gn;
  }
  cp_async_wait_all();
}

// P2, two tets per thread (tets 2p and 2p+1, C = 6 N^3 is even): the element
// formula runs in packed FP32x2 instructions (fe_df2.cuh), so each issued
// floating-point instruction serves both tets; map rows are read as int2,
// geometric factors as float4 (both tets' (hi, lo)).  Splitting, widening and
// the atomics stay per tet.  The pair's values take twice the registers of
// one tet; capped at 128 (16 warps per SM, 4 bytes of spill) the kernel has
// no room to prefetch the next pair, and with half as many independent
// instruction chains per warp it measured as fast as the per-tet kernel
// (0.129 ms at 64^3), not faster: 27% fewer instructions, lower issue rate.
__global__ void __launch_bounds__(kBlock, 2) k_apply_df2(int P, int Cs, const int* __restrict__ map,
                                                         const float2* __restrict__ geo,
                                                         const double* __restrict__ x, double* __restrict__ y,
                                                         int nb, const int* __restrict__ bnd) {
  constexpr int ND = 10;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < nb; i += stride) y[bnd[i]] = x[bnd[i]];  // Dirichlet rows: identity
  int p = tid;
  if (p >= P) return;
  int2 id[ND];
  double xa[ND], xb[ND];
  float4 gv[6];
  auto load = [&]() {
#pragma unroll
    for (int j = 0; j < ND; ++j) id[j] = __ldg(reinterpret_cast<const int2*>(map + (size_t)j * Cs) + p);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      xa[j] = id[j].x >= 0 ? __ldg(x + id[j].x) : 0.0;
      xb[j] = id[j].y >= 0 ? __ldg(x + id[j].y) : 0.0;
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) gv[a] = __ldg(reinterpret_cast<const float4*>(geo + (size_t)a * Cs) + p);
  };
  load();
  while (true) {
    const int ea = block_exponent<ND>(xa), eb = block_exponent<ND>(xb);
    DF2 u[ND], g[6], out[ND];
    F2 gneg[6];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      DF a = split_scaled(xa[j], ea), b = split_scaled(xb[j], eb);
      if (j == 0 && ea == 0x7FF) a = DF(__int_as_float(0x7fc00000), 0.0f);  // propagate NaN/inf dofs
      if (j == 0 && eb == 0x7FF) b = DF(__int_as_float(0x7fc00000), 0.0f);
      u[j] = DF2{f2_pack(a.hi, b.hi), f2_pack(a.lo, b.lo)};
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      g[a] = DF2{f2_pack(gv[a].x, gv[a].z), f2_pack(gv[a].y, gv[a].w)};
      gneg[a] = f2_pack(-gv[a].x, -gv[a].z);
    }
    p2_element_df2(u, g, gneg, out);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      float ha, hb, la, lb;
      f2_unpack(out[j].hi, ha, hb);
      f2_unpack(out[j].lo, la, lb);
      if (j >= 7) {  // edges 12, 13, 23 come out negated
        ha = -ha, hb = -hb, la = -la, lb = -lb;
      }
      if (id[j].x >= 0) atomicAdd(y + id[j].x, widen_scaled(ha, ea) + widen_scaled(la, ea));
      if (id[j].y >= 0) atomicAdd(y + id[j].y, widen_scaled(hb, eb) + widen_scaled(lb, eb));
    }
    p += stride;
    if (p >= P) break;
    load();
  }
}

// P3, one tet per thread (persistent grid-stride loop): the element through
// the gradient at the P2 nodes (fe_p3.cuh) in float pairs, on the geometric
// factors kappa G / 161280 split once per tet; dofs split and contributions
// widened per tet as in k_apply_df.  UNI: geo is L.cdf (G = c M per cell).
template <bool UNI>
__global__ void __launch_bounds__(kBlockP3, 2) k_apply_df3(int C, int Cs, const int* __restrict__ map,
                                                           const float2* __restrict__ geo,
                                                           const double* __restrict__ x, double* __restrict__ y,
                                                           int nb, const int* __restrict__ bnd) {
  constexpr int ND = 20;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < nb; i += stride) y[bnd[i]] = x[bnd[i]];  // Dirichlet rows: identity
  for (int c = tid; c < C; c += stride) {
    double xv[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int m = __ldg(map + (size_t)j * Cs + c);
      xv[j] = m >= 0 ? __ldg(x + m) : 0.0;
    }
    DF g[6];
#pragma unroll
    for (int a = 0; a < (UNI ? 1 : 6); ++a) {
      const float2 v = __ldg(geo + (size_t)a * Cs + c);
      g[a] = DF(v.x, v.y);
    }
    const int emax = block_exponent<ND>(xv);
    DF u[ND], out[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) u[j] = split_scaled(xv[j], emax);
    if (emax == 0x7FF) u[0] = DF(__int_as_float(0x7fc00000), 0.0f);  // propagate NaN/inf dofs
    fe_p3::p3_element_grad<fe_p3::DFOps, UNI>(u, g, out);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int m = __ldg(map + (size_t)j * Cs + c);
      if (m >= 0) atomicAdd(y + m, widen_scaled(out[j].hi, emax) + widen_scaled(out[j].lo, emax));
    }
  }
}

// Cube-aggregated variant: one thread per cube splits the cube's (k+1)^3 dofs
// once (scaled by their largest exponent), applies its six Kuhn tets into
// float-pair accumulators and widens/scatters (k+1)^3 values: 27 splits, 27
// FP64 adds and 27 atomics per cube for P2 instead of 60 of each.
// FUSE: the Chebyshev step as in k_apply_df, with cube countdowns.
template <int DEG, bool FUSE>
__global__ void __launch_bounds__(kBlock, 1) k_apply_cube_df(int Q, int Qs, int Cs, const int* __restrict__ cmap,
                                                             const float2* __restrict__ geo, const double* x,
                                                             double* __restrict__ y, int nb,
                                                             const int* __restrict__ bnd, ChebFuse<double> cf) {
  constexpr int NL = DEG == 1 ? 8 : 27, ND = DEG == 1 ? 4 : 10;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (int i = tid; i < nb; i += stride) {  // Dirichlet rows: identity
    const int k = bnd[i];
    const double xk = x[k];
    y[k] = xk;
    if constexpr (FUSE) cheb_update(k, xk, cf.b, cf.dinv, cf.x, cf.d, cf.c1, cf.c2, cf.store_d);
  }
  for (int q = tid; q < Q; q += stride) {
    double xv[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int i = __ldg(cmap + (size_t)l * Qs + q);
      xv[l] = i >= 0 ? (FUSE ? x[i] : __ldg(x + i)) : 0.0;
    }
    const int emax = block_exponent<NL>(xv);
    DF uc[NL], acc[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) uc[l] = split_scaled(xv[l], emax);
    if (emax == 0x7FF) uc[0] = DF(__int_as_float(0x7fc00000), 0.0f);
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      DF u[ND], g[6], o[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) u[j] = uc[cube_local(DEG, t, j)];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const float2 v = __ldg(geo + (size_t)a * Cs + 6 * q + t);
        g[a] = DF(v.x, v.y);
      }
      element_df<DEG>(u, g, o);
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int l = cube_local(DEG, t, j);
        acc[l] = (t == 0 || !touched_before(DEG, t, l)) ? o[j] : acc[l] + o[j];
      }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int i = __ldg(cmap + (size_t)l * Qs + q);
      if (i >= 0) atomicAdd(y + i, widen_scaled(acc[l].hi, emax) + widen_scaled(acc[l].lo, emax));
    }
    if constexpr (FUSE) {
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
  }
}

// Consistent mass, one tet per thread: y += s K u in float pairs (see
// p2_mass_df), dofs scaled by the tet's largest power of two like the operator.
template <int DEG>
__global__ void __launch_bounds__(kBlock) k_mass_df(int C, int Cs, const int* __restrict__ map,
                                                    const float2* __restrict__ mdf, const double* __restrict__ x,
                                                    double* __restrict__ y) {
  constexpr int ND = DEG == 1 ? 4 : 10;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int idx[ND];
  double xv[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int m = __ldg(map + (size_t)j * Cs + c);
    idx[j] = m < 0 ? -1 - m : m;  // the full mass matrix: Dirichlet dofs take part
    xv[j] = __ldg(x + idx[j]);
  }
  const int emax = block_exponent<ND>(xv);
  DF u[ND], out[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) u[j] = split_scaled(xv[j], emax);
  if (emax == 0x7FF) u[0] = DF(__int_as_float(0x7fc00000), 0.0f);  // propagate NaN/inf dofs
  const float2 sv = __ldg(mdf + c);
  if constexpr (DEG == 1)
    p1_mass_df(u, DF(sv.x, sv.y), out);
  else
    p2_mass_df(u, DF(sv.x, sv.y), out);
#pragma unroll
  for (int j = 0; j < ND; ++j) atomicAdd(y + idx[j], widen_scaled(out[j].hi, emax) + widen_scaled(out[j].lo, emax));
}

// P3 consistent mass in float pairs, one tet per thread: (K u)_i with the
// integer matrix K row by row (a runtime loop over rows keeps the code small;
// the columns are unrolled), exact products by the integers (TwoProd of the
// leading term), then times |det J| / 26880; every dof takes part.
__global__ void __launch_bounds__(kBlock) k_mass_df3(int C, int Cs, const int* __restrict__ map,
                                                     const float2* __restrict__ mdf, const double* __restrict__ x,
                                                     double* __restrict__ y) {
  constexpr int ND = 20;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double xv[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int m = __ldg(map + (size_t)j * Cs + c);
    xv[j] = __ldg(x + (m < 0 ? -1 - m : m));
  }
  const int emax = block_exponent<ND>(xv);
  DF u[ND];
#pragma unroll
  for (int j = 0; j < ND; ++j) u[j] = split_scaled(xv[j], emax);
  if (emax == 0x7FF) u[0] = DF(__int_as_float(0x7fc00000), 0.0f);  // propagate NaN/inf dofs
  const float2 sv = __ldg(mdf + c);
  const DF sdet(sv.x, sv.y);
#pragma unroll 1
  for (int i = 0; i < ND; ++i) {
    DF acc(0.0f);
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const float k = c_M3i[i * ND + j];
      const float p = __fmul_rn(u[j].hi, k);
      acc = acc + DF(p, __fmaf_rn(u[j].lo, k, __fmaf_rn(u[j].hi, k, -p)));
    }
    const DF yi = mul(sdet, acc);
    const int m = __ldg(map + (size_t)i * Cs + c);
    atomicAdd(y + (m < 0 ? -1 - m : m), widen_scaled(yi.hi, emax) + widen_scaled(yi.lo, emax));
  }
}

__global__ void k_split_geo(int C, int Cs, const double* __restrict__ geo64, double gscale,
                            float2* __restrict__ geodf, const double* __restrict__ detj, double wmass,
                            float2* __restrict__ mdf) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  for (int a = 0; a < 6; ++a) {
    const double g = geo64[(size_t)a * Cs + c] * gscale;
    const float hi = (float)g;
    geodf[(size_t)a * Cs + c] = make_float2(hi, (float)(g - (double)hi));
  }
  const double m = detj[c] * wmass;
  const float mh = (float)m;
  mdf[c] = make_float2(mh, (float)(m - (double)mh));
}

}  // namespace

void launch_split_geometry(Level& L, cudaStream_t s) {
  k_split_geo<<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(
      L.C, L.Cs, L.geo64, 1.0, L.geodf, L.detj, L.deg == 1 ? 1.0 / 120.0 : L.deg == 2 ? 1.0 / 2520.0 : 1.0 / 26880.0,
      L.massdf);
  LAUNCH_CHECK();
}

void upload_p3_mass_table(const float* m3i) { CUDA_CHECK(cudaMemcpyToSymbol(c_M3i, m3i, sizeof(float) * 400)); }

void launch_mass_df(const Level& L, const double* x, double* y, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)L.n, s));
  if (L.deg == 3)
    k_mass_df3<<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.massdf, x, y);
  else if (L.deg == 1)
    k_mass_df<1><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.massdf, x, y);
  else
    k_mass_df<2><<<ceil_div(L.C, kBlock), kBlock, 0, s>>>(L.C, L.Cs, L.map, L.massdf, x, y);
  LAUNCH_CHECK();
}


template <bool FUSE>
static void apply_cube_df(const Level& L, const double* x, double* y, const ChebFuse<double>& cf, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)L.n, s));
  if (L.deg == 1) {
    static int g1 = 0;
    if (!g1) g1 = resident_grid(k_apply_cube_df<1, FUSE>, kBlock, 1 << 30);
    k_apply_cube_df<1, FUSE><<<std::min(g1, ceil_div(std::max(L.Q, L.nb), kBlock)), kBlock, 0, s>>>(
        L.Q, L.Qs, L.Cs, L.cmap, L.geodf, x, y, L.nb, L.bnd, cf);
  } else {
    static int g2 = 0;
    if (!g2) g2 = resident_grid(k_apply_cube_df<2, FUSE>, kBlock, 1 << 30);
    k_apply_cube_df<2, FUSE><<<std::min(g2, ceil_div(std::max(L.Q, L.nb), kBlock)), kBlock, 0, s>>>(
        L.Q, L.Qs, L.Cs, L.cmap, L.geodf, x, y, L.nb, L.bnd, cf);
  }
  LAUNCH_CHECK();
}

template <int DEG, bool FUSE, bool PRE, bool UNI>
static void apply_df_launch(const Level& L, const double* x, const float2* xs, double* y, const ChebFuse<double>& cf,
                            cudaStream_t s) {
  constexpr int blk = UNI && PRE ? kBlockDfU : kBlock;
  static int g = 0;
  if (!g) g = resident_grid(k_apply_df<DEG, FUSE, PRE, UNI>, blk, 1 << 30);
  k_apply_df<DEG, FUSE, PRE, UNI><<<std::min(g, ceil_div(std::max(L.C, L.nb), blk)), blk, 0, s>>>(
      L.C, L.Cs, L.map, UNI ? L.cdf.p : L.geodf.p, x, xs, y, L.nb, L.bnd, cf);
}

template <int DEG, bool PRE>
static void apply_df_geo(const Level& L, const double* x, const float2* xs, double* y, cudaStream_t s) {
  if constexpr (DEG == 2 && PRE) {
    if (L.uniform && L.pair_uniform) {
      static int g = 0;
      if (!g) g = resident_grid(k_apply_lp<KuhnPair>, kBlockLp, 1 << 30);
      k_apply_lp<KuhnPair><<<std::min(g, ceil_div(std::max(L.C / 2, L.nb), kBlockLp)), kBlockLp, 0, s>>>(
          L.C / 2, L.Cs, L.map, L.cdf, x, xs, y, L.nb, L.bnd);
      return;
    }
    if (L.uniform) {
      static int g = 0;
      if (!g) g = resident_grid(k_apply_lp<KuhnTet>, kBlockLp, 1 << 30);
      k_apply_lp<KuhnTet><<<std::min(g, ceil_div(std::max(L.C, L.nb), kBlockLp)), kBlockLp, 0, s>>>(
          L.C, L.Cs, L.map, L.cdf, x, xs, y, L.nb, L.bnd);
      return;
    }
  }
  if (L.uniform)
    apply_df_launch<DEG, false, PRE, true>(L, x, xs, y, ChebFuse<double>{}, s);
  else
    apply_df_launch<DEG, false, PRE, false>(L, x, xs, y, ChebFuse<double>{}, s);
}

template <bool FUSE>
static void apply_df(const Level& L, const double* x, const float2* xs, double* y, const ChebFuse<double>& cf,
                     cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)L.n, s));
  if constexpr (FUSE) {
    if (L.deg == 1)
      apply_df_launch<1, true, false, false>(L, x, nullptr, y, cf, s);
    else
      apply_df_launch<2, true, false, false>(L, x, nullptr, y, cf, s);
  } else if (L.deg == 1) {
    if (xs)
      apply_df_geo<1, true>(L, x, xs, y, s);
    else
      apply_df_geo<1, false>(L, x, nullptr, y, s);
  } else {
    if (xs)
      apply_df_geo<2, true>(L, x, xs, y, s);
    else
      apply_df_geo<2, false>(L, x, nullptr, y, s);
  }
  LAUNCH_CHECK();
}

void launch_apply64_df2(const Level& L, const double* x, double* y, cudaStream_t s) {
  FE_REQUIRE(L.deg == 2 && L.C % 2 == 0, FE_ERR_UNSUPPORTED, "paired float-pair kernel is for P2 (6 N^3 cells)");
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)L.n, s));
  const int P = L.C / 2;
  static int g = 0;
  if (!g) g = resident_grid(k_apply_df2, kBlock, 1 << 30);
  k_apply_df2<<<std::min(g, ceil_div(std::max(P, L.nb), kBlock)), kBlock, 0, s>>>(P, L.Cs, L.map, L.geodf, x, y, L.nb,
                                                                                 L.bnd);
  LAUNCH_CHECK();
}

void launch_apply64_df3(const Level& L, const double* x, double* y, cudaStream_t s) {
  FE_REQUIRE(L.deg == 3, FE_ERR_UNSUPPORTED, "the float-pair P3 kernel needs a degree-3 level");
  CUDA_CHECK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)L.n, s));
  static int g = 0;
  if (!g) g = resident_grid(k_apply_df3<true>, kBlockP3, 1 << 30);
  const int grid = std::min(g, ceil_div(std::max(L.C, L.nb), kBlockP3));
  if (L.uniform)
    k_apply_df3<true><<<grid, kBlockP3, 0, s>>>(L.C, L.Cs, L.map, L.cdf, x, y, L.nb, L.bnd);
  else
    k_apply_df3<false><<<grid, kBlockP3, 0, s>>>(L.C, L.Cs, L.map, L.geodf, x, y, L.nb, L.bnd);
  LAUNCH_CHECK();
}

void launch_apply64_cube_df(const Level& L, const double* x, double* y, cudaStream_t s) {
  apply_cube_df<false>(L, x, y, ChebFuse<double>{}, s);
}

void launch_apply64_df(const Level& L, const double* x, double* y, cudaStream_t s, const float2* xs) {
  apply_df<false>(L, x, xs, y, ChebFuse<double>{}, s);
}

__global__ void k_split_pairs(int n, const double* __restrict__ x, float2* __restrict__ xs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) xs[i] = split_pair(x[i]);
}

void launch_split_pairs(const Level& L, const double* x, cudaStream_t s) {
  FE_REQUIRE(L.xs64.p, FE_ERR_UNSUPPORTED, "this level keeps no float-pair copy of x");
  static int g = 0;
  if (!g) g = resident_grid(k_split_pairs, kBlock, 1 << 30);
  k_split_pairs<<<std::min(g, std::max(1, ceil_div(L.n, kBlock))), kBlock, 0, s>>>(L.n, x, L.xs64.p);
  LAUNCH_CHECK();
}

void launch_apply_cheb64_df(const Level& L, const double* b, double* x, double* y, double* d, double c1, double c2,
                            bool store_d, cudaStream_t s) {
  apply_df<true>(L, x, nullptr, y, ChebFuse<double>{b, L.dinv64, x, d, L.val_tet, L.cnt_tet, c1, c2, store_d ? 1 : 0},
                 s);
}

void launch_apply_cheb64_cube_df(const Level& L, const double* b, double* x, double* y, double* d, double c1,
                                 double c2, bool store_d, cudaStream_t s) {
  apply_cube_df<true>(L, x, y, ChebFuse<double>{b, L.dinv64, x, d, L.val_cube, L.cnt_cube, c1, c2, store_d ? 1 : 0},
                      s);
}
