// Batched GMG-PCG: many independent variable-coefficient Poisson problems on
// meshes of different sizes (P1 and P2 mixed) solved by ONE persistent
// cooperative kernel launch, replayed from a captured CUDA graph.  Each is the
// Poisson problem of the paper's Section 2 (Eqs. 1-4) solved by the
// multigrid-preconditioned method of Section 3; batching them is an extension
// beyond the paper.
//
// Every problem is an ordinary hierarchy (same setup path as the single
// solver: maps, geometric factors, Jacobi diagonals, Chebyshev eigenvalue
// estimates, coarse Cholesky inverse factor).  The persistent kernel walks the
// whole PCG iteration - operator applications, dot products, vector updates
// and every phase of the V-cycle on every level - as a sequence of phases
// separated by grid-wide barriers.  In each phase the CTAs stride over a flat
// list of work items (problem, range, level) built on the host: cell blocks
// for operator applications, dof blocks for vector updates and transfers,
// boundary blocks for the Dirichlet rows and row blocks for the coarse
// triangular products.  Problems stop contributing work once converged
// (per-problem convergence flags).  The cell-block and dof-block sizes and the
// number of CTAs per SM come from a small autotuner that times complete batch
// solves.  Grid barriers are bounded in time: on expiry a CTA raises the abort
// flag, every CTA leaves at its next barrier and the host reports
// FE_ERR_TIMEOUT.  Per-problem dot products use FP64 atomics (the summation
// order is not fixed, so repeated solves agree to rounding, not bitwise).
#include <algorithm>
#include <chrono>
#include <memory>

#include "fe_df.cuh"
#include "fe_reftables.h"

namespace {

constexpr int kMaxLev = 6;
constexpr int kThreads = 256;

struct BLevel {
  int N, n, C, Cs, nb, deg;
  Numbering num;
  const int* map;
  const double* geo;
  const float2* geodf;  // geo as float pairs (double-float operator)
  const float2* cdf;    // with `uniform`: c per cell as a float pair, G = c M (the Kuhn tets' shared matrix)
  int uniform;
  const int4* rtab;     // restriction / prolongation index tables of this (fine) level: the dof of stencil entry e
  const int4* ptab;     // at base point (X, Y, Z) is t.x + K X + t.y Y + t.z Z
  const double* dinv;
  const double* detj;
  const int* bnd;
  double *b, *x, *y, *d, *w;
  double inv_theta, c1, c2;  // two Chebyshev steps: d0 = inv_theta D^-1 r0; d1 = c1 d0 + c2 D^-1 r1
};

struct BProb {
  int nlev, deg;
  BLevel lev[kMaxLev];
  const int* pro_start;
  const int4* pro_off;
  const double* pro_w;
  const int* res_start;
  const int4* res_off;
  const double* res_w;
  int res_margin;  // coarse points this far from the boundary need no bounds checks
  int nci;
  const int* ci;
  const int* dof2int;
  const double* Linv;
  const double* LinvT;
  double *t0, *t1;
  double *xs, *p, *q, *rhs;  // solution, CG direction, A p, load vector
  const double* f;           // nodal right-hand side
};

struct BScal {
  double rz, acc_pq, acc_rr, acc_rz, acc_bb, tol2, rr;
  int active, iters, status, pad;
};

struct GridBar {
  unsigned int count, gen;
  int abort, pad;
};

enum Range { R_CELL = 0, R_DOF = 1, R_BND = 2, R_ROW = 3, R_KINDS = 4 };

struct Work {
  const int4* items;  // (problem, begin, end, level)
  int beg[R_KINDS][kMaxLev], end[R_KINDS][kMaxLev];
};

struct Params {
  const BProb* prob;
  BScal* sc;
  GridBar* bar;
  const double* mref1;
  const double* mref2;
  int nprob, nlev, max_it;
  int df;  // FP64 operator in double-float arithmetic (the library default) or native FP64
  double rtol;
  unsigned long long timeout_ns;
  Work W;
  unsigned long long* ptime;  // profile: ns per (FE_PHASE_*, level), charged by block 0 between barriers; or null
};

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sense-counting grid barrier with a time limit; false once any CTA aborted.
__device__ bool grid_barrier(GridBar* gb, unsigned long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &gb->gen;
    volatile int* vabort = &gb->abort;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&gb->count, 1u);
    if (arrived == gridDim.x - 1) {
      gb->count = 0u;
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const uint64_t t0 = now_ns();
      while (*vgen == g) {
        if (*vabort) break;
        if (now_ns() - t0 > timeout_ns) {
          atomicOr(&gb->abort, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)&gb->abort == 0;
}

// Grid barrier that, when profiling, charges the wall time since the previous
// barrier (as block 0 sees it: the phase and its barrier) to (phase, level).
__device__ __forceinline__ bool pbar(const Params& A, int phase, int level, uint64_t& tlast) {
  const bool ok = grid_barrier(A.bar, A.timeout_ns);
  if (A.ptime && blockIdx.x == 0 && threadIdx.x == 0) {
    const uint64_t t = now_ns();
    A.ptime[phase * kMaxLev + level] += t - tlast;
    tlast = t;
  }
  return ok;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) s += sh[i];
  return s;  // valid in thread 0
}

enum DofOp {
  OP_INIT,         // rhs = 0, xs = 0
  OP_R_FROM_RHS,   // r = rhs, acc_bb += rhs.rhs
  OP_PRE0,         // x = d = inv_theta D^-1 b, y = 0
  OP_CHEB1_PRE,    // d = c1 d + c2 D^-1 (b - y), x += d, w = 0
  OP_PROLONG,      // x += P x_coarse, y = 0
  OP_CHEB0_POST,   // d = inv_theta D^-1 (b - y), x += d, w = 0
  OP_CHEB1_POST,   // d = c1 d + c2 D^-1 (b - w), x += d
  OP_RESTRICT,     // b = P^T (b_fine - w_fine), boundary 0   (items on the coarse level)
  OP_SCATTER,      // x_0 = coarse solution (interior), b_0 (boundary)
  OP_DOT_RZ,       // acc_rz += r.z
  OP_P_FROM_Z,     // p = z, q = 0
  OP_DOT_PQ,       // acc_pq += p.q
  OP_UPDATE_XR,    // alpha = rz/pq; xs += alpha p; r -= alpha q; acc_rr += r.r
  OP_UPDATE_P      // beta = acc_rz/rz; p = z + beta p; q = 0
};

// Prolongation of the coarse x at fine point i through the level's index
// table (each entry's coarse dof an affine form of the base cube).
template <int DEG>
__device__ double prolong_point(const BProb& P, const BLevel& F, const BLevel& Cl, int i) {
  int x, y, z;
  dof_to_lattice(F.num, i, x, y, z);
  constexpr int K2 = 2 * DEG;
  const int cx = x / K2, cy = y / K2, cz = z / K2;
  const int cls = (x - K2 * cx) + K2 * ((y - K2 * cy) + K2 * (z - K2 * cz));
  double s = 0.0;
  const int e1 = P.pro_start[cls + 1];
  for (int e = P.pro_start[cls]; e < e1; ++e) {
    const int4 t = F.ptab[e];
    s += P.pro_w[e] * Cl.x[t.x + cx + t.y * cy + t.z * cz];
  }
  return s;
}

// Restriction of the fine residual b - w at coarse point J through the fine
// level's index table (each stencil entry's dof an affine form of the base
// point; bounds tested only within res_margin of the boundary).  One thread
// per coarse point: in the persistent kernel a block's 256 points in flight
// measured faster (17.9 ms of the 64-problem workload) than 32 points with the
// stencil split over the block's warps (24.5 ms).
template <int DEG>
__device__ double restrict_point(const BProb& P, const BLevel& F, const BLevel& Cl, int J) {
  int X, Y, Z;
  dof_to_lattice(Cl.num, J, X, Y, Z);
  const int m = Cl.num.m;
  if (X == 0 || Y == 0 || Z == 0 || X == m || Y == m || Z == m) return 0.0;
  const int cls = DEG == 2 ? ((X & 1) | ((Y & 1) << 1) | ((Z & 1) << 2)) : 0;
  constexpr int KX = DEG == 2 ? 1 : 2;
  const int mf = F.num.m;
  const bool near = min(min(X, Y), Z) < P.res_margin || max(max(X, Y), Z) > m - P.res_margin;
  double s = 0.0;
  const int e1 = P.res_start[cls + 1];
  for (int e = P.res_start[cls]; e < e1; ++e) {
    const int4 t = F.rtab[e];
    if (near) {
      const int fx = 2 * X + (t.w & 255) - 8, fy = 2 * Y + ((t.w >> 8) & 255) - 8, fz = 2 * Z + ((t.w >> 16) & 255) - 8;
      if (fx < 0 || fy < 0 || fz < 0 || fx > mf || fy > mf || fz > mf) continue;
    }
    const int i = t.x + KX * X + t.y * Y + t.z * Z;
    s += P.res_w[e] * (F.b[i] - F.w[i]);
  }
  return s;
}

// One dof-range phase over the items of `level` (all problems).
__device__ void dof_phase(const Params& A, int level, int op, bool all_problems) {
  const Work& W = A.W;
  for (int it = W.beg[R_DOF][level] + blockIdx.x; it < W.end[R_DOF][level]; it += gridDim.x) {
    const int4 item = W.items[it];
    const BProb& P = A.prob[item.x];
    BScal& S = A.sc[item.x];
    if (!all_problems && !S.active) continue;
    const BLevel& L = P.lev[level];
    double acc = 0.0;
    const double alpha = (op == OP_UPDATE_XR) ? S.rz / S.acc_pq : 0.0;
    const double beta = (op == OP_UPDATE_P) ? S.acc_rz / S.rz : 0.0;
    for (int i = item.y + threadIdx.x; i < item.z; i += blockDim.x) {
      switch (op) {
        case OP_INIT:
          P.rhs[i] = 0.0;
          P.xs[i] = 0.0;
          break;
        case OP_R_FROM_RHS: {
          const double v = P.rhs[i];
          L.b[i] = v;
          acc += v * v;
        } break;
        case OP_PRE0: {
          const double v = L.inv_theta * L.dinv[i] * L.b[i];
          L.d[i] = v;
          L.x[i] = v;
          L.y[i] = 0.0;
        } break;
        case OP_CHEB1_PRE: {
          const double v = L.c1 * L.d[i] + L.c2 * L.dinv[i] * (L.b[i] - L.y[i]);
          L.d[i] = v;
          L.x[i] += v;
          L.w[i] = 0.0;
        } break;
        case OP_PROLONG: {
          const double v = P.deg == 1 ? prolong_point<1>(P, L, P.lev[level - 1], i)
                                      : prolong_point<2>(P, L, P.lev[level - 1], i);
          L.x[i] += v;
          L.y[i] = 0.0;
        } break;
        case OP_CHEB0_POST: {
          const double v = L.inv_theta * L.dinv[i] * (L.b[i] - L.y[i]);
          L.d[i] = v;
          L.x[i] += v;
          L.w[i] = 0.0;
        } break;
        case OP_CHEB1_POST: {
          const double v = L.c1 * L.d[i] + L.c2 * L.dinv[i] * (L.b[i] - L.w[i]);
          L.d[i] = v;
          L.x[i] += v;
        } break;
        case OP_RESTRICT:
          L.b[i] = P.deg == 1 ? restrict_point<1>(P, P.lev[level + 1], L, i)
                              : restrict_point<2>(P, P.lev[level + 1], L, i);
          break;
        case OP_SCATTER: {
          const int k = P.dof2int[i];
          L.x[i] = k >= 0 ? P.t0[k] : L.b[i];
        } break;
        case OP_DOT_RZ:
          acc += L.b[i] * L.x[i];
          break;
        case OP_P_FROM_Z:
          P.p[i] = L.x[i];
          P.q[i] = 0.0;
          break;
        case OP_DOT_PQ:
          acc += P.p[i] * P.q[i];
          break;
        case OP_UPDATE_XR: {
          P.xs[i] += alpha * P.p[i];
          const double r = L.b[i] - alpha * P.q[i];
          L.b[i] = r;
          acc += r * r;
        } break;
        case OP_UPDATE_P:
          P.p[i] = L.x[i] + beta * P.p[i];
          P.q[i] = 0.0;
          break;
      }
    }
    if (op == OP_R_FROM_RHS || op == OP_DOT_RZ || op == OP_DOT_PQ || op == OP_UPDATE_XR) {
      const double s = block_sum(acc);
      if (threadIdx.x == 0) {
        double* dst = op == OP_R_FROM_RHS ? &S.acc_bb : op == OP_DOT_RZ ? &S.acc_rz : op == OP_DOT_PQ ? &S.acc_pq : &S.acc_rr;
        atomicAdd(dst, s);
      }
    }
  }
}

enum VecSel { V_X_TO_Y, V_X_TO_W, V_P_TO_Q, V_F_TO_RHS };

template <int DEG>
__device__ void apply_cells(const Params& A, const BProb& P, const BLevel& L, int c0, int c1, int sel) {
  constexpr int ND = DEG == 1 ? 4 : 10;
  const double* in = sel == V_P_TO_Q ? P.p : sel == V_F_TO_RHS ? P.f : L.x;
  double* out = sel == V_X_TO_Y ? L.y : sel == V_X_TO_W ? L.w : sel == V_P_TO_Q ? P.q : P.rhs;
  const double* mref = DEG == 1 ? A.mref1 : A.mref2;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    int idx[ND];
    double u[ND], o[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) idx[j] = L.map[(size_t)j * L.Cs + c];
    if (sel == V_F_TO_RHS) {  // mass: all dofs, no boundary elimination
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        if (idx[j] < 0) idx[j] = -1 - idx[j];
        u[j] = in[idx[j]];
      }
      const double s = L.detj[c];
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        double a = 0.0;
#pragma unroll
        for (int j = 0; j < ND; ++j) a += mref[i * ND + j] * u[j];
        atomicAdd(out + idx[i], s * a);
      }
    } else if (A.df) {
#pragma unroll
      for (int j = 0; j < ND; ++j) u[j] = idx[j] >= 0 ? in[idx[j]] : 0.0;
      const int emax = fe_df::block_exponent<ND>(u);
      fe_df::DF ud[ND], gd[6], od[ND];
#pragma unroll
      for (int j = 0; j < ND; ++j) ud[j] = fe_df::split_scaled(u[j], emax);
      if (emax == 0x7FF) ud[0] = fe_df::DF(__int_as_float(0x7fc00000), 0.0f);
      if constexpr (DEG == 2) {
        if (L.uniform) {
          // the element matrix is 4 c K: exact fixed-point limbs of x' = c 2^(126 - ec) ud (as in k_apply_df)
          const float2 v = L.cdf[c];
          const unsigned int cb = __float_as_uint(v.x);
          const int ec = (int)((cb >> 23) & 0xFFu);
          const fe_df::DF cs(__uint_as_float((cb & 0x807FFFFFu) | (126u << 23)),
                             __fmul_rn(v.y, __uint_as_float((unsigned int)(253 - ec) << 23)));
          float la[10], lb[10], lc[10];
          fe_df::p2_kuhn_split(ud, cs, la, lb, lc);
          const int w = ec + emax - 124;
          fe_df::p2_kuhn_apply(la, lb, lc, [&](int j, fe_df::DF t) {
            if (idx[j] >= 0) atomicAdd(out + idx[j], fe_df::widen_scaled(t.hi, w) + fe_df::widen_scaled(t.lo, w));
          });
          continue;
        }
      }
      if (L.uniform) {
        const float2 v = L.cdf[c];
        fe_df::element_df_m<DEG>(ud, fe_df::DF(v.x, v.y), od);
      } else {
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const float2 v = L.geodf[(size_t)a * L.Cs + c];
          gd[a] = fe_df::DF(v.x, v.y);
        }
        fe_df::element_df<DEG>(ud, gd, od);
      }
#pragma unroll
      for (int j = 0; j < ND; ++j)
        if (idx[j] >= 0)
          atomicAdd(out + idx[j], fe_df::widen_scaled(od[j].hi, emax) + fe_df::widen_scaled(od[j].lo, emax));
    } else {
#pragma unroll
      for (int j = 0; j < ND; ++j) u[j] = idx[j] >= 0 ? in[idx[j]] : 0.0;
      double g[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) g[a] = L.geo[(size_t)a * L.Cs + c];
      element_apply<DEG, double>(u, g, o);
#pragma unroll
      for (int j = 0; j < ND; ++j)
        if (idx[j] >= 0) atomicAdd(out + idx[j], o[j]);
    }
  }
}

// Operator application on `level`: cell items (atomic scatter) and boundary
// items (identity rows; for the load vector, zero Dirichlet rows) in one phase.
__device__ void apply_phase(const Params& A, int level, int sel, bool all_problems) {
  const Work& W = A.W;
  const int nc = W.end[R_CELL][level] - W.beg[R_CELL][level];
  const int nbi = W.end[R_BND][level] - W.beg[R_BND][level];
  for (int t = blockIdx.x; t < nc + (sel == V_F_TO_RHS ? 0 : nbi); t += gridDim.x) {
    const bool is_cell = t < nc;
    const int4 item = W.items[is_cell ? W.beg[R_CELL][level] + t : W.beg[R_BND][level] + (t - nc)];
    const BProb& P = A.prob[item.x];
    if (!all_problems && !A.sc[item.x].active) continue;
    const BLevel& L = P.lev[level];
    if (is_cell) {
      if (P.deg == 1)
        apply_cells<1>(A, P, L, item.y, item.z, sel);
      else
        apply_cells<2>(A, P, L, item.y, item.z, sel);
    } else {
      const double* in = sel == V_P_TO_Q ? P.p : L.x;
      double* out = sel == V_X_TO_Y ? L.y : sel == V_X_TO_W ? L.w : P.q;
      for (int k = item.y + threadIdx.x; k < item.z; k += blockDim.x) out[L.bnd[k]] = in[L.bnd[k]];
    }
  }
}

__device__ void zero_rhs_boundary(const Params& A, int level) {
  const Work& W = A.W;
  for (int it = W.beg[R_BND][level] + blockIdx.x; it < W.end[R_BND][level]; it += gridDim.x) {
    const int4 item = W.items[it];
    const BProb& P = A.prob[item.x];
    const BLevel& L = P.lev[level];
    for (int k = item.y + threadIdx.x; k < item.z; k += blockDim.x) P.rhs[L.bnd[k]] = 0.0;
  }
}

// Coarse solve phases over row items: 0 gather, 1 t1 = L^-1 t0, 2 t0 = L^-T t1.
__device__ void coarse_phase(const Params& A, int which) {
  const Work& W = A.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int it = W.beg[R_ROW][0] + blockIdx.x; it < W.end[R_ROW][0]; it += gridDim.x) {
    const int4 item = W.items[it];
    const BProb& P = A.prob[item.x];
    if (!A.sc[item.x].active) continue;
    if (which == 0) {
      for (int r = item.y + threadIdx.x; r < item.z; r += blockDim.x) P.t0[r] = P.lev[0].b[P.ci[r]];
      continue;
    }
    const int n = P.nci;
    for (int r = item.y + warp; r < item.z; r += nw) {
      const double* M = (which == 1 ? P.Linv : P.LinvT) + (size_t)r * n;
      const double* in = which == 1 ? P.t0 : P.t1;
      const int j0 = which == 1 ? 0 : r, j1 = which == 1 ? r + 1 : n;
      double s = 0.0;
      for (int j = j0 + lane; j < j1; j += 32) s += M[j] * in[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) (which == 1 ? P.t1 : P.t0)[r] = s;
    }
  }
}

__device__ bool vcycle(const Params& A, uint64_t& tl) {
  const int fine = A.nlev - 1;
  for (int l = fine; l >= 1; --l) {
    dof_phase(A, l, OP_PRE0, false);
    if (!pbar(A, FE_PHASE_SMOOTH, l, tl)) return false;
    apply_phase(A, l, V_X_TO_Y, false);
    if (!pbar(A, FE_PHASE_SMOOTH, l, tl)) return false;
    dof_phase(A, l, OP_CHEB1_PRE, false);
    if (!pbar(A, FE_PHASE_SMOOTH, l, tl)) return false;
    apply_phase(A, l, V_X_TO_W, false);
    if (!pbar(A, FE_PHASE_APPLY, l, tl)) return false;
    dof_phase(A, l - 1, OP_RESTRICT, false);
    if (!pbar(A, FE_PHASE_TRANSFER, l, tl)) return false;
  }
  for (int k = 0; k < 3; ++k) {
    coarse_phase(A, k);
    if (!pbar(A, FE_PHASE_COARSE, 0, tl)) return false;
  }
  dof_phase(A, 0, OP_SCATTER, false);
  if (!pbar(A, FE_PHASE_COARSE, 0, tl)) return false;
  for (int l = 1; l <= fine; ++l) {
    dof_phase(A, l, OP_PROLONG, false);
    if (!pbar(A, FE_PHASE_TRANSFER, l, tl)) return false;
    apply_phase(A, l, V_X_TO_Y, false);
    if (!pbar(A, FE_PHASE_SMOOTH, l, tl)) return false;
    dof_phase(A, l, OP_CHEB0_POST, false);
    if (!pbar(A, FE_PHASE_SMOOTH, l, tl)) return false;
    apply_phase(A, l, V_X_TO_W, false);
    if (!pbar(A, FE_PHASE_SMOOTH, l, tl)) return false;
    dof_phase(A, l, OP_CHEB1_POST, false);
    if (!pbar(A, FE_PHASE_SMOOTH, l, tl)) return false;
  }
  return true;
}

__device__ bool any_active(const Params& A) {
  for (int p = 0; p < A.nprob; ++p)
    if (((volatile int*)&A.sc[p].active)[0]) return true;
  return false;
}

__global__ void __launch_bounds__(kThreads) k_batched_pcg(Params A) {
  const int fine = A.nlev - 1;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t tl = now_ns();  // profile clock of block 0
  // ---- setup: b = M f (Dirichlet rows 0), r = b, bb, x = 0
  dof_phase(A, fine, OP_INIT, true);
  if (gtid < A.nprob) {
    BScal& S = A.sc[gtid];
    S.acc_pq = S.acc_rr = S.acc_rz = S.acc_bb = 0.0;
    S.iters = 0;
    S.status = 0;
    S.active = 1;
  }
  if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
  apply_phase(A, fine, V_F_TO_RHS, true);
  if (!pbar(A, FE_PHASE_APPLY, fine, tl)) return;
  zero_rhs_boundary(A, fine);
  if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
  dof_phase(A, fine, OP_R_FROM_RHS, true);
  if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
  if (gtid < A.nprob) {
    BScal& S = A.sc[gtid];
    S.tol2 = A.rtol * A.rtol * S.acc_bb;
    S.rr = S.acc_bb;
    S.active = S.acc_bb > 0.0;
  }
  if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
  // ---- z = V(r), rz = r.z, p = z
  if (!vcycle(A, tl)) return;
  dof_phase(A, fine, OP_DOT_RZ, false);
  if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
  dof_phase(A, fine, OP_P_FROM_Z, false);
  if (gtid < A.nprob) {
    BScal& S = A.sc[gtid];
    S.rz = S.acc_rz;
    S.acc_rz = 0.0;
  }
  if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
  // ---- PCG iterations
  while (true) {
    apply_phase(A, fine, V_P_TO_Q, false);
    if (!pbar(A, FE_PHASE_APPLY, fine, tl)) return;
    dof_phase(A, fine, OP_DOT_PQ, false);
    if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
    dof_phase(A, fine, OP_UPDATE_XR, false);
    if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
    if (gtid < A.nprob) {
      BScal& S = A.sc[gtid];
      if (S.active) {
        S.iters += 1;
        S.rr = S.acc_rr;
        if (!isfinite(S.rr)) {
          S.status = FE_ERR_NAN;
          S.active = 0;
        } else if (S.rr <= S.tol2) {
          S.active = 0;
        } else if (S.iters >= A.max_it) {
          S.status = FE_ERR_NO_CONVERGENCE;
          S.active = 0;
        }
      }
      S.acc_pq = 0.0;
      S.acc_rr = 0.0;
    }
    if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
    if (!any_active(A)) break;
    if (!vcycle(A, tl)) return;
    dof_phase(A, fine, OP_DOT_RZ, false);
    if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
    dof_phase(A, fine, OP_UPDATE_P, false);
    if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
    if (gtid < A.nprob) {
      BScal& S = A.sc[gtid];
      if (S.active) S.rz = S.acc_rz;
      S.acc_rz = 0.0;
    }
    if (!pbar(A, FE_PHASE_BLAS1, fine, tl)) return;
  }
}

}  // namespace

// ================================================================== host
struct Schedule {
  int cell_block = 2048, dof_block = 8192, ctas_per_sm = 2;
};

struct fe_batch {
  std::vector<fe_hierarchy*> hs;
  int nlev = 0;
  DBuf<BProb> dprob;
  DBuf<BScal> dsc;
  DBuf<GridBar> dbar;
  DBuf<double> mref1, mref2;
  DBuf<int4> items;
  DBuf<unsigned long long> ptime;  // [FE_NUM_PHASES][kMaxLev] profile clock (ns)
  Work work{};
  Schedule sched;
  bool tuned = false;
  int sms = 148;
  std::vector<const double*> f_ptrs;
  std::vector<double*> u_ptrs;
  cudaGraphExec_t gexec = nullptr;
  Params gparams{};
  int ggrid = 0;
  ~fe_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto* h : hs) hierarchy_destroy(h);
  }
};

namespace {

void build_items(fe_batch* B) {
  std::vector<int4> it;
  Work W{};
  const int P = (int)B->hs.size();
  auto blocks = [&](int kind, int l, int per_item, auto count_of) {
    W.beg[kind][l] = (int)it.size();
    for (int p = 0; p < P; ++p) {
      const int n = count_of(B->hs[p], l);
      for (int s = 0; s < n; s += per_item) it.push_back(make_int4(p, s, std::min(n, s + per_item), l));
    }
    W.end[kind][l] = (int)it.size();
  };
  for (int l = 0; l < B->nlev; ++l) {
    blocks(R_CELL, l, B->sched.cell_block, [](fe_hierarchy* h, int l) { return h->L[l].C; });
    blocks(R_DOF, l, B->sched.dof_block, [](fe_hierarchy* h, int l) { return h->L[l].n; });
    blocks(R_BND, l, B->sched.dof_block, [](fe_hierarchy* h, int l) { return h->L[l].nb; });
  }
  blocks(R_ROW, 0, 64, [](fe_hierarchy* h, int) { return h->cs.nci; });
  B->items.alloc(it.size());
  CUDA_CHECK(cudaMemcpy(B->items.p, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
  W.items = B->items.p;
  B->work = W;
}

void fill_problems(fe_batch* B, double cheb_lo, double cheb_hi) {
  std::vector<BProb> hp(B->hs.size());
  for (size_t p = 0; p < B->hs.size(); ++p) {
    fe_hierarchy* h = B->hs[p];
    BProb& P = hp[p];
    P.nlev = h->nlev;
    P.deg = h->deg;
    for (int l = 0; l < h->nlev; ++l) {
      Level& L = h->L[l];
      BLevel& D = P.lev[l];
      D.N = L.N;
      D.n = L.n;
      D.C = L.C;
      D.Cs = L.Cs;
      D.nb = L.nb;
      D.deg = L.deg;
      D.num = L.num;
      D.map = L.map;
      D.geo = L.geo64;
      D.geodf = L.geodf;
      D.cdf = L.cdf;
      D.uniform = L.uniform;
      D.rtab = L.rtab;
      D.ptab = L.ptab;
      D.dinv = L.dinv64;
      D.detj = L.detj;
      D.bnd = L.bnd;
      D.b = L.b64;
      D.x = L.x64;
      D.y = L.y64;
      D.d = L.d64;
      D.w = L.w64;
      const double a = cheb_lo * L.lmax, bm = cheb_hi * L.lmax;
      const double theta = 0.5 * (bm + a), delta = 0.5 * (bm - a), sigma = theta / delta;
      const double rho0 = 1.0 / sigma, rho1 = 1.0 / (2.0 * sigma - rho0);
      D.inv_theta = 1.0 / theta;
      D.c1 = rho1 * rho0;
      D.c2 = 2.0 * rho1 / delta;
    }
    P.pro_start = h->tt.pro_start;
    P.pro_off = h->tt.pro_off;
    P.pro_w = h->tt.pro_w;
    P.res_start = h->tt.res_start;
    P.res_off = h->tt.res_off;
    P.res_w = h->tt.res_w;
    P.res_margin = h->tt.res_margin;
    P.nci = h->cs.nci;
    P.ci = h->cs.ci;
    P.dof2int = h->cs.dof2int;
    P.Linv = h->cs.Linv;
    P.LinvT = h->cs.LinvT;
    P.t0 = h->cs.t0;
    P.t1 = h->cs.t1;
    P.xs = h->x;
    P.p = h->p;
    P.q = h->q;
    P.rhs = h->b;
    P.f = B->f_ptrs.empty() ? nullptr : B->f_ptrs[p];
  }
  CUDA_CHECK(cudaMemcpy(B->dprob.p, hp.data(), sizeof(BProb) * hp.size(), cudaMemcpyHostToDevice));
}

int coop_grid(fe_batch* B) {
  int occ = 0;
  CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched_pcg, kThreads, 0));
  FE_REQUIRE(occ >= 1, FE_ERR_UNSUPPORTED, "persistent batched kernel does not fit on an SM");
  return B->sms * std::min(occ, B->sched.ctas_per_sm);
}

void launch_persistent(fe_batch* B, const Params& A, int grid, cudaStream_t s) {
  CUDA_CHECK(cudaMemsetAsync(B->dbar.p, 0, sizeof(GridBar), s));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_batched_pcg, A));
  fe_count_launch();
}

Params make_params(fe_batch* B, const fe_solver_opts& o) {
  Params A{};
  A.prob = B->dprob;
  A.sc = B->dsc;
  A.bar = B->dbar;
  A.mref1 = B->mref1;
  A.mref2 = B->mref2;
  A.nprob = (int)B->hs.size();
  A.nlev = B->nlev;
  A.df = B->hs[0]->f64_mode != FE_F64_NATIVE;
  A.max_it = o.max_it;
  A.rtol = o.rtol;
  A.timeout_ns = o.wait_timeout_us > 0 ? (unsigned long long)o.wait_timeout_us * 1000ull : 5000000000ull;
  A.W = B->work;
  A.ptime = o.profile ? B->ptime.p : nullptr;
  return A;
}

// One batch solve; returns the host wall time in ms.
double run_solve(fe_batch* B, const fe_solver_opts& o, cudaStream_t s) {
  const Params A = make_params(B, o);
  const int grid = coop_grid(B);
  const auto t0 = std::chrono::steady_clock::now();
  if (o.profile) {  // phase clock: a direct launch (the counters are zeroed first)
    B->ptime.alloc((size_t)FE_NUM_PHASES * kMaxLev);
    CUDA_CHECK(cudaMemsetAsync(B->ptime.p, 0, sizeof(unsigned long long) * FE_NUM_PHASES * kMaxLev, s));
    launch_persistent(B, make_params(B, o), grid, s);
  } else if (o.use_graph) {
    const bool same = B->gexec && B->ggrid == grid && memcmp(&B->gparams, &A, sizeof(Params)) == 0;
    if (!same) {
      if (B->gexec) cudaGraphExecDestroy(B->gexec);
      B->gexec = nullptr;
      cudaStream_t cs;
      CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t g;
      CUDA_CHECK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      CUDA_CHECK(cudaMemsetAsync(B->dbar.p, 0, sizeof(GridBar), cs));
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(kThreads);
      cfg.stream = cs;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      const cudaError_t le = cudaLaunchKernelEx(&cfg, k_batched_pcg, A);
      const cudaError_t ce = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      CUDA_CHECK(le);
      CUDA_CHECK(ce);
      CUDA_CHECK(cudaGraphInstantiate(&B->gexec, g, 0));
      cudaGraphDestroy(g);
      B->gparams = A;
      B->ggrid = grid;
    }
    CUDA_CHECK(cudaGraphLaunch(B->gexec, s));
    fe_count_launch();
  } else {
    launch_persistent(B, A, grid, s);
  }
  CUDA_CHECK(cudaStreamSynchronize(s));
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void autotune(fe_batch* B, const fe_solver_opts& o, cudaStream_t s) {
  const int cells[] = {1024, 4096};
  const int ctas[] = {1, 2, 4};
  Schedule best = B->sched;
  double best_ms = 1e300;
  fe_solver_opts t = o;
  t.use_graph = 0;
  for (int cb : cells)
    for (int cp : ctas) {
      B->sched.cell_block = cb;
      B->sched.dof_block = 4 * cb;
      B->sched.ctas_per_sm = cp;
      build_items(B);
      run_solve(B, t, s);  // warm
      const double ms = run_solve(B, t, s);
      GridBar hb;
      CUDA_CHECK(cudaMemcpy(&hb, B->dbar.p, sizeof(GridBar), cudaMemcpyDeviceToHost));
      if (hb.abort == 0 && ms < best_ms) {
        best_ms = ms;
        best = B->sched;
      }
    }
  B->sched = best;
  build_items(B);
  B->tuned = true;
}

}  // namespace

extern "C" {

int fe_batch_create(int nprob, const int* N0, const int* nrefine, const int* degree, fe_batch** out) {
  try {
    FE_REQUIRE(out && N0 && nrefine && degree && nprob >= 1, FE_ERR_ARG, "invalid batch arguments");
    *out = nullptr;
    std::unique_ptr<fe_batch> B(new fe_batch());
    for (int p = 0; p < nprob; ++p) {
      FE_REQUIRE(nrefine[p] >= 1 && nrefine[p] + 1 <= kMaxLev, FE_ERR_ARG, "each problem needs 2..6 levels");
      FE_REQUIRE(p == 0 || nrefine[p] == nrefine[0], FE_ERR_UNSUPPORTED, "all problems of a batch need the same level count");
      FE_REQUIRE(degree[p] == 1 || degree[p] == 2, FE_ERR_UNSUPPORTED, "the batched solver is for P1/P2");
      B->hs.push_back(hierarchy_create(N0[p], nrefine[p], degree[p]));
    }
    B->nlev = nrefine[0] + 1;
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, dev));
    B->dprob.alloc(nprob);
    B->dsc.alloc(nprob);
    B->dbar.alloc(1);
    CUDA_CHECK(cudaMemset(B->dsc.p, 0, sizeof(BScal) * nprob));
    double m1[16], m2[100];
    fe_ref::mass_tables(m1, m2);
    B->mref1.alloc(16);
    B->mref2.alloc(100);
    CUDA_CHECK(cudaMemcpy(B->mref1.p, m1, sizeof(m1), cudaMemcpyHostToDevice));
    CUDA_CHECK(cudaMemcpy(B->mref2.p, m2, sizeof(m2), cudaMemcpyHostToDevice));
    build_items(B.get());
    *out = B.release();
  } catch (const FeError& e) {
    fe_set_error(e.msg);
    return e.code;
  } catch (...) {
    fe_set_error("unexpected C++ exception");
    return FE_ERR_CUDA;
  }
  return FE_OK;
}

void fe_batch_destroy(fe_batch* B) {
  if (!B) return;
  cudaDeviceSynchronize();
  delete B;
}

int fe_batch_hierarchy(fe_batch* B, int p, fe_hierarchy** h) {
  if (!B || !h || p < 0 || p >= (int)B->hs.size()) {
    fe_set_error("invalid batch problem index");
    return FE_ERR_ARG;
  }
  *h = B->hs[p];
  return FE_OK;
}

int fe_solve_batched(fe_batch* B, const double* const* f_nodal, double* const* u, const fe_solver_opts* opts,
                     fe_solve_stats* stats, void* stream) {
  try {
    FE_REQUIRE(B && f_nodal && u, FE_ERR_ARG, "null argument");
    fe_solver_opts o;
    fe_default_opts(&o);
    if (opts) o = *opts;
    FE_REQUIRE(o.cheb_steps == 2, FE_ERR_UNSUPPORTED, "the batched solver runs 2 Chebyshev steps per smoothing");
    FE_REQUIRE(o.precision == FE_PREC_F64 && o.precond == FE_PC_GMG, FE_ERR_UNSUPPORTED,
               "the batched solver is FP64 GMG-PCG");
    FE_REQUIRE(o.rtol >= 0 && o.max_it >= 1 && o.cheb_hi > o.cheb_lo && o.cheb_lo > 0, FE_ERR_ARG, "invalid options");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int P = (int)B->hs.size();
    B->f_ptrs.assign(f_nodal, f_nodal + P);
    B->u_ptrs.assign(u, u + P);
    cudaPointerAttributes a;
    for (int p = 0; p < P; ++p) {
      FE_REQUIRE(f_nodal[p] && u[p], FE_ERR_ARG, "null problem vector");
      FE_REQUIRE(cudaPointerGetAttributes(&a, f_nodal[p]) == cudaSuccess && a.type == cudaMemoryTypeDevice, FE_ERR_ARG,
                 "batched vectors must be device pointers");
      FE_REQUIRE(cudaPointerGetAttributes(&a, u[p]) == cudaSuccess && a.type == cudaMemoryTypeDevice, FE_ERR_ARG,
                 "batched vectors must be device pointers");
    }
    fill_problems(B, o.cheb_lo, o.cheb_hi);
    if (!B->tuned && o.use_graph && !o.profile) autotune(B, o, s);
    const double ms = run_solve(B, o, s);
    std::vector<unsigned long long> pt;
    if (o.profile) {
      pt.resize((size_t)FE_NUM_PHASES * kMaxLev);
      CUDA_CHECK(cudaMemcpy(pt.data(), B->ptime.p, sizeof(unsigned long long) * pt.size(), cudaMemcpyDeviceToHost));
    }
    GridBar hb;
    CUDA_CHECK(cudaMemcpy(&hb, B->dbar.p, sizeof(GridBar), cudaMemcpyDeviceToHost));
    FE_REQUIRE(hb.abort == 0, FE_ERR_TIMEOUT, "a grid barrier of the persistent batched kernel timed out");
    std::vector<BScal> hs(P);
    CUDA_CHECK(cudaMemcpy(hs.data(), B->dsc.p, sizeof(BScal) * P, cudaMemcpyDeviceToHost));
    int worst = FE_OK;
    for (int p = 0; p < P; ++p) {
      const Level& F = B->hs[p]->L.back();
      CUDA_CHECK(cudaMemcpyAsync(u[p], B->hs[p]->x.p, sizeof(double) * F.n, cudaMemcpyDeviceToDevice, s));
      if (stats) {
        fe_solve_stats& st = stats[p];
        st = fe_solve_stats{};
        st.iterations = hs[p].iters;
        st.outer_iterations = 1;
        st.bnorm = std::sqrt(hs[p].acc_bb);
        st.rel_residual = hs[p].acc_bb > 0 ? std::sqrt(hs[p].rr / hs[p].acc_bb) : 0.0;
        st.solve_ms = ms;
        st.fine_applies_f64 = hs[p].iters;
        if (o.profile) {  // the persistent launch's wall time by phase and level, the same for every problem
          st.levels_timed = B->nlev;
          for (int ph = 0; ph < FE_NUM_PHASES; ++ph)
            for (int l = 0; l < B->nlev && l < FE_MAX_LEVELS; ++l) st.phase_ms[ph][l] = 1e-6 * (double)pt[ph * kMaxLev + l];
        }
      }
      if (hs[p].status != 0 && worst == FE_OK) worst = hs[p].status;
    }
    CUDA_CHECK(cudaStreamSynchronize(s));
    if (worst == FE_ERR_NAN) FE_FAIL(FE_ERR_NAN, "a residual norm of the batch is not finite");
    if (worst == FE_ERR_NO_CONVERGENCE) FE_FAIL(FE_ERR_NO_CONVERGENCE, "a problem of the batch reached max_it");
  } catch (const FeError& e) {
    fe_set_error(e.msg);
    return e.code;
  } catch (...) {
    fe_set_error("unexpected C++ exception");
    return FE_ERR_CUDA;
  }
  return FE_OK;
}

int fe_batch_schedule(const fe_batch* B, int* cell_block, int* dof_block, int* ctas_per_sm) {
  if (!B) {
    fe_set_error("null batch");
    return FE_ERR_ARG;
  }
  if (cell_block) *cell_block = B->sched.cell_block;
  if (dof_block) *dof_block = B->sched.dof_block;
  if (ctas_per_sm) *ctas_per_sm = B->sched.ctas_per_sm;
  return FE_OK;
}

}  // extern "C"
