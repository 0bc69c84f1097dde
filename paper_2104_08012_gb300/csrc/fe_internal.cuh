// Internal declarations of the GB300 finite element library: error handling,
// device buffers, the dof numbering, the per-level device data and the
// element kernels' arithmetic (the P1/P2 element actions of the bilinear form
// of the paper's Section 2, Eq. 4).  Not part of the public ABI (see
// include/fe.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "fe.h"

// ----------------------------------------------------------------- errors ---
struct FeError {
  int code;
  std::string msg;
};

#define FE_FAIL(code_, msg_) throw FeError{(code_), std::string(msg_)}
#define FE_REQUIRE(cond_, code_, msg_) \
  do {                                 \
    if (!(cond_)) FE_FAIL(code_, msg_); \
  } while (0)
#define CUDA_CHECK(x)                                                                               \
  do {                                                                                              \
    cudaError_t e_ = (x);                                                                           \
    if (e_ != cudaSuccess) {                                                                        \
      throw FeError{e_ == cudaErrorMemoryAllocation ? FE_ERR_NOMEM : FE_ERR_CUDA,                   \
                    std::string(#x) + " failed: " + cudaGetErrorString(e_) + " (" + __FILE__ + ":" + \
                        std::to_string(__LINE__) + ")"};                                            \
    }                                                                                               \
  } while (0)
// Every kernel launch is followed by LAUNCH_CHECK(), which also counts it
// (launches recorded into a graph under capture are counted at replay).
void fe_count_launch();
#define LAUNCH_CHECK()                \
  do {                                \
    CUDA_CHECK(cudaGetLastError());   \
    fe_count_launch();                \
  } while (0)

void fe_set_error(const std::string& msg);

// ------------------------------------------------------- device buffers ---
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    if (count == n && p) return;
    release();
    if (count == 0) return;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      throw FeError{FE_ERR_NOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                      " bytes failed: " + cudaGetErrorString(e)};
    }
    n = count;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  operator T*() const { return p; }
};

// ------------------------------------------------------------ numbering ---
// Global dof numbering of the (deg*N)-lattice, see include/fe.h.  P1: one
// class, lexicographic.  P2: 8 parity classes in the order
// (000),(100),(010),(001),(110),(101),(011),(111).
struct Numbering {
  int N, deg, m;  // cubes per axis, degree, lattice extent m = deg*N
  int off[9];     // first dof of each class, off[8] = n (P1: off[1] = n)
  int sx[8], sy[8], sz[8];
};

Numbering make_numbering(int N, int deg);

__host__ __device__ inline int class_parity_x(int c) { return (c == 1 || c == 4 || c == 5 || c == 7) ? 1 : 0; }
__host__ __device__ inline int class_parity_y(int c) { return (c == 2 || c == 4 || c == 6 || c == 7) ? 1 : 0; }
__host__ __device__ inline int class_parity_z(int c) { return (c == 3 || c == 5 || c == 6 || c == 7) ? 1 : 0; }

__host__ __device__ inline int lattice_to_dof(const Numbering& nb, int x, int y, int z) {
  if (nb.deg != 2) return x + (nb.m + 1) * (y + (nb.m + 1) * z);  // P1, P3: lexicographic
  const int code = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
  // code (px + 2py + 4pz) -> class index in the order above
  const int c = (code == 3) ? 4 : (code == 4) ? 3 : code;
  return nb.off[c] + (x >> 1) + nb.sx[c] * ((y >> 1) + nb.sy[c] * (z >> 1));
}

__host__ __device__ inline void dof_to_lattice(const Numbering& nb, int i, int& x, int& y, int& z) {
  if (nb.deg != 2) {
    const int n1 = nb.m + 1;
    x = i % n1;
    const int r = i / n1;
    y = r % n1;
    z = r / n1;
    return;
  }
  int c = 0;
#pragma unroll
  for (int k = 1; k < 8; ++k)
    if (i >= nb.off[k]) c = k;
  int r = i - nb.off[c];
  const int ax = r % nb.sx[c];
  r /= nb.sx[c];
  const int ay = r % nb.sy[c];
  const int az = r / nb.sy[c];
  x = 2 * ax + class_parity_x(c);
  y = 2 * ay + class_parity_y(c);
  z = 2 * az + class_parity_z(c);
}

// Kuhn simplex t of a cube: corners origin, +e[p0], +e[p0]+e[p1], +(1,1,1).
__host__ __device__ inline void kuhn_perm(int t, int& p0, int& p1, int& p2) {
  // (0,1,2),(0,2,1),(1,0,2),(1,2,0),(2,0,1),(2,1,0)
  p0 = t >> 1;
  const int lo = (p0 == 0) ? 1 : 0;
  const int hi = (p0 == 2) ? 1 : 2;
  p1 = (t & 1) ? hi : lo;
  p2 = 3 - p0 - p1;
}

// Local lattice index, inside the (k+1)^3 points of a cube, of local dof j of
// Kuhn tet t (vertices first, then the edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)).
__host__ __device__ constexpr int kuhn_p0(int t) { return t >> 1; }
__host__ __device__ constexpr int kuhn_p1(int t) {
  return (t & 1) ? ((t >> 1) == 2 ? 1 : 2) : ((t >> 1) == 0 ? 1 : 0);
}
__host__ __device__ constexpr int kuhn_vmask(int t, int k) {
  return k == 0 ? 0 : k == 1 ? (1 << kuhn_p0(t)) : k == 2 ? ((1 << kuhn_p0(t)) | (1 << kuhn_p1(t))) : 7;
}
__host__ __device__ constexpr int edge_a(int j) { return j <= 6 ? 0 : (j <= 8 ? 1 : 2); }
__host__ __device__ constexpr int edge_b(int j) { return j <= 6 ? j - 3 : (j <= 8 ? j - 5 : 3); }
__host__ __device__ constexpr int cube_local(int deg, int t, int j) {
  return deg == 1 ? kuhn_vmask(t, j)
                  : (j < 4 ? 2 * ((kuhn_vmask(t, j) & 1) + 3 * ((kuhn_vmask(t, j) >> 1) & 1) + 9 * ((kuhn_vmask(t, j) >> 2) & 1))
                           : ((kuhn_vmask(t, edge_a(j)) & 1) + (kuhn_vmask(t, edge_b(j)) & 1)) +
                                 3 * (((kuhn_vmask(t, edge_a(j)) >> 1) & 1) + ((kuhn_vmask(t, edge_b(j)) >> 1) & 1)) +
                                 9 * (((kuhn_vmask(t, edge_a(j)) >> 2) & 1) + ((kuhn_vmask(t, edge_b(j)) >> 2) & 1)));
}

// ------------------------------------------------- Chebyshev update ---
// One step of the Chebyshev semi-iteration on D^-1 A for one dof:
// d = c1 d + c2 D^-1 (b - y), x += d (c1 = 0: the previous d is not read).
// The same function serves the stand-alone vector kernel and the operator
// kernels that fuse the update (ChebFuse), so both give the same arithmetic.
template <typename T>
__device__ __forceinline__ void cheb_update(int i, T yi, const T* b, const T* dinv, T* x, T* d, T c1, T c2,
                                            int store_d) {
  const T r = b[i] - yi;
  const T dn = (c1 != T(0) ? c1 * d[i] : T(0)) + c2 * dinv[i] * r;
  if (store_d) d[i] = dn;  // the last step of a sweep does not need d again
  x[i] += dn;
}

// Release/acquire fence at GPU scope (orders this thread's earlier memory
// operations before its later ones as seen by other threads of the device).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Arguments of an operator kernel that finishes the smoother step itself.
template <typename T>
struct ChebFuse {
  const T* b;
  const T* dinv;
  T* x;  // the operator's input, updated in place by each dof's last contributor
  T* d;
  const unsigned* val;  // contributors per dof
  unsigned* cnt;        // countdown, equal to val between launches
  T c1, c2;
  int store_d;
};

// Asynchronous 4-byte global -> shared copies (cp.async, completed by
// cp_async_wait_all in the issuing thread; no other thread reads the slots).
__device__ __forceinline__ void cp_async4(int* smem, const int* gmem) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
// 16 bytes (both addresses 16-byte aligned), L2 only; with bytes = 0 the slot is
// zero-filled and gmem is not read.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// Until at most N of this thread's most recent groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Blocks of a persistent grid: resident blocks per SM of the kernel times the
// SM count, or fewer when there are fewer work items.
template <typename K>
inline int resident_grid(K kernel, int block, int work_items) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  int occ = 1;
  CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, 0));
  const int g = sms * (occ > 0 ? occ : 1);
  const int need = (int)(((long long)work_items + block - 1) / block);
  return need < g ? (need > 0 ? need : 1) : g;
}

// ---------------------------------------------------------- level data ---
struct Level {
  int N = 0, deg = 0, nd = 0;
  int n = 0, C = 0, V = 0, nb = 0;
  int Cs = 0;  // row stride of the [row][cell] arrays (map, geo): C rounded up to 128 (TMA rows)
  Numbering num{};
  DBuf<int> map;          // [nd][Cs]: dof j >= 0, or -1-j for a Dirichlet dof
  DBuf<double> vx, vy, vz;  // vertex coordinates
  DBuf<double> detj;      // |det J| per cell
  DBuf<double> kappa;     // cell coefficient
  DBuf<double> geo64;     // [6][Cs] kappa*|detJ| J^-1 J^-T / w  (w = 6 for P1, 120 for P2)
  DBuf<float> geo32;
  DBuf<float2> geodf;     // [6][Cs] geo64 split into float pairs (hi, lo) for the double-float apply
  // Every Kuhn tet of UnitCubeMesh has J = h P U (P a permutation, U the upper-triangular matrix of ones), so
  // G = |det J| J^-1 J^-T = h U^-1 U^-T = h M, M = [[2,-1,0],[-1,2,-1],[0,-1,1]], the same for every cell:
  // geo64 = c M with c = kappa h / w per cell.  Set-up checks this cell by cell against the G computed from the
  // vertex coordinates (uniform = 1 when every cell agrees) and keeps c for the operator kernels that then read
  // one value per cell instead of six.
  int uniform = 0;
  // 1 when also the two tets of every pair with the same first axis (cells 6q + 2k, 6q + 2k + 1: they share a face)
  // have the same c, so that the FP64 P2 operator applies such pairs as one unit
  int pair_uniform = 0;
  DBuf<float> c32;        // [C] c in FP32
  DBuf<float2> cdf;       // [C] c as a float pair
  DBuf<float2> massdf;    // |det J| / 120 (P1) or / 2520 (P2) per cell as a float pair (double-float mass)
  DBuf<double> dinv64;    // 1/diag(A)
  DBuf<float> dinv32;
  DBuf<int> bnd;          // Dirichlet dofs
  int Q = 0, Qs = 0;      // cubes and the row stride of the cube->dof map
  DBuf<int> cmap;         // [(k+1)^3][Qs] cube -> dof map (x fastest in the cube's lattice), signed like map
  double lmax = 2.0;
  // V-cycle work vectors (level-owned so the cycle can be captured in a graph)
  DBuf<double> b64, x64, y64, d64, w64;
  DBuf<double> fb64, fx64;  // full multigrid: this level's right-hand side and solution
  DBuf<float2> xs64;        // x64 as unscaled float pairs (split_pair), written with x64 for the FP64 operator
  // Transfer index tables (levels >= 1), one int4 per stencil entry of the
  // restriction to level-1 (fine dofs of this level around a coarse point) and
  // of the prolongation from level-1 (coarse dofs around a coarse cube): the
  // entry's dof at base point 0, its y and z strides, the packed lattice offset.
  DBuf<int4> rtab, ptab;
  DBuf<float> b32, x32, y32, d32;
  // Smoother fused with the operator (levels >= 1): per interior dof the number
  // of tets (val_tet) and of cubes (val_cube) that scatter into it, and the
  // countdown copies the apply kernels decrement; the thread that takes a
  // dof's count to zero holds its complete y_i and performs the Chebyshev
  // update of that dof, then restores the count.
  DBuf<unsigned> val_tet, cnt_tet, val_cube, cnt_cube;
  // Vertex-star patch smoother (levels >= 1, built by fe_set_smoother), one
  // patch per vertex.  P2: slot dofs [15][Pp], packed A_p^-1 [120][Pp] (FP64,
  // float pairs, FP32).  P3: patch-major slot dofs [P][65] and packed A_p^-1
  // [P][2145] (float pairs, FP32).  z: the preconditioned residuals.
  DBuf<int> pdof;
  DBuf<double> pinv, z64;
  DBuf<float2> pinvdf;  // A_p^-1 as float pairs for the FP64 smoother's float-pair product
  DBuf<float> pinv32, z32;
};

// Host-built transfer stencils (exact dyadic weights).
struct TransferTables {
  int deg = 0;
  int n_pro_class = 0, n_res_class = 0;
  int res_margin = 0;  // coarse points this far from the boundary need no bounds checks
  DBuf<int> pro_start, res_start;  // class -> first entry, size n_class+1
  DBuf<int4> pro_off, res_off;     // (dx,dy,dz,-) lattice offsets
  DBuf<double> pro_w, res_w;
  DBuf<float> pro_wf, res_wf;      // the same weights in FP32 (exact: dyadic with small numerators)
  std::vector<int> h_pro_start, h_res_start;
  std::vector<int4> h_pro_off, h_res_off;
  std::vector<double> h_pro_w, h_res_w;
};

// Scalars of the device-side CG recurrences.
enum ScalarSlot {
  S_RZ = 0, S_PQ, S_ALPHA, S_BETA, S_RR, S_RZNEW, S_DOT, S_BB, S_TMP0, S_TMP1, S_COUNT
};

struct ReduceCtx {
  int grid = 0;                 // fixed number of blocks of every reduction (deterministic order)
  DBuf<double> partials;        // grid * 2
  DBuf<unsigned int> counter;   // last-block ticket
  DBuf<double> scal;            // S_COUNT scalars
  double* h_scal = nullptr;     // pinned mirror
};

struct CoarseSolver {
  int nci = 0, band = 0;
  // Blocked form for large coarse levels (see fe_coarse.cu): the band factor in
  // band storage, then per block of B = band rows the inverse D of its
  // diagonal block and the block E to the left of it, with transposes.
  int blocked = 0, B = 0, nb = 0, npad = 0;
  double setup_ms = 0.0;
  size_t bytes = 0;     // device memory of the factor data
  DBuf<double> Ab;      // [npad][band + 1] band storage: row i holds A[i][i - band .. i]
  DBuf<double> D, DT;   // [nb][B][B] D_I = L_II^-1 and its transpose
  DBuf<double> E, ET;   // [nb][B][B] E_I = L_{I,I-1} (I >= 1) and its transpose
  DBuf<double> yb;      // [npad] forward-substitution result
  DBuf<int> ci;        // interior unknown j -> coarse dof
  DBuf<int> dof2int;   // coarse dof -> interior index or -1
  DBuf<double> A;      // nci*nci dense, then L (lower)
  DBuf<double> Linv, LinvT;
  // A^-1 = L^-T L^-1 times 2^(1023 - ainv_exp) (ainv_exp: the largest biased exponent of its diagonal) as float
  // pairs, rows padded to the even length ld: the dense coarse solve of the float-pair modes is one product with
  // it (k_coarse_inv_df: inv_smem bytes of shared memory, inv_grid64/32 blocks)
  DBuf<float2> AinvDF;
  int ld = 0, ainv_exp = 1023, inv_grid64 = 1, inv_grid32 = 1;
  size_t inv_smem = 0;
  DBuf<double> t0, t1;  // nci
  DBuf<int> flag;
};

struct fe_mesh {
  int N;
};

struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;  // kernel nodes of the captured graph
  cudaStream_t stream = nullptr;
  int steps = 0;  // smoother parameters baked into the captured launches
  double lo = 0, hi = 0;
  int extra = 0;  // another baked parameter (V-cycles per level of the full-multigrid graph)
};

// Per-phase, per-level CUDA-event timers of a profiled solve (fe_api.cu
// brackets each phase; collect() sums the brackets into the stats).
struct PhaseProf {
  struct Rec {
    int phase, level, e0, e1;
  };
  std::vector<cudaEvent_t> ev;  // pool, reused by later solves
  std::vector<Rec> recs;
  size_t used = 0;
  ~PhaseProf() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  int take() {
    if (used == ev.size()) {
      cudaEvent_t e;
      CUDA_CHECK(cudaEventCreate(&e));
      ev.push_back(e);
    }
    return (int)used++;
  }
  void reset() {
    used = 0;
    recs.clear();
  }
  // after the stream has been synchronised
  void collect(fe_solve_stats& st, int nlev) {
    st.levels_timed = nlev < FE_MAX_LEVELS ? nlev : FE_MAX_LEVELS;
    for (const Rec& r : recs) {
      float ms = 0.f;
      CUDA_CHECK(cudaEventElapsedTime(&ms, ev[r.e0], ev[r.e1]));
      if (r.level >= 0 && r.level < FE_MAX_LEVELS) st.phase_ms[r.phase][r.level] += ms;
    }
  }
};
struct fe_hierarchy {
  int N0 = 0, nlev = 0, deg = 0;
  int sms = 148;
  std::vector<Level> L;
  TransferTables tt;
  CoarseSolver cs;
  ReduceCtx red;
  DBuf<int> children;  // [6][8] coarse Kuhn type -> (subcube code * 8 + fine type)
  // fine-level Krylov vectors
  DBuf<double> x, r, z, p, q, b, e, tmp;
  DBuf<float2> ps;  // CG's p as unscaled float pairs (split_pair), written with p for the FP64 operator
  DBuf<float> r32, z32, p32, q32, e32;
  // staging for host pointers
  DBuf<unsigned char> stage[4];
  GraphCache vgraph[3];  // per dtype
  GraphCache fmggraph;   // the full-multigrid sequence (steps = V-cycles per level in `lo`)
  // device-side FP64 GMG-PCG loop: a graph whose while node repeats
  // (V-cycle, beta, p update, apply, alpha, x/r update, loop test)
  struct CgLoop {
    cudaGraphExec_t exec = nullptr;
    long long body_kernels = 0;
    int steps = 0;
    double lo = 0, hi = 0;
  } cgloop;
  DBuf<double> xcg, cgp;  // CG iterate of the graph loop; loop target
  DBuf<int> cgctl;        // loop counters
  bool lmax_valid = false;
  int f64_mode = FE_F64_DOUBLE_FLOAT;  // arithmetic of FP64 operator applications
  int fuse_smoother = 0;               // Chebyshev update fused into the operator kernel (measured slower on GB300)
  int smoother = FE_SMOOTHER_JACOBI;   // preconditioner of the Chebyshev smoother
  int coarse_mode = FE_COARSE_AUTO;    // dense inverse factor or blocked band factor
  int geometry_form = FE_GEOMETRY_AUTO;  // one value per cell (when uniform) or six stored factors
  PhaseProf prof;                      // per-phase timers of profiled solves
};

// ------------------------------------------------------- launch wrappers ---
// Operator kernels (fe_kernels.cu)
void launch_build_level(Level& L, cudaStream_t s);
void launch_geometry(Level& L, cudaStream_t s);
void launch_apply64(const Level& L, const double* x, double* y, cudaStream_t s);
void launch_apply32(const Level& L, const float* x, float* y, cudaStream_t s);
// xs (optional): x as unscaled float pairs (split_pair), gathered instead of x
void launch_apply64_df(const Level& L, const double* x, double* y, cudaStream_t s, const float2* xs = nullptr);
// x as the float pairs the pre-split P2 operator gathers (into L.xs64), for an application whose input no vector
// kernel has split.
void launch_split_pairs(const Level& L, const double* x, cudaStream_t s);
void launch_apply64_cube_df(const Level& L, const double* x, double* y, cudaStream_t s);
void launch_apply64_df2(const Level& L, const double* x, double* y, cudaStream_t s);
void launch_apply64_df3(const Level& L, const double* x, double* y, cudaStream_t s);
void upload_p3_mass_table(const float* m3i);
// The same operator kernels with the Chebyshev update fused (y = A x, then
// d = c1 d + c2 D^-1 (b - y), x += d per dof, in one launch).
void launch_apply_cheb32(const Level& L, const float* b, float* x, float* y, float* d, double c1, double c2,
                         bool store_d, cudaStream_t s);
void launch_apply_cheb64_df(const Level& L, const double* b, double* x, double* y, double* d, double c1, double c2,
                            bool store_d, cudaStream_t s);
void launch_apply_cheb64_cube_df(const Level& L, const double* b, double* x, double* y, double* d, double c1,
                                 double c2, bool store_d, cudaStream_t s);
void launch_build_valence(Level& L, cudaStream_t s);
// band < 0: dense nci x nci (both triangles); band >= 0: band storage [nci][band + 1], lower triangle only
void launch_coarse_assemble_p3(const Level& L0, const int* dof2int, int nci, double* A, int band, cudaStream_t s);
// Vertex-star patch smoother (fe_patch.cu; P3 setup in fe_kernels.cu)
void launch_patch_setup(Level& L, cudaStream_t s);
void launch_patch_setup_p3(Level& L, cudaStream_t s);
template <typename T>
void launch_patch_apply(const Level& L, const T* b, const T* y, T* z, bool df, cudaStream_t s);
template <typename T>
void launch_cheb_pc(int n, const T* z, T* x, T* d, double c1, double c2, bool first_from_zero, bool store_d,
                    cudaStream_t s);
void launch_split_geometry(Level& L, cudaStream_t s);
// Checks geo64 = c M cell by cell, fills c32 and cdf and sets L.uniform and L.pair_uniform (synchronises s).
void launch_uniform_geometry(Level& L, int* dflag, cudaStream_t s);
// b -= A g on interior rows and b = g on the boundary (inhomogeneous Dirichlet data, symmetric elimination)
void launch_bc_lift(const Level& L, const double* g, double* b, cudaStream_t s);
void launch_mass(const Level& L, const double* x, double* y, cudaStream_t s);
void launch_mass_df(const Level& L, const double* x, double* y, cudaStream_t s);
void launch_quad_points(const Level& L, double* xyz, cudaStream_t s);
void launch_load_quadrature(const Level& L, const double* fq, double* b, cudaStream_t s);
void launch_diag(Level& L, double* diag_out, cudaStream_t s);
void launch_gradient(const Level& L, const double* u, const double* lam, double* g, cudaStream_t s);
void launch_dof_coords(const Level& L, double* xyz, cudaStream_t s);
void launch_centroids(const Level& L, double* xyz, cudaStream_t s);
void launch_bmask(const Level& L, unsigned char* m, cudaStream_t s);
void launch_coarsen_kappa(const Level& Lc, const Level& Lf, const int* children, cudaStream_t s);
int launch_check_positive(const double* v, int n, int* dflag, cudaStream_t s);
// Transfers
// xs (optional, FP64): also write the result as unscaled float pairs
template <typename T>
void launch_prolong(const fe_hierarchy* h, int lf, const T* xc, T* xf, bool accumulate, cudaStream_t s,
                    float2* xs = nullptr);
// rc = P^T (bf - yf), or P^T bf when yf is null
template <typename T>
void launch_restrict(const fe_hierarchy* h, int lf, const T* bf, const T* yf, T* rc, bool zero_bd, cudaStream_t s);

// Vector kernels
// xs (optional, FP64): also write the new x as unscaled float pairs
template <typename T>
void launch_cheb_step(int n, const T* b, const T* y, const T* dinv, T* x, T* d, double c1, double c2, bool first_from_zero,
                      cudaStream_t s, bool store_d = true, float2* xs = nullptr);
// p = z and ps = split_pair(z)
void launch_copy_split(int n, const double* z, double* p, float2* ps, cudaStream_t s);
template <typename Ti, typename To>
void launch_convert(int n, const Ti* in, To* out, cudaStream_t s);
void launch_set_boundary(const Level& L, const double* src, double* dst, cudaStream_t s);
void launch_zero_boundary64(const Level& L, double* v, cudaStream_t s);
void launch_random(int n, uint64_t seed, double* v, cudaStream_t s);
// Reductions and CG updates (fe_blas.cu)
void red_init(ReduceCtx& R, int sms);
void red_free(ReduceCtx& R);
template <typename T>
void launch_dot(ReduceCtx& R, int n, const T* a, const T* b, int slot, cudaStream_t s);
// q-dot: pq = p.q; alpha = rz/pq
template <typename T>
void launch_cg_alpha(ReduceCtx& R, int n, const T* p, const T* q, cudaStream_t s);
// x += alpha p; r -= alpha q; rr = r.r; (jacobi: z = dinv r, rznew = r.z, beta = rznew/rz, rz = rznew)
template <typename T>
void launch_cg_update(ReduceCtx& R, int n, T* x, T* r, const T* p, const T* q, const T* dinv, T* z, cudaStream_t s);
// rznew = r.z; beta = rznew/rz; rz = rznew
template <typename T>
void launch_cg_beta(ReduceCtx& R, int n, const T* r, const T* z, cudaStream_t s);
// ps (optional, FP64): also write the new p as unscaled float pairs
template <typename T>
void launch_cg_update_p(ReduceCtx& R, int n, T* p, const T* z, cudaStream_t s, float2* ps = nullptr);
void launch_cg_cond(cudaGraphConditionalHandle hnd, const double* scal, const double* cgp, int* ctl, int inc,
                    cudaStream_t s);
void launch_cg_set(double* cgp, int* ctl, double tol2, int it0, int max_it, cudaStream_t s);
void launch_axpy64(int n, double a, const double* x, double* y, cudaStream_t s);
void launch_sub64(int n, const double* a, const double* b, double* out, cudaStream_t s);  // out = a - b
template <typename T>
void launch_scale_copy(int n, const double* in, const double* scale_slot, bool inverse, T* out, cudaStream_t s);
template <typename T>
void launch_add_scaled(int n, const T* e, const double* scale_slot, double* x, cudaStream_t s);
// Coarse solver (fe_coarse.cu)
void coarse_setup(fe_hierarchy* h, cudaStream_t s);
template <typename T>
void coarse_solve(const fe_hierarchy* h, const T* b, T* x, cudaStream_t s);

// Orchestration helpers (fe_api.cu)
fe_hierarchy* hierarchy_create(int N0, int nrefine, int degree);  // throws FeError
void hierarchy_set_coefficient(fe_hierarchy* h, const double* kappa, cudaStream_t s);
void hierarchy_destroy(fe_hierarchy* h);
template <typename T>
void vcycle_enqueue(fe_hierarchy* h, int dtype, cudaStream_t s);  // reads L.b of the finest level, writes L.x
// xs (optional): FP64 x as unscaled float pairs, current with x (the float-pair P2 kernel gathers it)
void apply_enqueue(const fe_hierarchy* h, int level, const void* x, void* y, int dtype, cudaStream_t s,
                   const float2* xs = nullptr);
void apply_bf16_enqueue(const Level& L, const float* x, float* y, cudaStream_t s);
bool bf16_supported();
int bf16_take_error(cudaStream_t s);      // nonzero if a tensor-core launch gave up a bounded wait
void bf16_prepare(const Level& L);        // build the level's tensor maps and tables (never inside a capture)
void bf16_forget_level(const Level* L);  // drop the cached tensor maps of a level being destroyed

// ------------------------------------------------------- element kernels ---
// Geometry of one tet from its vertex coordinates: G = |det J| J^-1 J^-T
// (symmetric, stored G00,G01,G02,G11,G12,G22) and |det J|.  With J = [a b c]
// (columns p1-p0, p2-p0, p3-p0) the rows of det(J) J^-1 are b x c, c x a,
// a x b, hence G_ij = r_i . r_j / |det J|.
template <typename T>
__host__ __device__ inline void tet_metric(const T p[4][3], T g[6], T& adet) {
  T a[3], b[3], c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    a[k] = p[1][k] - p[0][k];
    b[k] = p[2][k] - p[0][k];
    c[k] = p[3][k] - p[0][k];
  }
  T r0[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
  T r1[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
  T r2[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  const T det = a[0] * r0[0] + a[1] * r0[1] + a[2] * r0[2];
  adet = det < T(0) ? -det : det;
  const T inv = T(1) / adet;
  g[0] = (r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]) * inv;
  g[1] = (r0[0] * r1[0] + r0[1] * r1[1] + r0[2] * r1[2]) * inv;
  g[2] = (r0[0] * r2[0] + r0[1] * r2[1] + r0[2] * r2[2]) * inv;
  g[3] = (r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]) * inv;
  g[4] = (r1[0] * r2[0] + r1[1] * r2[1] + r1[2] * r2[2]) * inv;
  g[5] = (r2[0] * r2[0] + r2[1] * r2[1] + r2[2] * r2[2]) * inv;
}

// P1 tet: grad u is constant; with reference gradient d = (u1-u0, u2-u0, u3-u0)
// the element form is a(u,v) = (1/6) d^T G d', so y_{1..3} = G d / 6 and
// y_0 = -(y_1 + y_2 + y_3).  `g` holds kappa * G / 6.
template <typename T>
__host__ __device__ inline void p1_element(const T u[4], const T g[6], T y[4]) {
  const T d0 = u[1] - u[0], d1 = u[2] - u[0], d2 = u[3] - u[0];
  const T h0 = g[0] * d0 + g[1] * d1 + g[2] * d2;
  const T h1 = g[1] * d0 + g[3] * d1 + g[4] * d2;
  const T h2 = g[2] * d0 + g[4] * d1 + g[5] * d2;
  y[1] = h0;
  y[2] = h1;
  y[3] = h2;
  y[0] = -(h0 + h1 + h2);
}

// Local P2 edge numbering: edge (w,v) of the tet -> local dof 4..9 for the
// pairs (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).
__host__ __device__ constexpr int p2_edge(int w, int v) {
  return (w > v) ? p2_edge(v, w) : (w == 0 ? 3 + v : (w == 1 ? 5 + v : 9));
}

// P2 tet.  grad u is affine, so it is fixed by its values at the 4 vertices:
// in barycentric gradients, grad u(w) = sum_v c_wv grad(lambda_v) with
// c_ww = 3 u_w and c_wv = 4 u_(wv) - u_v.  In reference coordinates
// d_w = grad_ref u(w) = (c_w1 - c_w0, c_w2 - c_w0, c_w3 - c_w0).  With
// int_ref lambda_w lambda_w' = (1 + delta_ww')/120 the element form is
//   a(u,v) = (1/120) [ S^T G S' + sum_w d_w^T G d'_w ],  S = sum_w d_w,
// so y = (d/du)^T h with h_w = G (S + d_w) / 120.  `g` holds kappa G / 120.
// 124 operations per tet instead of the 10x10 element matrix; written
// without loops so that every value stays in a register.
// Local dofs: vertices 0..3, then edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).
template <typename T>
__host__ __device__ inline void p2_gmul(const T* g, T t0, T t1, T t2, T& h0, T& h1, T& h2) {
  h0 = g[0] * t0 + g[1] * t1 + g[2] * t2;
  h1 = g[1] * t0 + g[3] * t1 + g[4] * t2;
  h2 = g[2] * t0 + g[4] * t1 + g[5] * t2;
}

template <typename T>
__host__ __device__ inline void p2_element(const T* u, const T* g, T* y) {
  const T three = T(3), four = T(4);
  const T f01 = four * u[4], f02 = four * u[5], f03 = four * u[6];
  const T f12 = four * u[7], f13 = four * u[8], f23 = four * u[9];
  const T c00 = three * u[0], c01 = f01 - u[1], c02 = f02 - u[2], c03 = f03 - u[3];
  const T c10 = f01 - u[0], c11 = three * u[1], c12 = f12 - u[2], c13 = f13 - u[3];
  const T c20 = f02 - u[0], c21 = f12 - u[1], c22 = three * u[2], c23 = f23 - u[3];
  const T c30 = f03 - u[0], c31 = f13 - u[1], c32 = f23 - u[2], c33 = three * u[3];
  const T d00 = c01 - c00, d01 = c02 - c00, d02 = c03 - c00;
  const T d10 = c11 - c10, d11 = c12 - c10, d12 = c13 - c10;
  const T d20 = c21 - c20, d21 = c22 - c20, d22 = c23 - c20;
  const T d30 = c31 - c30, d31 = c32 - c30, d32 = c33 - c30;
  const T S0 = (d00 + d10) + (d20 + d30), S1 = (d01 + d11) + (d21 + d31), S2 = (d02 + d12) + (d22 + d32);
  T b01, b02, b03, b11, b12, b13, b21, b22, b23, b31, b32, b33;  // cb_wv = h_w[v-1]
  p2_gmul(g, S0 + d00, S1 + d01, S2 + d02, b01, b02, b03);
  p2_gmul(g, S0 + d10, S1 + d11, S2 + d12, b11, b12, b13);
  p2_gmul(g, S0 + d20, S1 + d21, S2 + d22, b21, b22, b23);
  p2_gmul(g, S0 + d30, S1 + d31, S2 + d32, b31, b32, b33);
  const T b00 = -(b01 + b02 + b03), b10 = -(b11 + b12 + b13), b20 = -(b21 + b22 + b23), b30 = -(b31 + b32 + b33);
  // y_v = 3 cb_vv - sum_{w != v} cb_wv;  y_(ab) = 4 (cb_ab + cb_ba)
  y[0] = three * b00 - ((b10 + b20) + b30);
  y[1] = three * b11 - ((b01 + b21) + b31);
  y[2] = three * b22 - ((b02 + b12) + b32);
  y[3] = three * b33 - ((b03 + b13) + b23);
  y[4] = four * (b01 + b10);
  y[5] = four * (b02 + b20);
  y[6] = four * (b03 + b30);
  y[7] = four * (b12 + b21);
  y[8] = four * (b13 + b31);
  y[9] = four * (b23 + b32);
}

// P1/P2 element formulas; the P3 element (through the gradient at the P2
// nodes) is fe_p3::p3_element_grad in fe_p3.cuh.
template <int DEG, typename T>
__host__ __device__ inline void element_apply(const T* u, const T* g, T* y) {
  static_assert(DEG == 1 || DEG == 2, "P3 uses fe_p3::p3_element_grad (fe_p3.cuh)");
  if constexpr (DEG == 1)
    p1_element<T>(u, g, y);
  else
    p2_element<T>(u, g, y);
}

// Dofs of one tet: 4 (P1), 10 (P2), 20 (P3).
__host__ __device__ constexpr int tet_ndof(int deg) { return deg == 1 ? 4 : deg == 2 ? 10 : 20; }

// P3 local dofs: vertices 0..3; edge e = (a, b), a < b, in the P2 edge order
// (p2_edge - 4) holds node 4 + 2e, the one nearer a (lattice 2 v_a + v_b), and
// node 4 + 2e + 1 (v_a + 2 v_b); the face opposite vertex f holds node 16 + f
// (the sum of its three vertices).
__host__ __device__ constexpr int p3_face_vertex(int f, int k) {  // k-th vertex of the face opposite f
  return k + (k >= f ? 1 : 0);
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
