// C ABI of the library (include/fe.h): mesh and hierarchy construction,
// coefficient setup, and the host orchestration of the multigrid V-cycle,
// preconditioned CG, mixed-precision iterative refinement and the adjoint
// gradient.  Every arithmetic step runs in the CUDA kernels of fe_kernels.cu,
// fe_blas.cu, fe_coarse.cu and fe_tc.cu; the host only sequences launches and
// tests convergence.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>

#include "fe_checks.h"
#include "fe_internal.cuh"
#include "fe_stencils.h"

void upload_mass_tables();
void launch_fill64(size_t n, double v, double* p, cudaStream_t s);

// ------------------------------------------------------------- errors
static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;
void fe_count_launch() {
  if (!g_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void fe_set_error(const std::string& m) { g_err = m; }

#define API_BEGIN try {
#define API_END                                   \
  }                                               \
  catch (const FeError& e) {                      \
    fe_set_error(e.msg);                          \
    return e.code;                                \
  }                                               \
  catch (const std::bad_alloc&) {                 \
    fe_set_error("host allocation failed");       \
    return FE_ERR_NOMEM;                          \
  }                                               \
  catch (...) {                                   \
    fe_set_error("unexpected C++ exception");     \
    return FE_ERR_CUDA;                           \
  }                                               \
  return FE_OK;

// ----------------------------------------------------------- numbering
Numbering make_numbering(int N, int deg) {
  Numbering nb{};
  nb.N = N;
  nb.deg = deg;
  nb.m = deg * N;
  if (deg != 2) {  // P1, P3: one lexicographic class over the (kN+1)^3 lattice
    const int n1 = deg * N + 1, n = n1 * n1 * n1;
    nb.off[0] = 0;
    for (int k = 1; k < 9; ++k) nb.off[k] = n;
    for (int k = 0; k < 8; ++k) nb.sx[k] = nb.sy[k] = nb.sz[k] = n1;
    return nb;
  }
  int acc = 0;
  for (int c = 0; c < 8; ++c) {
    nb.sx[c] = N + 1 - class_parity_x(c);
    nb.sy[c] = N + 1 - class_parity_y(c);
    nb.sz[c] = N + 1 - class_parity_z(c);
    nb.off[c] = acc;
    acc += nb.sx[c] * nb.sy[c] * nb.sz[c];
  }
  nb.off[8] = acc;
  return nb;
}

// ------------------------------------------------- host pointer staging
// FE_DEBUG_CHECKS=1 in the environment turns on host-side consistency checks
// of the device tables (read back once per hierarchy).
static bool debug_checks() {
  static const bool on = [] {
    const char* v = std::getenv("FE_DEBUG_CHECKS");
    return v != nullptr && v[0] != '\0' && std::strcmp(v, "0") != 0;
  }();
  return on;
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void* stage_buf(fe_hierarchy* h, int slot, size_t bytes) {
  DBuf<unsigned char>& b = h->stage[slot];
  if (b.n < bytes) b.alloc(bytes);
  return b.p;
}

template <typename T>
static const T* stage_in(fe_hierarchy* h, int slot, const T* p, size_t n, cudaStream_t s) {
  if (!p || is_device_ptr(p)) return p;
  T* d = (T*)stage_buf(h, slot, n * sizeof(T));
  CUDA_CHECK(cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

template <typename T>
static T* stage_out(fe_hierarchy* h, int slot, T* p, size_t n) {
  if (!p || is_device_ptr(p)) return p;
  return (T*)stage_buf(h, slot, n * sizeof(T));
}

template <typename T>
static void finish_out(T* user, const T* dev, size_t n, cudaStream_t s) {
  if (user && user != dev) {
    CUDA_CHECK(cudaMemcpyAsync(user, dev, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
  }
}

static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

// Transfer index tables.  A stencil entry names the lattice point
// (k X + ox, k Y + oy, k Z + oz) of numbering `num` for a base point (X, Y, Z):
// the restriction's fine points 2 Xc + o, the prolongation's coarse points
// DEG c + o.  Its dof is then affine in (X, Y, Z): P1 numbers the lattice
// lexicographically, P2 numbers each parity class lexicographically by
// halved coordinates, and for k = 2 the class of k X + o is that of o.  The
// entry stores (dof at X = Y = Z = 0, y stride, z stride, o packed as three
// bytes biased by 8); the x stride is k for P1/P3 and 1 for P2.
static int4 entry_index(const Numbering& num, int k, int ox, int oy, int oz) {
  FE_REQUIRE(ox >= -8 && ox < 8 && oy >= -8 && oy < 8 && oz >= -8 && oz < 8, FE_ERR_UNSUPPORTED,
             "transfer offset out of the packed range");
  const int packed = (ox + 8) | ((oy + 8) << 8) | ((oz + 8) << 16);
  if (num.deg != 2) {  // lexicographic (P1, P3): x stride k
    const int n1 = num.m + 1;
    return make_int4(ox + n1 * (oy + n1 * oz), k * n1, k * n1 * n1, packed);
  }
  FE_REQUIRE(k == 2, FE_ERR_UNSUPPORTED, "P2 transfer base points sit on even lattice coordinates");
  const int code = (ox & 1) | ((oy & 1) << 1) | ((oz & 1) << 2);
  const int c = code == 3 ? 4 : code == 4 ? 3 : code;
  const int sx = num.sx[c], sy = num.sy[c];
  const int dx = ox >> 1, dy = oy >> 1, dz = oz >> 1;  // floor halving (offsets may be negative)
  return make_int4(num.off[c] + dx + sx * (dy + sy * dz), sx, sx * sy, packed);
}

static void build_level_transfer_index(Level& F, const Level& Cc, const TransferTables& t) {
  std::vector<int4> r(t.h_res_off.size()), p(t.h_pro_off.size());
  for (size_t e = 0; e < r.size(); ++e) {
    const int4 o = t.h_res_off[e];  // fine point 2 Xc + o of level F
    r[e] = entry_index(F.num, 2, o.x, o.y, o.z);
  }
  for (size_t e = 0; e < p.size(); ++e) {
    const int4 o = t.h_pro_off[e];  // coarse point DEG c + o of level Cc
    p[e] = entry_index(Cc.num, F.deg, o.x, o.y, o.z);
  }
  // the affine forms against the numbering itself, at base points near both
  // ends of each axis (host only, once per hierarchy)
  auto check = [](const Numbering& num, int k, const std::vector<int4>& off, const std::vector<int4>& tab,
                  int kx, int bmax) {
    const int B[4] = {0, 1, bmax - 1, bmax};
    for (size_t e = 0; e < off.size(); ++e)
      for (int a = 0; a < 64; ++a) {
        const int X = B[a & 3], Y = B[(a >> 2) & 3], Z = B[a >> 4];
        const int x = k * X + off[e].x, y = k * Y + off[e].y, z = k * Z + off[e].z;
        if (X < 0 || Y < 0 || Z < 0 || x < 0 || y < 0 || z < 0 || x > num.m || y > num.m || z > num.m) continue;
        FE_REQUIRE(tab[e].x + kx * X + tab[e].y * Y + tab[e].z * Z == lattice_to_dof(num, x, y, z), FE_ERR_CUDA,
                   "transfer index table disagrees with the numbering");
      }
  };
  check(F.num, 2, t.h_res_off, r, F.deg == 2 ? 1 : 2, Cc.num.m);
  check(Cc.num, F.deg, t.h_pro_off, p, F.deg == 3 ? 3 : 1, Cc.num.N);
  F.rtab.alloc(r.size());
  CUDA_CHECK(cudaMemcpy(F.rtab, r.data(), sizeof(int4) * r.size(), cudaMemcpyHostToDevice));
  F.ptab.alloc(p.size());
  CUDA_CHECK(cudaMemcpy(F.ptab, p.data(), sizeof(int4) * p.size(), cudaMemcpyHostToDevice));
}

// -------------------------------------------------- transfer stencils
// The stencils of fe_stencils.h as per-class device tables (FP64 and FP32
// weights: dyadic with small numerators, so the FP32 copies are exact).
static void build_transfer_tables(TransferTables& t, int deg) {
  t.deg = deg;
  t.n_pro_class = 8 * deg * deg * deg;
  t.n_res_class = deg * deg * deg;
  std::vector<fe_stencil::Entry> pro;
  fe_stencil::prolongation(deg, t.h_pro_start, pro);
  t.h_pro_off.clear();
  t.h_pro_w.clear();
  for (const auto& e : pro) {
    t.h_pro_off.push_back(make_int4(e.d[0], e.d[1], e.d[2], 0));
    t.h_pro_w.push_back(e.w);
  }
  std::vector<fe_stencil::Tap> res;
  fe_stencil::restriction(deg, pro, t.h_res_start, res);
  t.h_res_off.clear();
  t.h_res_w.clear();
  for (const auto& r : res) {
    t.h_res_off.push_back(make_int4(r.off[0], r.off[1], r.off[2], 0));
    t.h_res_w.push_back(r.w);
  }
  // coarse points with every coordinate in [margin, m - margin] have all their
  // fine points inside the lattice (2 X + o in [0, 2 m] for |o| <= 2 margin)
  int omax = 0;
  for (const int4& o : t.h_res_off) omax = std::max({omax, std::abs(o.x), std::abs(o.y), std::abs(o.z)});
  t.res_margin = (omax + 1) / 2;
  // the prolongation kernel unrolls at most 2 (P1), 10 (P2) or 20 (P3) entries per fine point
  for (int c = 0; c < t.n_pro_class; ++c)
    FE_REQUIRE(t.h_pro_start[c + 1] - t.h_pro_start[c] <= (deg == 1 ? 2 : tet_ndof(deg)), FE_ERR_UNSUPPORTED,
               "prolongation stencil longer than the kernel's bound");
  auto up = [](auto& dbuf, const auto& vec) {
    using T = typename std::decay_t<decltype(vec)>::value_type;
    dbuf.alloc(vec.size());
    CUDA_CHECK(cudaMemcpy(dbuf.p, vec.data(), sizeof(T) * vec.size(), cudaMemcpyHostToDevice));
  };
  up(t.pro_start, t.h_pro_start);
  up(t.pro_off, t.h_pro_off);
  up(t.pro_w, t.h_pro_w);
  up(t.pro_wf, std::vector<float>(t.h_pro_w.begin(), t.h_pro_w.end()));
  up(t.res_wf, std::vector<float>(t.h_res_w.begin(), t.h_res_w.end()));
  up(t.res_start, t.h_res_start);
  up(t.res_off, t.h_res_off);
  up(t.res_w, t.h_res_w);
}

// The 8 children of each coarse Kuhn type: (subcube code, fine type) whose
// centroid lies in it (the Kuhn meshes at N and 2N are nested).
static std::vector<int> build_children() {
  std::vector<int> ch(48, -1), cnt(6, 0);
  for (int code = 0; code < 8; ++code)
    for (int t = 0; t < 6; ++t) {
      int p0, p1, p2;
      kuhn_perm(t, p0, p1, p2);
      double c[3] = {0, 0, 0};
      int v[3] = {0, 0, 0};
      for (int k = 0; k < 4; ++k) {
        if (k == 1) v[p0] = 1;
        if (k == 2) v[p1] = 1;
        if (k == 3) v[p2] = 1;
        for (int a = 0; a < 3; ++a) c[a] += 0.25 * v[a];
      }
      const double s[3] = {0.5 * (((code >> 0) & 1) + c[0]), 0.5 * (((code >> 1) & 1) + c[1]),
                           0.5 * (((code >> 2) & 1) + c[2])};
      int sig[3] = {0, 1, 2};
      std::sort(sig, sig + 3, [&](int a, int b) { return s[a] > s[b]; });
      const int T = 2 * sig[0] + (sig[1] > sig[2] ? 1 : 0);
      FE_REQUIRE(cnt[T] < 8, FE_ERR_CUDA, "refinement table construction failed");
      ch[T * 8 + cnt[T]++] = code * 8 + t;
    }
  for (int T = 0; T < 6; ++T) FE_REQUIRE(cnt[T] == 8, FE_ERR_CUDA, "refinement table construction failed");
  return ch;
}

// --------------------------------------------------- eigenvalue estimate
// Largest eigenvalue of the symmetric tridiagonal (a, b) by Sturm bisection.
static double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int k = (int)a.size();
  double lo = 0.0, hi = 0.0;
  for (int i = 0; i < k; ++i) {
    const double r = std::fabs(i > 0 ? b[i - 1] : 0.0) + std::fabs(i + 1 < k ? b[i] : 0.0);
    hi = std::max(hi, a[i] + r);
    lo = std::min(lo, a[i] - r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
      const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      q = (a[i] - x) - (i > 0 ? bb / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= k)
      hi = mid;
    else
      lo = mid;
  }
  return hi;
}

// lambda_max(D^-1 A_l) from `steps` Jacobi-PCG iterations on a seeded random
// right-hand side: the CG coefficients define the Lanczos tridiagonal.
// Whether level l smooths with the vertex-star patches (P2 levels >= 1; for P1
// the patches are single vertices and the preconditioner is Jacobi).
static bool use_patch(const fe_hierarchy* h, int l) {
  return h->smoother == FE_SMOOTHER_PATCH && h->deg >= 2 && l >= 1 && h->L[l].pdof.p;
}

// lambda_max(M^-1 A) from the Lanczos tridiagonal of `steps` PCG iterations
// (M = D, or the patch preconditioner on patch-smoothed levels).
static double estimate_lmax(fe_hierarchy* h, int l, int steps, cudaStream_t s) {
  Level& L = h->L[l];
  const int n = L.n;
  ReduceCtx& R = h->red;
  double *b = h->b, *x = h->x, *r = h->r, *z = h->z, *p = h->p, *q = h->q;
  const bool patch = use_patch(h, l);
  launch_random(n, 0x2104080120210416ull + (uint64_t)l, b, s);
  launch_zero_boundary64(L, b, s);
  CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  CUDA_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (patch) {
    launch_patch_apply<double>(L, r, nullptr, z, h->f64_mode != FE_F64_NATIVE, s);  // z = M^-1 r
    CUDA_CHECK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    launch_cheb_step<double>(n, r, nullptr, L.dinv64, p, z, 0.0, 1.0, true, s);  // z = p = D^-1 r
  }
  launch_dot<double>(R, n, r, z, S_RZ, s);
  CUDA_CHECK(cudaMemcpyAsync(R.h_scal, R.scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  if (!(R.h_scal[S_RZ] > 0.0)) return 1.0;  // no interior dofs: D^-1 A is the identity
  std::vector<double> al, be;
  for (int it = 0; it < steps; ++it) {
    apply_enqueue(h, l, p, q, FE_F64, s);
    launch_cg_alpha<double>(R, n, p, q, s);
    if (patch) {
      launch_cg_update<double>(R, n, x, r, p, q, nullptr, nullptr, s);
      launch_patch_apply<double>(L, r, nullptr, z, h->f64_mode != FE_F64_NATIVE, s);
      launch_cg_beta<double>(R, n, r, z, s);
    } else {
      launch_cg_update<double>(R, n, x, r, p, q, L.dinv64, z, s);
    }
    launch_cg_update_p<double>(R, n, p, z, s);
    CUDA_CHECK(cudaMemcpyAsync(R.h_scal, R.scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    const double alpha = R.h_scal[S_ALPHA], beta = R.h_scal[S_BETA];
    if (!(std::isfinite(alpha) && std::isfinite(beta)) || alpha <= 0) break;
    al.push_back(alpha);
    be.push_back(beta);
    if (R.h_scal[S_RR] <= 0.0) break;
  }
  FE_REQUIRE(!al.empty(), FE_ERR_NAN, "eigenvalue estimate failed");
  const int k = (int)al.size();
  std::vector<double> a(k), off(k > 1 ? k - 1 : 0);
  for (int i = 0; i < k; ++i) {
    a[i] = 1.0 / al[i] + (i > 0 ? be[i - 1] / al[i - 1] : 0.0);
    if (i + 1 < k) off[i] = std::sqrt(be[i]) / al[i];
  }
  return tridiag_max_eig(a, off);
}

// -------------------------------------------------------- V-cycle
// ------------------------------------------------ per-phase timers (profile)
// With fe_solver_opts.profile set, each phase of the solve on each level is
// bracketed by a pair of CUDA events; after the solve the elapsed times are
// summed into fe_solve_stats.phase_ms (a per-level multigrid log).  Graph
// replay is off while profiling, so every bracket holds real launches.
static thread_local PhaseProf* g_prof = nullptr;

struct PhaseScope {
  PhaseProf* p;
  cudaStream_t s;
  size_t rec = 0;
  PhaseScope(int phase, int level, cudaStream_t st) : p(g_capturing ? nullptr : g_prof), s(st) {
    if (!p) return;
    const int e0 = p->take();
    CUDA_CHECK(cudaEventRecord(p->ev[e0], s));
    rec = p->recs.size();
    p->recs.push_back({phase, level, e0, -1});
  }
  ~PhaseScope() {
    if (!p) return;
    const int e1 = p->take();
    p->recs[rec].e1 = e1;
    cudaEventRecord(p->ev[e1], s);  // no throw from a destructor; a failed record shows up at the next check
  }
  PhaseScope(const PhaseScope&) = delete;
  PhaseScope& operator=(const PhaseScope&) = delete;
};

struct SmootherParams {
  int steps = 2;
  double lo = 0.1, hi = 1.1;
};
static thread_local SmootherParams g_sp;

template <typename T> static T* lv_b(Level& L);
template <typename T> static T* lv_x(Level& L);
template <typename T> static T* lv_y(Level& L);
template <typename T> static T* lv_d(Level& L);
template <typename T> static const T* lv_dinv(const Level& L);
template <> double* lv_b<double>(Level& L) { return L.b64; }
template <> double* lv_x<double>(Level& L) { return L.x64; }
template <> double* lv_y<double>(Level& L) { return L.y64; }
template <> double* lv_d<double>(Level& L) { return L.d64; }
template <> const double* lv_dinv<double>(const Level& L) { return L.dinv64; }
template <> float* lv_b<float>(Level& L) { return L.b32; }
template <> float* lv_x<float>(Level& L) { return L.x32; }
template <> float* lv_y<float>(Level& L) { return L.y32; }
template <> float* lv_d<float>(Level& L) { return L.d32; }
template <> const float* lv_dinv<float>(const Level& L) { return L.dinv32; }
template <typename T> static T* lv_z(Level& L);
template <> double* lv_z<double>(Level& L) { return L.z64; }
template <> float* lv_z<float>(Level& L) { return L.z32; }

// Consistent mass y = M x in FP64: float-pair arithmetic unless the hierarchy
// is in native-FP64 mode (the operator's mode decides both).
static void mass_enqueue(const fe_hierarchy* h, const Level& L, const double* x, double* y, cudaStream_t s) {
  if (h->f64_mode == FE_F64_NATIVE)
    launch_mass(L, x, y, s);
  else
    launch_mass_df(L, x, y, s);
}

// Whether the FP64 operator on level l is the per-tet float-pair kernel that can
// gather pre-split dofs (P1 in FE_F64_DOUBLE_FLOAT_TET mode, P2 in the default
// mode), so that the vector kernels producing its inputs write float pairs too.
// FE_F64_DOUBLE_FLOAT_TET keeps the split inside the operator kernel (for
// comparison); the fused and patch smoothers update x without pairs.
static bool presplit(const fe_hierarchy* h, int l) {
  const Level& L = h->L[l];
  return h->f64_mode == FE_F64_DOUBLE_FLOAT && L.deg == 2 && L.xs64.p && !h->fuse_smoother &&
         !(h->smoother == FE_SMOOTHER_PATCH && h->deg >= 2 && l >= 1 && L.pdof.p);
}

void apply_enqueue(const fe_hierarchy* h, int level, const void* x, void* y, int dtype, cudaStream_t s,
                   const float2* xs) {
  const Level& L = h->L[level];
  if (L.deg == 3) {  // P3: element through the gradient at the P2 nodes in FP64, float pairs (default), FP32 or bf16
    if (dtype == FE_F64 && h->f64_mode == FE_F64_NATIVE)
      launch_apply64(L, (const double*)x, (double*)y, s);
    else if (dtype == FE_F64)
      launch_apply64_df3(L, (const double*)x, (double*)y, s);
    else if (dtype == FE_F32)
      launch_apply32(L, (const float*)x, (float*)y, s);
    else if (dtype == FE_BF16)
      apply_bf16_enqueue(L, (const float*)x, (float*)y, s);
    else
      FE_FAIL(FE_ERR_ARG, "unknown dtype");
    return;
  }
  // measured on GB300 (P*64^3): P1 per cube 0.025 ms vs per tet 0.041 ms; P2 per tet 0.139 ms vs per cube
  // 0.209 ms (the P2 cube kernel needs 254 registers, i.e. 8 warps per SM)
  const bool cube = h->f64_mode == FE_F64_DOUBLE_FLOAT_CUBE || (h->f64_mode == FE_F64_DOUBLE_FLOAT && L.deg == 1);
  if (dtype == FE_F64 && h->f64_mode == FE_F64_DOUBLE_FLOAT_PAIR && L.deg == 2)
    launch_apply64_df2(L, (const double*)x, (double*)y, s);
  else if (dtype == FE_F64 && h->f64_mode != FE_F64_NATIVE && cube)
    launch_apply64_cube_df(L, (const double*)x, (double*)y, s);
  else if (dtype == FE_F64 && h->f64_mode != FE_F64_NATIVE)
    launch_apply64_df(L, (const double*)x, (double*)y, s, h->f64_mode == FE_F64_DOUBLE_FLOAT ? xs : nullptr);
  else if (dtype == FE_F64)
    launch_apply64(L, (const double*)x, (double*)y, s);
  else if (dtype == FE_F32)
    launch_apply32(L, (const float*)x, (float*)y, s);
  else if (dtype == FE_BF16)
    apply_bf16_enqueue(L, (const float*)x, (float*)y, s);
  else
    FE_FAIL(FE_ERR_ARG, "unknown dtype");
}

// y = A x followed by the Chebyshev update of every dof: with fusion on, one
// launch when the operator kernel of this precision and mode has the fused
// form (FP32 cube kernel, float-pair tet and cube kernels); otherwise the
// operator kernel and the vector kernel.
template <typename T>
static void apply_cheb_enqueue(fe_hierarchy* h, int l, const T* b, T* x, T* y, T* d, double c1, double c2,
                               bool store_d, int dtype, cudaStream_t s, const float2* xs_in = nullptr,
                               float2* xs_out = nullptr) {
  Level& L = h->L[l];
  if (h->fuse_smoother && L.cnt_tet.p && L.deg <= 2) {
    const bool cube = h->f64_mode == FE_F64_DOUBLE_FLOAT_CUBE || (h->f64_mode == FE_F64_DOUBLE_FLOAT && L.deg == 1);
    if constexpr (sizeof(T) == 8) {
      if (dtype == FE_F64 && h->f64_mode != FE_F64_NATIVE) {
        if (cube)
          launch_apply_cheb64_cube_df(L, b, x, y, d, c1, c2, store_d, s);
        else
          launch_apply_cheb64_df(L, b, x, y, d, c1, c2, store_d, s);
        return;
      }
    } else {
      if (dtype == FE_F32) {
        launch_apply_cheb32(L, b, x, y, d, c1, c2, store_d, s);
        return;
      }
    }
  }
  apply_enqueue(h, l, x, y, dtype, s, xs_in);
  launch_cheb_step<T>(L.n, b, y, lv_dinv<T>(L), x, d, c1, c2, false, s, store_d, xs_out);
}

// Chebyshev iterations on level l (the level smoother of Section 3): the
// three-term Chebyshev semi-iteration for the preconditioned operator on
// [lo, hi] * lambda_max, theta = centre, delta = half-width of the interval.
// xs_fresh_in: L.xs64 holds x as float pairs on entry (FP64, presplit levels);
// xs_after: leave L.xs64 current with the smoothed x (an operator application
// reads it next).
template <typename T>
static void smooth_enqueue(fe_hierarchy* h, int l, const T* b, T* x, T* y, T* d, int steps, double lo, double hi,
                           bool x_zero, int dtype, cudaStream_t s, bool xs_fresh_in = false, bool xs_after = false) {
  Level& L = h->L[l];
  const double a = lo * L.lmax, bmax = hi * L.lmax;
  const double theta = 0.5 * (bmax + a), delta = 0.5 * (bmax - a), sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (use_patch(h, l)) {  // z = M^-1 (b - A x) by the vertex-star patches, then d = c1 d + c2 z, x += d
    T* z = lv_z<T>(L);
    for (int k = 0; k < steps; ++k) {
      const bool last = k + 1 == steps;
      const bool from_zero = k == 0 && x_zero;
      if (!from_zero) apply_enqueue(h, l, x, y, dtype, s);
      launch_patch_apply<T>(L, b, from_zero ? nullptr : y, z, h->f64_mode != FE_F64_NATIVE, s);
      if (k == 0) {
        launch_cheb_pc<T>(L.n, z, x, d, 0.0, 1.0 / theta, from_zero, !last, s);
      } else {
        const double rn = 1.0 / (2.0 * sigma - rho);
        launch_cheb_pc<T>(L.n, z, x, d, rn * rho, 2.0 * rn / delta, false, !last, s);
        rho = rn;
      }
    }
    return;
  }
  float2* xs = nullptr;  // x's float pairs, written by each step whose x an operator application reads next
  if constexpr (sizeof(T) == 8)
    if (dtype == FE_F64 && presplit(h, l)) xs = L.xs64.p;
  for (int k = 0; k < steps; ++k) {
    const bool last = k + 1 == steps;  // its direction d is not used again
    float2* xs_out = (!last || xs_after) ? xs : nullptr;
    const float2* xs_in = (k > 0 || xs_fresh_in) ? xs : nullptr;
    if (k == 0) {
      if (x_zero)
        launch_cheb_step<T>(L.n, b, nullptr, lv_dinv<T>(L), x, d, 0.0, 1.0 / theta, true, s, !last, xs_out);
      else
        apply_cheb_enqueue<T>(h, l, b, x, y, d, 0.0, 1.0 / theta, !last, dtype, s, xs_in, xs_out);
    } else {
      const double rn = 1.0 / (2.0 * sigma - rho);
      apply_cheb_enqueue<T>(h, l, b, x, y, d, rn * rho, 2.0 * rn / delta, !last, dtype, s, xs_in, xs_out);
      rho = rn;
    }
  }
}

// One V-cycle on levels l..0: approximately solves A_l x_l = b_l.
template <typename T>
static void vcycle_level(fe_hierarchy* h, int l, int dtype, cudaStream_t s) {
  Level& L = h->L[l];
  T *b = lv_b<T>(L), *x = lv_x<T>(L), *y = lv_y<T>(L), *d = lv_d<T>(L);
  if (l == 0) {
    PhaseScope ps(FE_PHASE_COARSE, 0, s);
    coarse_solve<T>(h, b, x, s);
    return;
  }
  const int rdt = (dtype == FE_BF16) ? FE_F32 : dtype;  // residuals in FP32 when smoothing in bf16
  float2* xs = nullptr;  // x as float pairs on presplit FP64 levels (see smooth_enqueue)
  if constexpr (sizeof(T) == 8)
    if (dtype == FE_F64 && presplit(h, l)) xs = L.xs64.p;
  {
    PhaseScope ps(FE_PHASE_SMOOTH, l, s);
    smooth_enqueue<T>(h, l, b, x, y, d, g_sp.steps, g_sp.lo, g_sp.hi, true, dtype, s, false, true);
  }
  {
    PhaseScope ps(FE_PHASE_APPLY, l, s);
    apply_enqueue(h, l, x, y, rdt, s, xs);
  }
  Level& Lc = h->L[l - 1];
  {
    PhaseScope ps(FE_PHASE_TRANSFER, l, s);
    launch_restrict<T>(h, l, b, y, lv_b<T>(Lc), true, s);
  }
  vcycle_level<T>(h, l - 1, dtype, s);
  {
    PhaseScope ps(FE_PHASE_TRANSFER, l, s);
    launch_prolong<T>(h, l, lv_x<T>(Lc), x, true, s, xs);
  }
  PhaseScope ps(FE_PHASE_SMOOTH, l, s);
  smooth_enqueue<T>(h, l, b, x, y, d, g_sp.steps, g_sp.lo, g_sp.hi, false, dtype, s, xs != nullptr, false);
}

// Enqueue one fine-level V-cycle (reads L.b of the finest level, writes
// L.x); replays a captured CUDA graph when `use_graph` is set.
static void run_vcycle(fe_hierarchy* h, int dtype, bool use_graph, cudaStream_t s) {
  auto enqueue = [&](cudaStream_t st) {
    if (dtype == FE_F64)
      vcycle_level<double>(h, h->nlev - 1, dtype, st);
    else
      vcycle_level<float>(h, h->nlev - 1, dtype, st);
  };
  if (!use_graph) {
    enqueue(s);
    return;
  }
  GraphCache& gc = h->vgraph[dtype];
  if (gc.exec && (gc.steps != g_sp.steps || gc.lo != g_sp.lo || gc.hi != g_sp.hi)) {
    cudaGraphExecDestroy(gc.exec);
    gc.exec = nullptr;
  }
  if (!gc.exec) {
    // everything a captured launch needs must exist before the capture starts
    if (dtype == FE_BF16)
      for (int l = 1; l < h->nlev; ++l) bf16_prepare(h->L[l]);
    if (!gc.stream) CUDA_CHECK(cudaStreamCreateWithFlags(&gc.stream, cudaStreamNonBlocking));
    cudaGraph_t g;
    CUDA_CHECK(cudaStreamBeginCapture(gc.stream, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    try {
      enqueue(gc.stream);
    } catch (...) {
      g_capturing = false;
      cudaStreamEndCapture(gc.stream, &g);
      throw;
    }
    g_capturing = false;
    CUDA_CHECK(cudaStreamEndCapture(gc.stream, &g));
    size_t nn = 0;
    CUDA_CHECK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) CUDA_CHECK(cudaGraphGetNodes(g, nodes.data(), &nn));
    gc.kernels = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      CUDA_CHECK(cudaGraphNodeGetType(nd, &ty));
      if (ty == cudaGraphNodeTypeKernel) ++gc.kernels;
    }
    CUDA_CHECK(cudaGraphInstantiate(&gc.exec, g, 0));
    cudaGraphDestroy(g);
    gc.steps = g_sp.steps;
    gc.lo = g_sp.lo;
    gc.hi = g_sp.hi;
  }
  CUDA_CHECK(cudaGraphLaunch(gc.exec, s));
  g_launches.fetch_add(gc.kernels, std::memory_order_relaxed);
}

static void invalidate_graphs(fe_hierarchy* h) {
  for (auto& g : h->vgraph)
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
  if (h->cgloop.exec) {
    cudaGraphExecDestroy(h->cgloop.exec);
    h->cgloop.exec = nullptr;
  }
  if (h->fmggraph.exec) {
    cudaGraphExecDestroy(h->fmggraph.exec);
    h->fmggraph.exec = nullptr;
  }
}

static long long count_kernel_nodes(cudaGraph_t g);

// Full multigrid as the whole solve (paper Section 3): b restricted to every
// level (boundary entries zero), the coarsest level solved directly, then on
// each finer level x_l = P x_{l-1} corrected by `cycles` V-cycles in defect
// form x_l += V(b_l - A_l x_l) (a V-cycle started from x_l; the smoother is
// linear).  The solution is left in the fine level's fx64.
static void fmg_enqueue(fe_hierarchy* h, const double* b, int cycles, cudaStream_t s) {
  const int top = h->nlev - 1;
  if (b != h->L[top].fb64.p)
    CUDA_CHECK(cudaMemcpyAsync(h->L[top].fb64, b, sizeof(double) * h->L[top].n, cudaMemcpyDeviceToDevice, s));
  for (int l = top; l >= 1; --l) {
    PhaseScope ps(FE_PHASE_TRANSFER, l, s);
    launch_restrict<double>(h, l, h->L[l].fb64, nullptr, h->L[l - 1].fb64, true, s);
  }
  {
    PhaseScope ps(FE_PHASE_COARSE, 0, s);
    coarse_solve<double>(h, h->L[0].fb64, h->L[0].fx64, s);
  }
  for (int l = 1; l <= top; ++l) {
    Level& L = h->L[l];
    {
      PhaseScope ps(FE_PHASE_TRANSFER, l, s);
      launch_prolong<double>(h, l, h->L[l - 1].fx64, L.fx64, false, s);
    }
    for (int c = 0; c < cycles; ++c) {
      {
        PhaseScope ps(FE_PHASE_APPLY, l, s);
        apply_enqueue(h, l, L.fx64, L.y64, FE_F64, s);
      }
      {
        PhaseScope ps(FE_PHASE_BLAS1, l, s);
        launch_sub64(L.n, L.fb64, L.y64, L.b64, s);
      }
      vcycle_level<double>(h, l, FE_F64, s);
      PhaseScope ps(FE_PHASE_BLAS1, l, s);
      launch_axpy64(L.n, 1.0, L.x64, L.fx64, s);
    }
  }
}

static void run_fmg(fe_hierarchy* h, const double* b, int cycles, bool use_graph, cudaStream_t s) {
  GraphCache& gc = h->fmggraph;
  const int top = h->nlev - 1;
  if (!use_graph) {
    fmg_enqueue(h, b, cycles, s);
    return;
  }
  // the graph reads the fine right-hand side from fb64 (copied in outside the graph)
  if (b != h->L[top].fb64.p)
    CUDA_CHECK(cudaMemcpyAsync(h->L[top].fb64, b, sizeof(double) * h->L[top].n, cudaMemcpyDeviceToDevice, s));
  if (gc.exec && (gc.steps != g_sp.steps || gc.lo != g_sp.lo || gc.hi != g_sp.hi || gc.extra != cycles)) {
    cudaGraphExecDestroy(gc.exec);
    gc.exec = nullptr;
  }
  if (!gc.exec) {
    if (!gc.stream) CUDA_CHECK(cudaStreamCreateWithFlags(&gc.stream, cudaStreamNonBlocking));
    cudaGraph_t g;
    CUDA_CHECK(cudaStreamBeginCapture(gc.stream, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    try {
      fmg_enqueue(h, h->L[top].fb64, cycles, gc.stream);
    } catch (...) {
      g_capturing = false;
      cudaStreamEndCapture(gc.stream, &g);
      throw;
    }
    g_capturing = false;
    CUDA_CHECK(cudaStreamEndCapture(gc.stream, &g));
    gc.kernels = count_kernel_nodes(g);
    CUDA_CHECK(cudaGraphInstantiate(&gc.exec, g, 0));
    cudaGraphDestroy(g);
    gc.steps = g_sp.steps;
    gc.lo = g_sp.lo;
    gc.hi = g_sp.hi;
    gc.extra = cycles;
  }
  CUDA_CHECK(cudaGraphLaunch(gc.exec, s));
  g_launches.fetch_add(gc.kernels, std::memory_order_relaxed);
}

// ------------------------------------------------------------ PCG
struct PcgResult {
  int it = 0;
  double rr = 0, bb = 0;
  int status = FE_OK;
  int applies = 0;
  double apply_ms = 0.0;
  int apply_timed = 0;
};

// CUDA events around the CG operator application when profiling.
struct ApplyTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool on = false;
  explicit ApplyTimer(bool enable) : on(enable) {
    if (on) {
      CUDA_CHECK(cudaEventCreate(&e0));
      CUDA_CHECK(cudaEventCreate(&e1));
    }
  }
  ~ApplyTimer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  void start(cudaStream_t s) { if (on) CUDA_CHECK(cudaEventRecord(e0, s)); }
  void stop(cudaStream_t s) { if (on) CUDA_CHECK(cudaEventRecord(e1, s)); }
  // after the stream has been synchronised
  void collect(PcgResult& r) {
    if (!on) return;
    float ms = 0.f;
    CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    r.apply_ms += ms;
    ++r.apply_timed;
  }
};

// FP64 PCG on the finest level: b, x device vectors (x overwritten).
// Kernel nodes of a captured graph.
static long long count_kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  CUDA_CHECK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) CUDA_CHECK(cudaGraphGetNodes(g, nodes.data(), &nn));
  long long k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    CUDA_CHECK(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// The FP64 GMG-PCG iterations after the first as one graph: a loop test, then
// a while node whose body is one CG iteration ending with the same test, so the
// host neither waits for nor relaunches anything between iterations.
static void build_cg_loop(fe_hierarchy* h) {
  GraphCache& gc = h->vgraph[FE_F64];
  if (!gc.stream) CUDA_CHECK(cudaStreamCreateWithFlags(&gc.stream, cudaStreamNonBlocking));
  const cudaStream_t cs = gc.stream;
  Level& F = h->L[h->nlev - 1];
  const int n = F.n;
  ReduceCtx& R = h->red;
  double *r = F.b64, *z = F.x64, *p = h->p, *q = h->q, *x = h->xcg;
  cudaGraph_t g, out;
  CUDA_CHECK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond;
  CUDA_CHECK(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
  auto capture = [&](cudaGraph_t into, auto&& body) {
    CUDA_CHECK(cudaStreamBeginCaptureToGraph(cs, into, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    try {
      body();
    } catch (...) {
      g_capturing = false;
      cudaStreamEndCapture(cs, &out);
      cudaGraphDestroy(g);
      throw;
    }
    g_capturing = false;
    CUDA_CHECK(cudaStreamEndCapture(cs, &out));
  };
  capture(g, [&] { launch_cg_cond(cond, R.scal, h->cgp, h->cgctl, 0, cs); });
  cudaGraphNode_t test;
  size_t one = 1;
  CUDA_CHECK(cudaGraphGetNodes(g, &test, &one));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  CUDA_CHECK(cudaGraphAddNode(&loop, g, &test, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  capture(body, [&] {
    float2* ps = presplit(h, h->nlev - 1) ? h->ps.p : nullptr;
    run_vcycle(h, FE_F64, false, cs);
    launch_cg_beta<double>(R, n, r, z, cs);
    launch_cg_update_p<double>(R, n, p, z, cs, ps);
    apply_enqueue(h, h->nlev - 1, p, q, FE_F64, cs, ps);
    launch_cg_alpha<double>(R, n, p, q, cs);
    launch_cg_update<double>(R, n, x, r, p, q, nullptr, z, cs);
    launch_cg_cond(cond, R.scal, h->cgp, h->cgctl, 1, cs);
  });
  h->cgloop.body_kernels = count_kernel_nodes(body);
  CUDA_CHECK(cudaGraphInstantiate(&h->cgloop.exec, g, 0));
  cudaGraphDestroy(g);
  h->cgloop.steps = g_sp.steps;
  h->cgloop.lo = g_sp.lo;
  h->cgloop.hi = g_sp.hi;
}

static PcgResult pcg64_graph(fe_hierarchy* h, double* x, const fe_solver_opts& o, double tol2, PcgResult res,
                             cudaStream_t s) {
  Level& F = h->L[h->nlev - 1];
  const int n = F.n;
  ReduceCtx& R = h->red;
  double *r = F.b64, *z = F.x64, *p = h->p, *q = h->q, *xw = h->xcg;
  auto& cl = h->cgloop;
  if (cl.exec && (cl.steps != g_sp.steps || cl.lo != g_sp.lo || cl.hi != g_sp.hi)) {
    cudaGraphExecDestroy(cl.exec);
    cl.exec = nullptr;
  }
  if (!cl.exec) build_cg_loop(h);
  // first iteration from the host, then the loop
  CUDA_CHECK(cudaMemsetAsync(xw, 0, sizeof(double) * n, s));
  apply_enqueue(h, h->nlev - 1, p, q, FE_F64, s, presplit(h, h->nlev - 1) ? h->ps.p : nullptr);
  launch_cg_alpha<double>(R, n, p, q, s);
  launch_cg_update<double>(R, n, xw, r, p, q, nullptr, z, s);
  launch_cg_set(h->cgp, h->cgctl, tol2, 1, o.max_it, s);
  CUDA_CHECK(cudaGraphLaunch(cl.exec, s));
  int ctl[2] = {0, 0};
  CUDA_CHECK(cudaMemcpyAsync(ctl, h->cgctl, sizeof(ctl), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaMemcpyAsync(R.h_scal + S_RR, R.scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaMemcpyAsync(x, xw, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  res.it = ctl[0];
  res.applies = ctl[0];
  g_launches.fetch_add(1 + (long long)(ctl[0] - 1) * cl.body_kernels, std::memory_order_relaxed);
  res.rr = R.h_scal[S_RR];
  if (!std::isfinite(res.rr))
    res.status = FE_ERR_NAN;
  else if (res.rr > tol2)
    res.status = FE_ERR_NO_CONVERGENCE;
  return res;
}

static PcgResult pcg64(fe_hierarchy* h, const double* b, double* x, const fe_solver_opts& o, cudaStream_t s) {
  Level& F = h->L[h->nlev - 1];
  const int n = F.n;
  ReduceCtx& R = h->red;
  double *r = F.b64, *z = F.x64, *p = h->p, *q = h->q;
  const bool gmg = o.precond == FE_PC_GMG && h->nlev > 1;
  PcgResult res;
  const int top = h->nlev - 1;
  const bool graphs = o.use_graph != 0 && !o.profile;
  {
    PhaseScope ps(FE_PHASE_BLAS1, top, s);
    CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    CUDA_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    launch_dot<double>(R, n, b, b, S_BB, s);
  }
  if (gmg) {
    run_vcycle(h, FE_F64, graphs, s);
  } else {
    PhaseScope ps(FE_PHASE_SMOOTH, top, s);
    launch_cheb_step<double>(n, r, nullptr, F.dinv64, q, z, 0.0, 1.0, true, s);  // z = D^-1 r
  }
  float2* psplit = presplit(h, top) ? h->ps.p : nullptr;  // p as float pairs for the operator
  {
    PhaseScope ps(FE_PHASE_BLAS1, top, s);
    launch_dot<double>(R, n, r, z, S_RZ, s);
    if (psplit)
      launch_copy_split(n, z, p, psplit, s);
    else
      CUDA_CHECK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  CUDA_CHECK(cudaMemcpyAsync(R.h_scal, R.scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  res.bb = R.h_scal[S_BB];
  res.rr = res.bb;
  const double tol2 = o.rtol * o.rtol * res.bb;
  if (res.bb == 0.0) return res;
  if (gmg && o.use_graph && !o.profile && o.max_it >= 1) return pcg64_graph(h, x, o, tol2, res, s);
  ApplyTimer timer(o.profile != 0);
  while (true) {
    if (res.it >= o.max_it) {
      res.status = FE_ERR_NO_CONVERGENCE;
      break;
    }
    {
      PhaseScope ps(FE_PHASE_APPLY, top, s);
      timer.start(s);
      apply_enqueue(h, top, p, q, FE_F64, s, psplit);
      timer.stop(s);
    }
    ++res.applies;
    {
      PhaseScope ps(FE_PHASE_BLAS1, top, s);
      launch_cg_alpha<double>(R, n, p, q, s);
      launch_cg_update<double>(R, n, x, r, p, q, gmg ? nullptr : F.dinv64.p, z, s);
    }
    CUDA_CHECK(cudaMemcpyAsync(R.h_scal + S_RR, R.scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    timer.collect(res);
    ++res.it;
    res.rr = R.h_scal[S_RR];
    if (!std::isfinite(res.rr)) {
      res.status = FE_ERR_NAN;
      break;
    }
    if (res.rr <= tol2) break;
    if (gmg) run_vcycle(h, FE_F64, graphs, s);
    PhaseScope ps(FE_PHASE_BLAS1, top, s);
    if (gmg) launch_cg_beta<double>(R, n, r, z, s);
    launch_cg_update_p<double>(R, n, p, z, s, psplit);
  }
  return res;
}

// Inner reduced-precision GMG-PCG for A e = r32 (||r32|| = 1), e in h->e32.
static PcgResult pcg_low(fe_hierarchy* h, int dtype, const fe_solver_opts& o, cudaStream_t s) {
  Level& F = h->L[h->nlev - 1];
  const int n = F.n;
  ReduceCtx& R = h->red;
  float *r = F.b32, *z = F.x32, *p = h->p32, *q = h->q32, *e = h->e32;
  PcgResult res;
  const int top = h->nlev - 1;
  const bool graphs = o.use_graph != 0 && !o.profile;
  {
    PhaseScope ps(FE_PHASE_BLAS1, top, s);
    CUDA_CHECK(cudaMemsetAsync(e, 0, sizeof(float) * n, s));
    launch_dot<float>(R, n, r, r, S_BB, s);
  }
  run_vcycle(h, dtype, graphs, s);
  {
    PhaseScope ps(FE_PHASE_BLAS1, top, s);
    launch_dot<float>(R, n, r, z, S_RZ, s);
    CUDA_CHECK(cudaMemcpyAsync(p, z, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  }
  CUDA_CHECK(cudaMemcpyAsync(R.h_scal, R.scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  res.bb = R.h_scal[S_BB];
  const double tol2 = o.inner_rtol * o.inner_rtol * res.bb;
  while (res.it < o.inner_max_it) {
    {
      PhaseScope ps(FE_PHASE_APPLY, top, s);
      launch_apply32(F, p, q, s);
    }
    ++res.applies;
    {
      PhaseScope ps(FE_PHASE_BLAS1, top, s);
      launch_cg_alpha<float>(R, n, p, q, s);
      launch_cg_update<float>(R, n, e, r, p, q, nullptr, z, s);
    }
    CUDA_CHECK(cudaMemcpyAsync(R.h_scal + S_RR, R.scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    ++res.it;
    res.rr = R.h_scal[S_RR];
    if (!std::isfinite(res.rr)) {
      res.status = FE_ERR_NAN;
      break;
    }
    if (res.rr <= tol2) break;
    run_vcycle(h, dtype, graphs, s);
    PhaseScope ps(FE_PHASE_BLAS1, top, s);
    launch_cg_beta<float>(R, n, r, z, s);
    launch_cg_update_p<float>(R, n, p, z, s);
  }
  return res;
}

// FP64 iterative refinement: r = b - A x in FP64, inner low-precision solve,
// x += e, until ||r|| <= rtol ||b||.
static PcgResult refine(fe_hierarchy* h, const double* b, double* x, const fe_solver_opts& o, int dtype,
                        fe_solve_stats* st, cudaStream_t s) {
  Level& F = h->L[h->nlev - 1];
  const int n = F.n;
  ReduceCtx& R = h->red;
  double* r = h->r;
  double* y = h->tmp;
  PcgResult res;
  CUDA_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  CUDA_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  launch_dot<double>(R, n, b, b, S_BB, s);
  CUDA_CHECK(cudaMemcpyAsync(R.h_scal, R.scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  res.bb = R.h_scal[S_BB];
  double rr = res.bb;
  const double bb = res.bb;
  int outer = 0, inner_total = 0, low_applies = 0, stalled = 0;
  const int max_outer = std::min(o.max_it, 100);
  if (bb > 0.0) {
    while (rr > o.rtol * o.rtol * bb) {
      // stop when the limit is reached or refinement stagnates (3 steps in a row
      // reducing ||r|| by less than 2x: the low-precision solve no longer helps)
      if (outer >= max_outer || stalled >= 3) {
        res.status = FE_ERR_NO_CONVERGENCE;
        break;
      }
      const double rr_prev = rr;
      // r32 = r / ||r||; ||r||^2 parked in S_TMP0 for the correction
      CUDA_CHECK(cudaMemcpyAsync(R.scal + S_TMP0, R.scal + (outer == 0 ? S_BB : S_DOT), sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
      {
        PhaseScope ps(FE_PHASE_BLAS1, h->nlev - 1, s);
        launch_scale_copy<float>(n, r, R.scal + S_TMP0, true, F.b32, s);
      }
      PcgResult in = pcg_low(h, dtype, o, s);
      inner_total += in.it;
      low_applies += in.applies;
      if (in.status == FE_ERR_NAN) {
        res.status = FE_ERR_NAN;
        break;
      }
      {
        PhaseScope ps(FE_PHASE_BLAS1, h->nlev - 1, s);
        launch_add_scaled<float>(n, h->e32, R.scal + S_TMP0, x, s);
      }
      {
        PhaseScope ps(FE_PHASE_APPLY, h->nlev - 1, s);
        apply_enqueue(h, h->nlev - 1, x, y, FE_F64, s);
      }
      ++res.applies;
      PhaseScope ps(FE_PHASE_BLAS1, h->nlev - 1, s);
      launch_sub64(n, b, y, r, s);
      launch_dot<double>(R, n, r, r, S_DOT, s);
      CUDA_CHECK(cudaMemcpyAsync(R.h_scal + S_DOT, R.scal + S_DOT, sizeof(double), cudaMemcpyDeviceToHost, s));
      CUDA_CHECK(cudaStreamSynchronize(s));
      rr = R.h_scal[S_DOT];
      ++outer;
      if (!std::isfinite(rr)) {
        res.status = FE_ERR_NAN;
        break;
      }
      stalled = (rr > 0.25 * rr_prev) ? stalled + 1 : 0;
    }
  }
  res.rr = rr;
  res.it = inner_total;
  if (st) {
    st->outer_iterations = outer;
    st->fine_applies_low = low_applies;
  }
  return res;
}

// --------------------------------------------------------- setup
static void set_coefficient_impl(fe_hierarchy* h, const double* kappa, cudaStream_t s) {
  Level& F = h->L[h->nlev - 1];
  if (kappa) {
    const double* kd = stage_in<double>(h, 0, kappa, F.C, s);
    FE_REQUIRE(launch_check_positive(kd, F.C, h->cs.flag, s) == 0, FE_ERR_ARG, "kappa must be positive and finite");
    CUDA_CHECK(cudaMemcpyAsync(F.kappa, kd, sizeof(double) * F.C, cudaMemcpyDeviceToDevice, s));
  } else {
    launch_fill64(F.C, 1.0, F.kappa, s);
  }
  for (int l = h->nlev - 1; l >= 1; --l) launch_coarsen_kappa(h->L[l - 1], h->L[l], h->children, s);
  for (int l = 0; l < h->nlev; ++l) {
    launch_geometry(h->L[l], s);
    launch_split_geometry(h->L[l], s);
    launch_uniform_geometry(h->L[l], h->cs.flag, s);
    if (h->geometry_form == FE_GEOMETRY_PER_CELL) h->L[l].uniform = 0;
    launch_diag(h->L[l], h->tmp, s);
  }
  if (h->smoother == FE_SMOOTHER_PATCH && h->deg >= 2)
    for (int l = 1; l < h->nlev; ++l) launch_patch_setup(h->L[l], s);
  for (int l = 0; l < h->nlev; ++l) h->L[l].lmax = estimate_lmax(h, l, 20, s);
  if (h->nlev > 1) coarse_setup(h, s);
  invalidate_graphs(h);
  CUDA_CHECK(cudaStreamSynchronize(s));
}

static const double* rhs_to_load(fe_hierarchy* h, const double* rhs, int kind, cudaStream_t s) {
  Level& F = h->L[h->nlev - 1];
  const double* rd = stage_in<double>(h, 1, rhs, kind == FE_RHS_QUAD_F ? (size_t)F.C * FE_QUAD_POINTS : F.n, s);
  if (kind == FE_RHS_QUAD_F) {
    launch_load_quadrature(F, rd, h->b, s);
    launch_zero_boundary64(F, h->b, s);
  } else if (kind == FE_RHS_LOAD) {
    if (rd != h->b.p) CUDA_CHECK(cudaMemcpyAsync(h->b, rd, sizeof(double) * F.n, cudaMemcpyDeviceToDevice, s));
  } else if (kind == FE_RHS_NODAL_F) {
    mass_enqueue(h, F, rd, h->b, s);
    launch_zero_boundary64(F, h->b, s);
  } else {
    FE_FAIL(FE_ERR_ARG, "unknown rhs kind");
  }
  return h->b;
}

static void check_level(const fe_hierarchy* h, int level) {
  FE_REQUIRE(h, FE_ERR_ARG, "null hierarchy");
  FE_REQUIRE(level >= 0 && level < h->nlev, FE_ERR_ARG, "level out of range");
}

static fe_solver_opts resolve_opts(const fe_solver_opts* o) {
  fe_solver_opts d;
  fe_default_opts(&d);
  if (o) d = *o;
  FE_REQUIRE(d.rtol >= 0 && d.max_it >= 0 && d.cheb_steps >= 1 && d.cheb_hi > d.cheb_lo && d.cheb_lo > 0,
             FE_ERR_ARG, "invalid solver options");
  FE_REQUIRE(d.precond == FE_PC_JACOBI || d.precond == FE_PC_GMG || d.precond == FE_PC_FMG, FE_ERR_ARG,
             "unknown preconditioner");
  FE_REQUIRE(d.precond != FE_PC_FMG || (d.precision == FE_PREC_F64 && d.max_it >= 1 && d.max_it <= 100), FE_ERR_ARG,
             "full multigrid runs in FP64 with 1..100 V-cycles per level (max_it)");
  return d;
}

// Builds every level of UnitCubeMesh(N0 * 2^l), l = 0..nrefine, on the current
// device and sets kappa = 1 (throws FeError).
fe_hierarchy* hierarchy_create(int N0, int nrefine, int degree) {
  FE_REQUIRE(N0 >= 1, FE_ERR_ARG, "mesh size must be >= 1");
  FE_REQUIRE(nrefine >= 0 && nrefine <= 8, FE_ERR_ARG, "nrefine must be in [0, 8]");
  FE_REQUIRE(degree >= 1 && degree <= 3, FE_ERR_UNSUPPORTED, "degree must be 1, 2 or 3");
  const long long Nf = (long long)N0 << nrefine;
  const long long nf = (long long)(degree * Nf + 1) * (degree * Nf + 1) * (degree * Nf + 1);
  FE_REQUIRE(6 * Nf * Nf * Nf < (1ll << 31) && nf < (1ll << 31), FE_ERR_ARG, "finest level too large for 32-bit indices");
  FE_REQUIRE(fe_device_count() > 0, FE_ERR_CUDA, "no CUDA device");
  std::unique_ptr<fe_hierarchy> h(new fe_hierarchy());
  int dev = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  CUDA_CHECK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
  {
    // constant-memory tables live in each device's context: upload them once per device
    static std::mutex mu;
    static std::vector<char> uploaded;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= (int)uploaded.size()) uploaded.resize(dev + 1, 0);
    if (!uploaded[dev]) {
      upload_mass_tables();
      uploaded[dev] = 1;
    }
  }
  h->N0 = N0;
  h->nlev = nrefine + 1;
  h->deg = degree;
  h->L.resize(h->nlev);
  cudaStream_t s = 0;
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->L[l];
    L.N = N0 << l;
    L.deg = degree;
    L.nd = tet_ndof(degree);
    L.num = make_numbering(L.N, degree);
    const int m = degree * L.N;
    L.n = (m + 1) * (m + 1) * (m + 1);
    L.C = 6 * L.N * L.N * L.N;
    L.V = (L.N + 1) * (L.N + 1) * (L.N + 1);
    L.Cs = (L.C + 127) / 128 * 128;
    L.Q = L.N * L.N * L.N;
    L.Qs = (L.Q + 127) / 128 * 128;
    L.cmap.alloc((size_t)(degree + 1) * (degree + 1) * (degree + 1) * L.Qs);
    L.map.alloc((size_t)L.nd * L.Cs);
    CUDA_CHECK(cudaMemset(L.map, 0, sizeof(int) * (size_t)L.nd * L.Cs));
    // P3 vertex dofs are not numbered first: coordinates of every dof instead
    const int ncoord = degree == 3 ? L.n : L.V;
    L.vx.alloc(ncoord);
    L.vy.alloc(ncoord);
    L.vz.alloc(ncoord);
    L.detj.alloc(L.C);
    L.kappa.alloc(L.C);
    L.geo64.alloc((size_t)6 * L.Cs);
    L.geo32.alloc((size_t)6 * L.Cs);
    CUDA_CHECK(cudaMemset(L.geo32, 0, sizeof(float) * (size_t)6 * L.Cs));
    L.geodf.alloc((size_t)6 * L.Cs);
    L.massdf.alloc(L.C);
    L.dinv64.alloc(L.n);
    L.dinv32.alloc(L.n);
    for (auto* v : {&L.b64, &L.x64, &L.y64, &L.d64, &L.w64, &L.fb64, &L.fx64}) v->alloc(L.n);
    if (degree == 2) L.xs64.alloc(L.n);  // float pairs of x for the P2 float-pair operator
    for (auto* v : {&L.b32, &L.x32, &L.y32, &L.d32}) v->alloc(L.n);
    std::vector<int> bnd;
    bnd.reserve((size_t)6 * (m + 1) * (m + 1));
    for (int z = 0; z <= m; ++z)
      for (int y = 0; y <= m; ++y)
        for (int x = 0; x <= m; ++x)
          if (x == 0 || y == 0 || z == 0 || x == m || y == m || z == m) {
            bnd.push_back(lattice_to_dof(L.num, x, y, z));
            if (!(z == 0 || z == m || y == 0 || y == m) && x == 0) x = m - 1;  // skip the interior of the row
          }
    std::sort(bnd.begin(), bnd.end());
    L.nb = (int)bnd.size();
    L.bnd.alloc(L.nb);
    CUDA_CHECK(cudaMemcpy(L.bnd, bnd.data(), sizeof(int) * L.nb, cudaMemcpyHostToDevice));
    launch_build_level(L, s);
    if (debug_checks()) {  // FE_DEBUG_CHECKS=1: bounds and boundary check of both maps on the host
      CUDA_CHECK(cudaStreamSynchronize(s));
      const int nq = (degree + 1) * (degree + 1) * (degree + 1);
      std::vector<int> hm((size_t)std::max(L.nd * (size_t)L.Cs, nq * (size_t)L.Qs));
      CUDA_CHECK(cudaMemcpy(hm.data(), L.map, sizeof(int) * (size_t)L.nd * L.Cs, cudaMemcpyDeviceToHost));
      FE_REQUIRE(fe_check::bad_map_entries(hm.data(), L.nd, L.C, L.Cs, L.n, bnd) == 0, FE_ERR_CUDA,
                 "tet->dof map failed its consistency check");
      CUDA_CHECK(cudaMemcpy(hm.data(), L.cmap, sizeof(int) * (size_t)nq * L.Qs, cudaMemcpyDeviceToHost));
      FE_REQUIRE(fe_check::bad_map_entries(hm.data(), nq, L.Q, L.Qs, L.n, bnd) == 0, FE_ERR_CUDA,
                 "cube->dof map failed its consistency check");
    }
  }
  build_transfer_tables(h->tt, degree);
  for (int l = 0; l < h->nlev; ++l) {
    if (l > 0) build_level_transfer_index(h->L[l], h->L[l - 1], h->tt);
    launch_build_valence(h->L[l], s);
  }
  std::vector<int> ch = build_children();
  h->children.alloc(48);
  CUDA_CHECK(cudaMemcpy(h->children, ch.data(), sizeof(int) * 48, cudaMemcpyHostToDevice));
  red_init(h->red, h->sms);
  const int nF = h->L.back().n;
  for (auto* v : {&h->x, &h->r, &h->z, &h->p, &h->q, &h->b, &h->e, &h->tmp, &h->xcg}) v->alloc(nF);
  if (degree == 2) h->ps.alloc(nF);
  h->cgp.alloc(1);
  h->cgctl.alloc(2);
  for (auto* v : {&h->r32, &h->z32, &h->p32, &h->q32, &h->e32}) v->alloc(nF);
  h->cs.flag.alloc(1);
  set_coefficient_impl(h.get(), nullptr, s);
  return h.release();
}

void hierarchy_set_coefficient(fe_hierarchy* h, const double* kappa, cudaStream_t s) { set_coefficient_impl(h, kappa, s); }

void hierarchy_destroy(fe_hierarchy* h) { fe_hierarchy_destroy(h); }

// =================================================================== ABI
extern "C" {

void fe_default_opts(fe_solver_opts* o) {
  if (!o) return;
  o->rtol = 1e-8;
  o->max_it = 500;
  o->precond = FE_PC_GMG;
  o->precision = FE_PREC_F64;
  o->cheb_steps = 2;
  o->cheb_lo = 0.1;
  o->cheb_hi = 1.1;
  o->inner_rtol = 3e-5;  // P2 128^3: 2 refinement steps of 5 inner iterations (1e-4: 3 steps, 14 iterations, 40% slower)
  o->inner_max_it = 60;
  o->use_graph = 1;
  o->profile = 0;
  o->wait_timeout_us = 0;
}

long long fe_kernel_launches(void) { return g_launches.load(); }

const char* fe_last_error(void) { return g_err.c_str(); }

int fe_device_count(void) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int fe_mesh_create(int nx, int ny, int nz, fe_mesh** out) {
  API_BEGIN
  FE_REQUIRE(out, FE_ERR_ARG, "null output handle");
  *out = nullptr;
  FE_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1, FE_ERR_ARG, "mesh sizes must be >= 1");
  FE_REQUIRE(nx == ny && ny == nz, FE_ERR_UNSUPPORTED, "only cubic UnitCubeMesh(N,N,N) is supported");
  FE_REQUIRE(nx <= 1024, FE_ERR_ARG, "mesh too large");
  *out = new fe_mesh{nx};
  API_END
}

void fe_mesh_destroy(fe_mesh* m) { delete m; }

int fe_hierarchy_refine(const fe_mesh* coarse, int nrefine, int degree, fe_hierarchy** out) {
  API_BEGIN
  FE_REQUIRE(out, FE_ERR_ARG, "null output handle");
  *out = nullptr;
  FE_REQUIRE(coarse, FE_ERR_ARG, "null mesh");
  *out = hierarchy_create(coarse->N, nrefine, degree);
  API_END
}

void fe_hierarchy_destroy(fe_hierarchy* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  invalidate_graphs(h);
  for (auto& g : h->vgraph)
    if (g.stream) cudaStreamDestroy(g.stream);
  for (auto& L : h->L) bf16_forget_level(&L);
  red_free(h->red);
  delete h;
}

int fe_num_levels(const fe_hierarchy* h) {
  if (!h) {
    fe_set_error("null hierarchy");
    return FE_ERR_ARG;
  }
  return h->nlev;
}

int fe_level_sizes(const fe_hierarchy* h, int level, int* N, long long* n_dofs, long long* n_cells) {
  API_BEGIN
  check_level(h, level);
  const Level& L = h->L[level];
  if (N) *N = L.N;
  if (n_dofs) *n_dofs = L.n;
  if (n_cells) *n_cells = L.C;
  API_END
}

int fe_dof_coordinates(const fe_hierarchy* hc, int level, double* xyz) {
  API_BEGIN
  check_level(hc, level);
  FE_REQUIRE(xyz, FE_ERR_ARG, "null output");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  const Level& L = h->L[level];
  cudaStream_t s = 0;
  double* d = stage_out<double>(h, 2, xyz, (size_t)3 * L.n);
  launch_dof_coords(L, d, s);
  finish_out(xyz, d, (size_t)3 * L.n, s);
  CUDA_CHECK(cudaStreamSynchronize(s));
  API_END
}

int fe_cell_centroids(const fe_hierarchy* hc, int level, double* xyz) {
  API_BEGIN
  check_level(hc, level);
  FE_REQUIRE(xyz, FE_ERR_ARG, "null output");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  const Level& L = h->L[level];
  cudaStream_t s = 0;
  double* d = stage_out<double>(h, 2, xyz, (size_t)3 * L.C);
  launch_centroids(L, d, s);
  finish_out(xyz, d, (size_t)3 * L.C, s);
  CUDA_CHECK(cudaStreamSynchronize(s));
  API_END
}

int fe_boundary_mask(const fe_hierarchy* hc, int level, unsigned char* mask) {
  API_BEGIN
  check_level(hc, level);
  FE_REQUIRE(mask, FE_ERR_ARG, "null output");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  const Level& L = h->L[level];
  cudaStream_t s = 0;
  unsigned char* d = stage_out<unsigned char>(h, 2, mask, (size_t)L.n);
  launch_bmask(L, d, s);
  finish_out(mask, d, (size_t)L.n, s);
  CUDA_CHECK(cudaStreamSynchronize(s));
  API_END
}

int fe_set_coefficient(fe_hierarchy* h, const double* kappa, void* stream) {
  API_BEGIN
  FE_REQUIRE(h, FE_ERR_ARG, "null hierarchy");
  set_coefficient_impl(h, kappa, as_stream(stream));
  API_END
}

int fe_apply_operator(const fe_hierarchy* hc, int level, const void* x, void* y, int dtype, void* stream) {
  API_BEGIN
  check_level(hc, level);
  FE_REQUIRE(x && y && x != y, FE_ERR_ARG, "x and y must be distinct non-null vectors");
  FE_REQUIRE(dtype == FE_F64 || dtype == FE_F32 || dtype == FE_BF16, FE_ERR_ARG, "unknown dtype");
  if (dtype == FE_BF16) FE_REQUIRE(bf16_supported(), FE_ERR_UNSUPPORTED, "bf16 tensor-core apply not available");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  const Level& L = h->L[level];
  cudaStream_t s = as_stream(stream);
  if (dtype == FE_F64) {
    const double* xd = stage_in<double>(h, 0, (const double*)x, L.n, s);
    double* yd = stage_out<double>(h, 1, (double*)y, L.n);
    if (presplit(h, level)) {  // the solver's operator: x split into float pairs first
      launch_split_pairs(L, xd, s);
      apply_enqueue(h, level, xd, yd, dtype, s, L.xs64.p);
    } else {
      apply_enqueue(h, level, xd, yd, dtype, s);
    }
    finish_out((double*)y, yd, L.n, s);
  } else {
    const float* xd = stage_in<float>(h, 0, (const float*)x, L.n, s);
    float* yd = stage_out<float>(h, 1, (float*)y, L.n);
    apply_enqueue(h, level, xd, yd, dtype, s);
    finish_out((float*)y, yd, L.n, s);
    if (dtype == FE_BF16) FE_REQUIRE(bf16_take_error(s) == 0, FE_ERR_TIMEOUT, "tensor-core apply gave up a bounded wait");
  }
  API_END
}

int fe_set_f64_mode(fe_hierarchy* h, int mode) {
  API_BEGIN
  FE_REQUIRE(h, FE_ERR_ARG, "null hierarchy");
  FE_REQUIRE(mode >= FE_F64_NATIVE && mode <= FE_F64_DOUBLE_FLOAT_PAIR, FE_ERR_ARG, "unknown FP64 mode");
  if (h->f64_mode != mode) {
    CUDA_CHECK(cudaDeviceSynchronize());
    h->f64_mode = mode;
    invalidate_graphs(h);
  }
  API_END
}

int fe_set_smoother(fe_hierarchy* h, int smoother) {
  API_BEGIN
  FE_REQUIRE(h, FE_ERR_ARG, "null hierarchy");
  FE_REQUIRE(smoother == FE_SMOOTHER_JACOBI || smoother == FE_SMOOTHER_PATCH, FE_ERR_ARG, "unknown smoother");

  if (h->smoother != smoother) {
    CUDA_CHECK(cudaDeviceSynchronize());
    cudaStream_t s = 0;
    h->smoother = smoother;
    if (smoother == FE_SMOOTHER_PATCH && h->deg >= 2)
      for (int l = 1; l < h->nlev; ++l) {
        Level& L = h->L[l];
        launch_patch_setup(L, s);
        if (!L.z64.p) {
          L.z64.alloc(L.n);
          L.z32.alloc(L.n);
        }
      }
    for (int l = 0; l < h->nlev; ++l) h->L[l].lmax = estimate_lmax(h, l, 20, s);
    invalidate_graphs(h);
    CUDA_CHECK(cudaStreamSynchronize(s));
  }
  API_END
}

int fe_set_geometry_form(fe_hierarchy* h, int form) {
  API_BEGIN
  FE_REQUIRE(h, FE_ERR_ARG, "null hierarchy");
  FE_REQUIRE(form == FE_GEOMETRY_AUTO || form == FE_GEOMETRY_PER_CELL, FE_ERR_ARG, "unknown geometry form");
  CUDA_CHECK(cudaDeviceSynchronize());
  h->geometry_form = form;
  for (int l = 0; l < h->nlev; ++l) {
    launch_uniform_geometry(h->L[l], h->cs.flag, nullptr);
    if (form == FE_GEOMETRY_PER_CELL) h->L[l].uniform = 0;
  }
  invalidate_graphs(h);
  API_END
}

int fe_set_coarse_solver(fe_hierarchy* h, int mode) {
  API_BEGIN
  FE_REQUIRE(h, FE_ERR_ARG, "null hierarchy");
  FE_REQUIRE(mode == FE_COARSE_AUTO || mode == FE_COARSE_DENSE || mode == FE_COARSE_BLOCKED, FE_ERR_ARG,
             "unknown coarse solver");
  CUDA_CHECK(cudaDeviceSynchronize());
  h->coarse_mode = mode;
  if (h->nlev > 1) coarse_setup(h, nullptr);
  invalidate_graphs(h);
  API_END
}

int fe_coarse_info(const fe_hierarchy* h, long long* n_interior, int* bandwidth, int* blocked, long long* bytes,
                   double* setup_ms) {
  API_BEGIN
  FE_REQUIRE(h, FE_ERR_ARG, "null hierarchy");
  if (n_interior) *n_interior = h->cs.nci;
  if (bandwidth) *bandwidth = h->cs.band;
  if (blocked) *blocked = h->cs.blocked;
  if (bytes) *bytes = (long long)h->cs.bytes;
  if (setup_ms) *setup_ms = h->cs.setup_ms;
  API_END
}

int fe_set_smoother_fusion(fe_hierarchy* h, int on) {
  API_BEGIN
  FE_REQUIRE(h, FE_ERR_ARG, "null hierarchy");
  FE_REQUIRE(on == 0 || on == 1, FE_ERR_ARG, "fusion flag must be 0 or 1");
  if (h->fuse_smoother != on) {
    CUDA_CHECK(cudaDeviceSynchronize());
    h->fuse_smoother = on;
    invalidate_graphs(h);
  }
  API_END
}

int fe_apply_mass(const fe_hierarchy* hc, int level, const double* x, double* y, void* stream) {
  API_BEGIN
  check_level(hc, level);
  FE_REQUIRE(x && y && x != y, FE_ERR_ARG, "x and y must be distinct non-null vectors");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  const Level& L = h->L[level];
  cudaStream_t s = as_stream(stream);
  const double* xd = stage_in<double>(h, 0, x, L.n, s);
  double* yd = stage_out<double>(h, 1, y, L.n);
  mass_enqueue(h, L, xd, yd, s);
  finish_out(y, yd, L.n, s);
  API_END
}

int fe_diagonal(const fe_hierarchy* hc, int level, double* diag, void* stream) {
  API_BEGIN
  check_level(hc, level);
  FE_REQUIRE(diag, FE_ERR_ARG, "null output");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  Level& L = h->L[level];
  cudaStream_t s = as_stream(stream);
  double* d = stage_out<double>(h, 1, diag, L.n);
  launch_diag(L, d, s);
  finish_out(diag, d, L.n, s);
  API_END
}

int fe_lambda_max(const fe_hierarchy* h, int level, double* lmax) {
  API_BEGIN
  check_level(h, level);
  FE_REQUIRE(lmax, FE_ERR_ARG, "null output");
  *lmax = h->L[level].lmax;
  API_END
}

int fe_prolong(const fe_hierarchy* hc, int lf, const double* xc, double* xf, int accumulate, void* stream) {
  API_BEGIN
  check_level(hc, lf);
  FE_REQUIRE(lf >= 1, FE_ERR_ARG, "level_fine must be >= 1");
  FE_REQUIRE(xc && xf, FE_ERR_ARG, "null vector");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  cudaStream_t s = as_stream(stream);
  const Level &F = h->L[lf], &C = h->L[lf - 1];
  const double* xcd = stage_in<double>(h, 0, xc, C.n, s);
  double* xfd = stage_out<double>(h, 1, xf, F.n);
  if (accumulate && xfd != xf) CUDA_CHECK(cudaMemcpyAsync(xfd, xf, sizeof(double) * F.n, cudaMemcpyHostToDevice, s));
  launch_prolong<double>(h, lf, xcd, xfd, accumulate != 0, s);
  finish_out(xf, xfd, F.n, s);
  API_END
}

int fe_restrict(const fe_hierarchy* hc, int lf, const double* rf, double* rc, int zero_boundary, void* stream) {
  API_BEGIN
  check_level(hc, lf);
  FE_REQUIRE(lf >= 1, FE_ERR_ARG, "level_fine must be >= 1");
  FE_REQUIRE(rf && rc, FE_ERR_ARG, "null vector");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  cudaStream_t s = as_stream(stream);
  const Level &F = h->L[lf], &C = h->L[lf - 1];
  const double* rfd = stage_in<double>(h, 0, rf, F.n, s);
  double* rcd = stage_out<double>(h, 1, rc, C.n);
  launch_restrict<double>(h, lf, rfd, nullptr, rcd, zero_boundary != 0, s);
  finish_out(rc, rcd, C.n, s);
  API_END
}

int fe_smooth(const fe_hierarchy* hc, int level, const void* b, void* x, int steps, double lo, double hi, int dtype,
              void* stream) {
  API_BEGIN
  check_level(hc, level);
  FE_REQUIRE(b && x && steps >= 1 && hi > lo && lo > 0, FE_ERR_ARG, "invalid smoother arguments");
  FE_REQUIRE(dtype == FE_F64 || dtype == FE_F32 || dtype == FE_BF16, FE_ERR_ARG, "unknown dtype");
  if (dtype == FE_BF16) FE_REQUIRE(bf16_supported(), FE_ERR_UNSUPPORTED, "bf16 tensor-core apply not available");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  Level& L = h->L[level];
  cudaStream_t s = as_stream(stream);
  if (dtype == FE_F64) {
    const double* bd = stage_in<double>(h, 0, (const double*)b, L.n, s);
    double* xd = stage_out<double>(h, 1, (double*)x, L.n);
    if (xd != x) CUDA_CHECK(cudaMemcpyAsync(xd, x, sizeof(double) * L.n, cudaMemcpyHostToDevice, s));
    smooth_enqueue<double>(h, level, bd, xd, h->tmp, h->e, steps, lo, hi, false, dtype, s);
    finish_out((double*)x, xd, L.n, s);
  } else {
    const float* bd = stage_in<float>(h, 0, (const float*)b, L.n, s);
    float* xd = stage_out<float>(h, 1, (float*)x, L.n);
    if (xd != x) CUDA_CHECK(cudaMemcpyAsync(xd, x, sizeof(float) * L.n, cudaMemcpyHostToDevice, s));
    smooth_enqueue<float>(h, level, bd, xd, h->q32, h->p32, steps, lo, hi, false, dtype, s);
    finish_out((float*)x, xd, L.n, s);
  }
  API_END
}

int fe_coarse_solve(const fe_hierarchy* hc, const double* b, double* x, void* stream) {
  API_BEGIN
  FE_REQUIRE(hc && hc->nlev > 1, FE_ERR_ARG, "coarse solve needs a hierarchy with at least 2 levels");
  FE_REQUIRE(b && x && (const void*)b != (const void*)x, FE_ERR_ARG, "b and x must be distinct non-null vectors");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  cudaStream_t s = as_stream(stream);
  const Level& L0 = h->L[0];
  const double* bd = stage_in<double>(h, 0, b, L0.n, s);
  double* xd = stage_out<double>(h, 1, x, L0.n);
  coarse_solve<double>(h, bd, xd, s);
  finish_out(x, xd, L0.n, s);
  API_END
}

int fe_vcycle(const fe_hierarchy* hc, const void* b, void* x, int dtype, void* stream) {
  API_BEGIN
  FE_REQUIRE(hc && hc->nlev > 1, FE_ERR_ARG, "V-cycle needs a hierarchy with at least 2 levels");
  FE_REQUIRE(b && x, FE_ERR_ARG, "null vector");
  FE_REQUIRE(dtype == FE_F64 || dtype == FE_F32 || dtype == FE_BF16, FE_ERR_ARG, "unknown dtype");
  if (dtype == FE_BF16) FE_REQUIRE(bf16_supported(), FE_ERR_UNSUPPORTED, "bf16 tensor-core apply not available");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  Level& F = h->L[h->nlev - 1];
  cudaStream_t s = as_stream(stream);
  g_sp = SmootherParams{};
  const size_t es = dtype == FE_F64 ? sizeof(double) : sizeof(float);
  void* fb = dtype == FE_F64 ? (void*)F.b64.p : (void*)F.b32.p;
  void* fx = dtype == FE_F64 ? (void*)F.x64.p : (void*)F.x32.p;
  CUDA_CHECK(cudaMemcpyAsync(fb, b, es * F.n, cudaMemcpyDefault, s));
  run_vcycle(h, dtype, false, s);
  CUDA_CHECK(cudaMemcpyAsync(x, fx, es * F.n, cudaMemcpyDefault, s));
  if (!is_device_ptr(x)) CUDA_CHECK(cudaStreamSynchronize(s));
  if (dtype == FE_BF16) FE_REQUIRE(bf16_take_error(s) == 0, FE_ERR_TIMEOUT, "tensor-core apply gave up a bounded wait");
  API_END
}

int fe_load_vector(const fe_hierarchy* hc, const double* f, double* b, void* stream) {
  API_BEGIN
  FE_REQUIRE(hc && f && b, FE_ERR_ARG, "null argument");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  cudaStream_t s = as_stream(stream);
  const Level& F = h->L[h->nlev - 1];
  const double* bd = rhs_to_load(h, f, FE_RHS_NODAL_F, s);
  CUDA_CHECK(cudaMemcpyAsync(b, bd, sizeof(double) * F.n, cudaMemcpyDefault, s));
  if (!is_device_ptr(b)) CUDA_CHECK(cudaStreamSynchronize(s));
  API_END
}

int fe_quadrature_points(const fe_hierarchy* hc, double* xyz) {
  API_BEGIN
  FE_REQUIRE(hc && xyz, FE_ERR_ARG, "null argument");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  const Level& F = h->L[h->nlev - 1];
  const size_t n = (size_t)3 * FE_QUAD_POINTS * F.C;
  cudaStream_t s = 0;
  double* d = stage_out<double>(h, 2, xyz, n);
  launch_quad_points(F, d, s);
  finish_out(xyz, d, n, s);
  CUDA_CHECK(cudaStreamSynchronize(s));
  API_END
}

int fe_load_vector_quadrature(const fe_hierarchy* hc, const double* f_qp, double* b, void* stream) {
  API_BEGIN
  FE_REQUIRE(hc && f_qp && b, FE_ERR_ARG, "null argument");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  cudaStream_t s = as_stream(stream);
  const Level& F = h->L[h->nlev - 1];
  const double* bd = rhs_to_load(h, f_qp, FE_RHS_QUAD_F, s);
  CUDA_CHECK(cudaMemcpyAsync(b, bd, sizeof(double) * F.n, cudaMemcpyDefault, s));
  if (!is_device_ptr(b)) CUDA_CHECK(cudaStreamSynchronize(s));
  API_END
}

int fe_solve_poisson(fe_hierarchy* h, const double* rhs, int rhs_kind, const double* bc_values,
                     const fe_solver_opts* opts, double* u, fe_solve_stats* stats, void* stream) {
  API_BEGIN
  FE_REQUIRE(h && rhs && u, FE_ERR_ARG, "null argument");
  const fe_solver_opts o = resolve_opts(opts);
  FE_REQUIRE(o.precision == FE_PREC_F64 || o.precond == FE_PC_GMG, FE_ERR_ARG, "mixed precision needs the GMG preconditioner");
  if (o.precision == FE_PREC_MIXED_BF16) {
    FE_REQUIRE(bf16_supported(), FE_ERR_UNSUPPORTED, "bf16 tensor-core apply not available");
  }
  FE_REQUIRE(o.precision == FE_PREC_F64 || h->nlev > 1, FE_ERR_ARG, "mixed precision needs at least 2 levels");
  cudaStream_t s = as_stream(stream);
  const Level& F = h->L[h->nlev - 1];
  const auto t0 = std::chrono::steady_clock::now();
  g_sp = SmootherParams{o.cheb_steps, o.cheb_lo, o.cheb_hi};
  // per-phase timers for this call (thread-local, cleared again on every exit path)
  struct ProfGuard {
    PhaseProf* p;
    explicit ProfGuard(PhaseProf* q) : p(q) {
      if (p) p->reset();
      g_prof = p;
    }
    ~ProfGuard() { g_prof = nullptr; }
  } prof_guard(o.profile ? &h->prof : nullptr);
  const double* b = rhs_to_load(h, rhs, rhs_kind, s);
  const double* g = nullptr;
  if (bc_values) {  // symmetric elimination of u = g on the boundary
    g = stage_in<double>(h, 2, bc_values, F.n, s);
    launch_bc_lift(F, g, h->b, s);
  }
  double* ud = is_device_ptr(u) ? u : h->x.p;
  fe_solve_stats st{};
  st.outer_iterations = 1;
  PcgResult res;
  if (o.precond == FE_PC_FMG) {
    // one full-multigrid cycle, then the residual of its solution for the stats
    run_fmg(h, b, o.max_it, o.use_graph != 0 && !o.profile, s);
    Level& Ft = h->L[h->nlev - 1];
    CUDA_CHECK(cudaMemcpyAsync(ud, Ft.fx64, sizeof(double) * Ft.n, cudaMemcpyDeviceToDevice, s));
    apply_enqueue(h, h->nlev - 1, Ft.fx64, Ft.y64, FE_F64, s);
    launch_sub64(Ft.n, b, Ft.y64, Ft.w64, s);
    ReduceCtx& R = h->red;
    launch_dot<double>(R, Ft.n, b, b, S_BB, s);
    launch_dot<double>(R, Ft.n, Ft.w64.p, Ft.w64.p, S_RR, s);
    CUDA_CHECK(cudaMemcpyAsync(R.h_scal, R.scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
    CUDA_CHECK(cudaStreamSynchronize(s));
    res.bb = R.h_scal[S_BB];
    res.rr = R.h_scal[S_RR];
    res.it = o.max_it;
    if (!std::isfinite(res.rr)) res.status = FE_ERR_NAN;
  } else if (o.precision == FE_PREC_F64) {
    res = pcg64(h, b, ud, o, s);
    st.fine_applies_f64 = res.applies;
    st.apply_ms = res.apply_ms;
    st.apply_timed = res.apply_timed;
  } else {
    res = refine(h, b, ud, o, o.precision == FE_PREC_MIXED_F32 ? FE_F32 : FE_BF16, &st, s);
    st.fine_applies_f64 = res.applies;
  }
  // the boundary rows are the decoupled identity equations u_j = g_j: set them exactly (an iterative solve
  // leaves them within its tolerance)
  if (g) launch_set_boundary(F, g, ud, s);
  finish_out(u, ud, F.n, s);
  CUDA_CHECK(cudaStreamSynchronize(s));
  if (o.precision == FE_PREC_MIXED_BF16)
    FE_REQUIRE(bf16_take_error(s) == 0, FE_ERR_TIMEOUT, "tensor-core apply gave up a bounded wait");
  st.iterations = res.it;
  st.bnorm = std::sqrt(res.bb);
  st.rel_residual = res.bb > 0 ? std::sqrt(res.rr / res.bb) : 0.0;
  st.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (o.profile) h->prof.collect(st, h->nlev);
  if (stats) *stats = st;
  if (res.status == FE_ERR_NO_CONVERGENCE) FE_FAIL(FE_ERR_NO_CONVERGENCE, "iteration limit reached before rtol");
  if (res.status == FE_ERR_NAN) FE_FAIL(FE_ERR_NAN, "residual norm is not finite");
  API_END
}

int fe_adjoint_gradient(fe_hierarchy* h, const double* rhs, int rhs_kind, const double* u_d, const double* u_ckpt,
                        const fe_solver_opts* opts, double* dJ, double* J, double* u_out, void* stream) {
  API_BEGIN
  FE_REQUIRE(h && rhs && u_d && dJ, FE_ERR_ARG, "null argument");
  fe_solver_opts o = resolve_opts(opts);
  o.precision = FE_PREC_F64;
  cudaStream_t s = as_stream(stream);
  Level& F = h->L[h->nlev - 1];
  const int n = F.n;
  g_sp = SmootherParams{o.cheb_steps, o.cheb_lo, o.cheb_hi};
  double *u = h->e, *Me = h->tmp, *lam = h->z;
  if (u_ckpt) {
    const double* uc = stage_in<double>(h, 0, u_ckpt, n, s);
    CUDA_CHECK(cudaMemcpyAsync(u, uc, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    const double* b = rhs_to_load(h, rhs, rhs_kind, s);
    PcgResult r1 = pcg64(h, b, u, o, s);
    if (r1.status != FE_OK) FE_FAIL(r1.status, "forward solve failed");
  }
  const double* ud = stage_in<double>(h, 1, u_d, n, s);
  // Me = M (u - u_d); J = (u - u_d)^T M (u - u_d)
  launch_sub64(n, u, ud, h->b, s);
  mass_enqueue(h, F, h->b, Me, s);
  launch_dot<double>(h->red, n, h->b, Me, S_DOT, s);
  double Jh = 0.0;
  CUDA_CHECK(cudaMemcpyAsync(&Jh, h->red.scal + S_DOT, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  // adjoint right-hand side -2 M (u - u_d), zero on the Dirichlet dofs
  CUDA_CHECK(cudaMemsetAsync(h->b, 0, sizeof(double) * n, s));
  launch_axpy64(n, -2.0, Me, h->b, s);
  launch_zero_boundary64(F, h->b, s);
  PcgResult r2 = pcg64(h, h->b, lam, o, s);
  if (r2.status != FE_OK) FE_FAIL(r2.status, "adjoint solve failed");
  double* g = stage_out<double>(h, 3, dJ, F.C);
  launch_gradient(F, u, lam, g, s);
  finish_out(dJ, g, F.C, s);
  if (u_out) {
    CUDA_CHECK(cudaMemcpyAsync(u_out, u, sizeof(double) * n, cudaMemcpyDefault, s));
  }
  CUDA_CHECK(cudaStreamSynchronize(s));
  if (J) *J = Jh;
  API_END
}

int fe_objective(const fe_hierarchy* hc, const double* u, const double* u_d, double* J, void* stream) {
  API_BEGIN
  FE_REQUIRE(hc && u && u_d && J, FE_ERR_ARG, "null argument");
  fe_hierarchy* h = const_cast<fe_hierarchy*>(hc);
  cudaStream_t s = as_stream(stream);
  const Level& F = h->L[h->nlev - 1];
  const double* ud = stage_in<double>(h, 0, u, F.n, s);
  const double* udd = stage_in<double>(h, 1, u_d, F.n, s);
  launch_sub64(F.n, ud, udd, h->tmp, s);
  mass_enqueue(h, F, h->tmp, h->q, s);
  launch_dot<double>(h->red, F.n, h->tmp.p, h->q.p, S_DOT, s);
  CUDA_CHECK(cudaMemcpyAsync(J, h->red.scal + S_DOT, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_CHECK(cudaStreamSynchronize(s));
  API_END
}

}  // extern "C"
