/*
 * fe.h -- C ABI of the GB300 matrix-free finite element Poisson library.
 *
 * The library solves -div(kappa grad u) = f on the unit cube with Dirichlet
 * conditions on all six faces, discretised with continuous Lagrange P1, P2 or
 * P3 elements on a tetrahedral UnitCubeMesh, by conjugate gradients
 * preconditioned with a geometric multigrid V-cycle over a nested mesh
 * hierarchy, or by full multigrid.  This is the Poisson model problem of the
 * paper (Section 2, Eqs. 1-4: mesh, function space, Dirichlet BCs, right-hand
 * side, bilinear form; Section 3: multigrid with two Chebyshev smoothing
 * iterations per level, Jacobi or vertex-star patch preconditioned, and a
 * direct coarse solve).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Return value: FE_OK (0) on success, a negative FE_ERR_* code on failure; no
 *   entry point aborts or throws.  fe_last_error() returns a message for the
 *   last failure on the calling thread.
 * Vectors: every double/float pointer argument may point to HOST memory
 *   (pageable or pinned) or to DEVICE memory of the current CUDA device.  The
 *   library detects which (cudaPointerGetAttributes) and stages host data
 *   through its own device buffers; results are complete in host memory when
 *   the call returns.  Device data is read/written in stream order on
 *   `stream` (a cudaStream_t, NULL = the legacy default stream); the call may
 *   return before device-side work finishes unless stated otherwise.
 * Ownership: handles are created and owned by the library and released with
 *   the matching *_destroy.  Vectors are owned by the caller.  A hierarchy
 *   holds device workspace on the device that was current when it was
 *   created, which must be current for every call on it; calls on the same
 *   hierarchy must not run concurrently (from several host threads or on
 *   several streams at once).  Hierarchies on different devices of one
 *   process are independent.
 * Mesh: UnitCubeMesh(N,N,N), vertex (i,j,k) at (i,j,k)/N with index
 *   i + (N+1)(j + (N+1)k); cube (ci,cj,ck) has index q = ci + N(cj + N ck) and
 *   is split into the six Kuhn tetrahedra 6q..6q+5 that share its main
 *   diagonal (the paper does not state the split; this is the reading taken).
 *   Level l of a hierarchy is the same construction with N0 * 2^l cubes.
 * Degrees of freedom: P1 dofs are the vertices.  P2 dofs are the points of
 *   the 2N lattice (2N+1 per axis); dofs 0..(N+1)^3-1 are the vertices in
 *   vertex order, followed by edge midpoints grouped by the parity class of
 *   their lattice coordinates in the order (1,0,0),(0,1,0),(0,0,1),(1,1,0),
 *   (1,0,1),(0,1,1),(1,1,1); inside a class the sub-lattice (L - parity)/2 is
 *   numbered x fastest.  P3 dofs are the points of the 3N lattice numbered
 *   lexicographically (x fastest).  Use fe_dof_coordinates() to evaluate
 *   fields.
 * Boundary: a dof is a boundary dof if any lattice coordinate is 0 or kN.  The
 *   operator is the symmetric elimination of the Dirichlet dofs: boundary
 *   rows and columns of A are replaced by the identity.
 * Coefficient: kappa is one FP64 value per fine cell (NULL means kappa = 1);
 *   coarse levels use the arithmetic mean of the 8 child cells.
 * Debug checks: with FE_DEBUG_CHECKS=1 in the environment, fe_hierarchy_refine
 *   also reads every level's tet->dof and cube->dof maps back to the host and
 *   checks them (dofs in range, Dirichlet encoding consistent with the
 *   boundary, no dof repeated within a cell), failing with FE_ERR_CUDA.
 */
#ifndef FE_GB300_H
#define FE_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FE_OK 0
#define FE_ERR_ARG (-1)             /* invalid argument (null handle, bad size, level out of range) */
#define FE_ERR_CUDA (-2)            /* a CUDA runtime call or kernel launch failed */
#define FE_ERR_NOMEM (-3)           /* device or host allocation failed */
#define FE_ERR_NO_CONVERGENCE (-4)  /* the iteration limit was reached before the tolerance */
#define FE_ERR_NAN (-5)             /* a residual norm became NaN or Inf */
#define FE_ERR_TIMEOUT (-6)         /* a bounded device-side wait gave up */
#define FE_ERR_UNSUPPORTED (-7)     /* valid request that the library does not support */

/* ---- arithmetic types of an operator application ---- */
#define FE_F64 0   /* vectors double, arithmetic FP64 */
#define FE_F32 1   /* vectors float, arithmetic FP32 */
#define FE_BF16 2  /* vectors float; each dof split into two bf16 terms and contracted on the tensor cores
                      (tcgen05, FP32 accumulation in TMEM) against exact bf16 reference tables; P1, P2, P3 */

/* ---- arithmetic of FP64 operator applications (fe_set_f64_mode) ---- */
#define FE_F64_NATIVE 0        /* FP64 FMA on the FP64 pipe */
#define FE_F64_DOUBLE_FLOAT 1       /* float-pair (hi + lo, ~48-bit) arithmetic on the FP32 pipes, FP64 in and
                                       out, with the faster layout per degree (P1: per cube, P2: per tet); on
                                       Kuhn tets (G = c M) the P2 element is c times one integer matrix, applied
                                       to exact fixed-point FP32 limbs of the float-pair products c x */
#define FE_F64_DOUBLE_FLOAT_TET 2   /* the same arithmetic, one thread per tet (persistent, prefetching) */
#define FE_F64_DOUBLE_FLOAT_CUBE 3  /* the same arithmetic, one thread per cube (27/8 dofs split and scattered once) */
#define FE_F64_DOUBLE_FLOAT_PAIR 4  /* P2: the same arithmetic, two tets per thread in packed FP32x2 instructions */

/* ---- preconditioners and precision modes of fe_solve_poisson ---- */
#define FE_PC_JACOBI 0
#define FE_PC_GMG 1
#define FE_PC_FMG 2   /* no Krylov method: full multigrid is the whole solve (paper Section 3): b restricted to every
                         level, a direct solve on the coarsest, then on each finer level the interpolated coarser
                         solution corrected by max_it V-cycles; rtol is not a stopping test (stats report the
                         final residual); FP64 only */
#define FE_PREC_F64 0         /* everything FP64 */
#define FE_PREC_MIXED_F32 1   /* FP64 iterative refinement around an FP32 GMG-PCG */
#define FE_PREC_MIXED_BF16 2  /* as FE_PREC_MIXED_F32 with bf16 tensor-core smoother applications */

/* ---- right-hand side kinds ---- */
#define FE_RHS_LOAD 0     /* rhs is the assembled load vector b (boundary entries = Dirichlet values) */
#define FE_RHS_NODAL_F 1  /* rhs holds nodal values of f; b = M f on interior rows, 0 on the boundary */
#define FE_RHS_QUAD_F 2   /* rhs holds f at the quadrature points of fe_quadrature_points ([n_cells][FE_QUAD_POINTS]);
                             b_i = sum_K sum_q w_q |det J_K| f(x_Kq) phi_i(xi_q) on interior rows, 0 on the boundary */

/* Quadrature rule of FE_RHS_QUAD_F: the conical-product Gauss rule with 3
 * points per direction on the reference tet (27 points, exact for polynomials
 * of degree 3): xi = (u, (1-u) v, (1-u)(1-v) w) for u, v, w in the 3 Gauss-
 * Legendre nodes of [0, 1], u slowest and w fastest. */
#define FE_QUAD_POINTS 27

/* ---- phases of the per-level solve timers (fe_solve_stats.phase_ms, with opts.profile) ---- */
#define FE_MAX_LEVELS 9      /* levels of a hierarchy: nrefine <= 8 */
#define FE_PHASE_APPLY 0     /* operator applications outside the smoother: CG's A p, multigrid residuals */
#define FE_PHASE_SMOOTH 1    /* Chebyshev smoothing: its operator applications and vector (or patch) updates */
#define FE_PHASE_TRANSFER 2  /* restriction and prolongation */
#define FE_PHASE_COARSE 3    /* the direct coarse solve */
#define FE_PHASE_BLAS1 4     /* dot products and vector updates of CG and of iterative refinement */
#define FE_NUM_PHASES 5

typedef struct fe_mesh fe_mesh;
typedef struct fe_hierarchy fe_hierarchy;
typedef struct fe_batch fe_batch;

typedef struct fe_solver_opts {
  double rtol;        /* stop when ||b - A u||_2 <= rtol ||b||_2 (unpreconditioned 2-norm) */
  int max_it;         /* CG iteration limit (mixed precision: outer refinement steps, at most 100; refinement
                         also stops with FE_ERR_NO_CONVERGENCE after 3 steps in a row that reduce ||r|| < 2x) */
  int precond;        /* FE_PC_JACOBI, FE_PC_GMG (CG preconditioned by one V-cycle) or FE_PC_FMG */
  int precision;      /* FE_PREC_* */
  int cheb_steps;     /* Chebyshev iterations per smoothing (2 in the paper's options) */
  double cheb_lo;     /* Chebyshev interval [cheb_lo, cheb_hi] * lambda_max(D^-1 A) */
  double cheb_hi;
  double inner_rtol;  /* mixed precision: inner FP32 solve tolerance */
  int inner_max_it;   /* mixed precision: inner iteration limit per refinement step */
  int use_graph;      /* nonzero: replay each V-cycle from a captured CUDA graph */
  int profile;        /* nonzero: time every CG operator application (stats.apply_ms) and every phase of every
                         level (stats.phase_ms) with CUDA events; graph replay is off while profiling */
  int wait_timeout_us; /* bound of every device-side wait of the persistent batched kernel (0 = 5 s) */
} fe_solver_opts;

typedef struct fe_solve_stats {
  int iterations;        /* CG iterations (sum of inner iterations for mixed precision) */
  int outer_iterations;  /* refinement steps (mixed precision), else 1 */
  double rel_residual;   /* final ||b - A u|| / ||b|| in FP64 */
  double bnorm;          /* ||b||_2 */
  double solve_ms;       /* host wall time of the solve */
  int fine_applies_f64;  /* FP64 fine-level operator applications */
  int fine_applies_low;  /* FP32/bf16 fine-level operator applications */
  double apply_ms;       /* profile: summed device time of the timed CG operator applications */
  int apply_timed;       /* profile: number of operator applications in apply_ms */
  int levels_timed;      /* profile: levels with entries in phase_ms (the hierarchy's levels), else 0 */
  double phase_ms[FE_NUM_PHASES][FE_MAX_LEVELS]; /* profile: device time (ms) of each phase FE_PHASE_* on each level
                         (index 0 = coarsest), summed over the solve: the per-level multigrid log */
} fe_solve_stats;

/* Fill `opts` with the defaults: rtol 1e-8, max_it 500, GMG, FP64,
 * 2 Chebyshev steps on [0.1, 1.1] lambda_max, inner_rtol 3e-5, inner_max_it 60,
 * graphs on, profiling off, default wait bound. */
void fe_default_opts(fe_solver_opts* opts);

/* Message of the last failure on this thread ("" if none).  The string is
 * owned by the library and valid until the next call on this thread. */
const char* fe_last_error(void);

/* Number of visible CUDA devices (0 without a GPU); never fails. */
int fe_device_count(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (each replay of a captured graph counts every kernel node); never fails. */
long long fe_kernel_launches(void);

/* ---- mesh and hierarchy (paper Section 2: UnitCubeMesh, MeshHierarchy, FunctionSpace) ---- */

/* Create UnitCubeMesh(nx, ny, nz).  The library supports cubes only:
 * nx == ny == nz >= 1, else FE_ERR_UNSUPPORTED / FE_ERR_ARG.  Host-only. */
int fe_mesh_create(int nx, int ny, int nz, fe_mesh** out);
void fe_mesh_destroy(fe_mesh* mesh);

/* Refine `coarse` uniformly `nrefine` times (0..8) and build the degree-1, 2
 * or 3 Lagrange space on every level (Sec. 2; degree 3 is the paper's),
 * uploading the levels to the current CUDA device; other degrees give
 * FE_ERR_UNSUPPORTED.  Level 0 is the coarse mesh, level nrefine the finest.
 * The coefficient is kappa = 1 until fe_set_coefficient() is called.
 * Degree 3 (20 dofs per tet, dofs numbered lexicographically on the 3N
 * lattice): the operator applies each tet's element through the gradient at
 * its 10 P2 nodes (677 operations), in float pairs (FP64 default), FP64
 * (FE_F64_NATIVE), FP32 or on the bf16 tensor cores; the batched solver is
 * P1/P2 only and returns FE_ERR_UNSUPPORTED for a degree-3 hierarchy. */
int fe_hierarchy_refine(const fe_mesh* coarse, int nrefine, int degree, fe_hierarchy** out);
void fe_hierarchy_destroy(fe_hierarchy* h);

/* Number of levels (nrefine + 1), or a negative code. */
int fe_num_levels(const fe_hierarchy* h);

/* Sizes of `level`: cubes per axis N, dofs n = (kN+1)^3, cells 6 N^3. */
int fe_level_sizes(const fe_hierarchy* h, int level, int* N, long long* n_dofs, long long* n_cells);

/* Coordinates of the dofs of `level`: xyz[3*i + a], n_dofs x 3 doubles. */
int fe_dof_coordinates(const fe_hierarchy* h, int level, double* xyz);

/* Centroids of the cells of `level`: xyz[3*c + a], n_cells x 3 doubles. */
int fe_cell_centroids(const fe_hierarchy* h, int level, double* xyz);

/* Boundary flags of the dofs of `level` (1 = Dirichlet dof), n_dofs bytes. */
int fe_boundary_mask(const fe_hierarchy* h, int level, unsigned char* mask);

/* Set the cell coefficient kappa (n_cells of the finest level, FP64; NULL =
 * 1) and rebuild everything that depends on it on every level: per-cell
 * geometric factors, Jacobi diagonals, Chebyshev eigenvalue estimates and the
 * coarse Cholesky factor.  Synchronises `stream`. */
int fe_set_coefficient(fe_hierarchy* h, const double* kappa_cells, void* stream);

/* ---- operator application (paper Section 2, Eq. 4: the bilinear form) ---- */

/* y = A_l x on `level`, matrix-free: for every tet K, y_K += kappa_K
 * int_K grad(u) . grad(v) applied to the gathered dofs x_K, scatter-added
 * into y; boundary rows give y_i = x_i and boundary entries of x are treated
 * as 0 in interior rows.  dtype FE_F64: x, y double (P2 in the default FP64
 * mode: x is first split into the float pairs that the solver's operator
 * gathers, held by the hierarchy, then applied by that operator).  FE_F32: float.
 * FE_BF16: float vectors, each dof entering as two bf16 terms (16 significant
 * bits) contracted on the tensor cores with FP32 accumulation: per tile of 128
 * cells one GEMM against the reference stiffness tables (one combined table
 * when every cell's G is c M, the case on UnitCubeMesh; else six), P1/P2/P3.
 * x and y must not overlap. */
int fe_apply_operator(const fe_hierarchy* h, int level, const void* x, void* y, int dtype, void* stream);

/* Choose how FP64 operator applications (dtype FE_F64, the FP64 solver and
 * V-cycle) compute the element contraction: FE_F64_NATIVE (FP64 FMAs) or
 * FE_F64_DOUBLE_FLOAT (default: the same operator on the FP32 pipes, in
 * float-pair arithmetic with error-free transformations or, for P2 on Kuhn
 * tets, exact fixed-point limbs; about 47 significant bits, several times
 * faster on GB300 whose FP64 pipe issues 2 FMAs/clk/SM).  Dofs, results and
 * every other step stay FP64. */
int fe_set_f64_mode(fe_hierarchy* h, int mode);

/* ---- preconditioner of the Chebyshev level smoother (fe_set_smoother) ---- */
#define FE_SMOOTHER_JACOBI 0  /* D^-1 (the default) */
#define FE_SMOOTHER_PATCH 1   /* vertex-star patches, additive, exact local solves (Sec. 3, PatchPC star) */

/* Precondition the Chebyshev smoother of every level >= 1 with D^-1
 * (FE_SMOOTHER_JACOBI) or with the vertex-star patch preconditioner
 * (FE_SMOOTHER_PATCH): M^-1 r = sum_p R_p^T (R_p A R_p^T)^-1 R_p r over one
 * patch per mesh vertex, the dofs of the vertex's open star (the vertex and,
 * for P2, the midpoints of its 14 Kuhn edges) without Dirichlet dofs, and
 * M^-1 r = r on Dirichlet rows (Sec. 3: PatchPC with star patches around
 * vertices as the preconditioner of the level smoother).  The Chebyshev
 * interval becomes [lo, hi] * lambda_max(M^-1 A) (re-estimated here and after
 * every fe_set_coefficient).  P2 builds one 15 x 15 local inverse per vertex,
 * P3 one 65 x 65 (the vertex, the 2 nodes of each of its 14 edges, its 36 face
 * centroids), stored in FP64 (P2 only), float pairs and FP32 (P3: 25.7 KB per
 * vertex, 0.9 GB at UnitCubeMesh 32^3); for P1 a star patch is its vertex
 * alone and the patch preconditioner is exactly Jacobi. */
int fe_set_smoother(fe_hierarchy* h, int smoother);

/* ---- geometric factors of the operator kernels (fe_set_geometry_form) ---- */
#define FE_GEOMETRY_AUTO 0      /* one value per cell when every cell's G is c M (always on UnitCubeMesh), else six */
#define FE_GEOMETRY_PER_CELL 1  /* the six stored factors of G per cell in every operator kernel */

/* Every Kuhn tet of UnitCubeMesh(N) has J = (1/N) P U (P a permutation, U the
 * upper-triangular matrix of ones), so G = |det J| J^-1 J^-T = (1/N) M with
 * M = [[2,-1,0],[-1,2,-1],[0,-1,1]] for every cell (Sec. 2: the mesh of the
 * paper's Poisson problem).  Set-up computes G per cell from the vertex
 * coordinates and checks this cell by cell; with FE_GEOMETRY_AUTO the operator
 * kernels then read one value kappa_K h / w per cell and use M, with
 * FE_GEOMETRY_PER_CELL they read the six stored factors (for comparison; the
 * results agree to rounding).  Synchronises the current device. */
int fe_set_geometry_form(fe_hierarchy* h, int form);

/* ---- coarse direct solver (fe_set_coarse_solver) ---- */
#define FE_COARSE_AUTO 0     /* dense inverse factor up to 16384 interior coarse dofs, blocked band factor above */
#define FE_COARSE_DENSE 1    /* explicit L^-1 and L^-T: two parallel dense triangular products per solve
                                (native FP64), or one dense product with A^-1 = L^-T L^-1 held as float
                                pairs (the float-pair FP64 modes and FP32) */
#define FE_COARSE_BLOCKED 2  /* band Cholesky factor; blocks of B = bandwidth rows with the inverse of each
                                diagonal block and the block left of it: 4 nb block products per solve */

/* Choose how the coarsest level's interior block A = L L^T (FP64 Cholesky,
 * Sec. 3: a direct factorisation of the coarsest multigrid level) is applied:
 * the dense explicit inverse of L (fast for small coarse levels; n^2 storage),
 * or the band factor in blocks of B = w rows (w the half-bandwidth
 * k (1 + e + e^2) for e interior points per axis): forward substitution
 * y_I = D_I (b_I - E_I y_{I-1}) and the transposed backward pass, with D_I the
 * inverse of the I-th diagonal block and E_I = L_{I,I-1}; storage about
 * 4 n B doubles, e.g. 23 GB for the P3 16^3 coarse level (103,823 unknowns,
 * w = 6771).  Refactors the coarse level (synchronises the current device). */
int fe_set_coarse_solver(fe_hierarchy* h, int mode);

/* The coarse solver in use: interior unknowns, half-bandwidth, 1 if blocked,
 * device bytes of its factor data and the time of its last factorisation (ms). */
int fe_coarse_info(const fe_hierarchy* h, long long* n_interior, int* bandwidth, int* blocked, long long* bytes,
                   double* setup_ms);

/* Chebyshev-Jacobi smoothing (Sec. 3: two Chebyshev iterations per level
 * visit) with the operator fused (on = 1) or not (on = 0, the default).
 * Fused, each smoothing step that needs y = A x is one launch: every interior
 * dof carries a countdown of the tets (or cubes) that scatter into it, and
 * the thread whose contribution ends it applies d = c1 d + c2 D^-1 (b - y),
 * x += d to that dof, so no separate vector kernel streams y, x and d again.
 * On GB300 the countdown atomics (one per scattered value, with the result
 * returned) cost about three times the operator itself, so the default is the
 * operator kernel followed by one vector kernel.  The fused forms exist for
 * the FP32 operator and the float-pair FP64 operators; native-FP64 and bf16
 * smoothing always use two kernels.  Results agree up to the rounding order
 * of the atomic sums. */
int fe_set_smoother_fusion(fe_hierarchy* h, int on);

/* y = M_l x with the consistent mass matrix (all dofs, no boundary change). */
int fe_apply_mass(const fe_hierarchy* h, int level, const double* x, double* y, void* stream);

/* diag = diagonal of A_l (boundary entries 1), n_dofs doubles. */
int fe_diagonal(const fe_hierarchy* h, int level, double* diag, void* stream);

/* Largest eigenvalue estimate of D^-1 A_l (or of M^-1 A_l with the patch
 * smoother) that scales the Chebyshev interval of `level`. */
int fe_lambda_max(const fe_hierarchy* h, int level, double* lmax);

/* ---- multigrid components (paper Section 3: MG with Chebyshev smoothing, direct coarse solve) ---- */

/* xf (+)= P xc: prolongation from level_fine-1 to level_fine by exact
 * interpolation of the coarse Lagrange function at the fine nodes.
 * accumulate != 0 adds to xf.  FP64. */
int fe_prolong(const fe_hierarchy* h, int level_fine, const double* xc, double* xf, int accumulate, void* stream);

/* rc = P^T rf: restriction from level_fine to level_fine-1 (the transpose of
 * fe_prolong).  zero_boundary != 0 sets the coarse boundary entries to 0. */
int fe_restrict(const fe_hierarchy* h, int level_fine, const double* rf, double* rc, int zero_boundary, void* stream);

/* `steps` Chebyshev iterations for A_l x = b preconditioned as chosen by
 * fe_set_smoother (Jacobi by default) on [cheb_lo, cheb_hi] * lambda_max,
 * starting from x (in/out).  dtype FE_F64 (double vectors) or FE_F32/FE_BF16
 * (float vectors). */
int fe_smooth(const fe_hierarchy* h, int level, const void* b, void* x, int steps, double cheb_lo, double cheb_hi,
              int dtype, void* stream);

/* x = A_0^-1 b on the coarsest level with the FP64 Cholesky factor of its
 * interior block (x_bd = b_bd).  b and x must not overlap (FE_ERR_ARG when
 * they are the same vector). */
int fe_coarse_solve(const fe_hierarchy* h, const double* b, double* x, void* stream);

/* x = V(b): one V-cycle on the finest level (pre-smoothing from 0, residual,
 * restriction, recursion, coarse Cholesky solve, prolongation,
 * post-smoothing).  dtype as fe_smooth; the coarse solve is FP64. */
int fe_vcycle(const fe_hierarchy* h, const void* b, void* x, int dtype, void* stream);

/* ---- solves ---- */

/* b = M f on interior rows and b_bd = 0, from nodal values f (n_dofs). */
int fe_load_vector(const fe_hierarchy* h, const double* f_nodal, double* b, void* stream);

/* Physical coordinates of the FE_QUAD_POINTS quadrature points of every cell of
 * the finest level (paper Section 2: the linear form of f v dx evaluated by
 * quadrature): xyz[(cell * FE_QUAD_POINTS + q) * 3 + axis], host or device
 * pointer of 3 * FE_QUAD_POINTS * n_cells doubles (caller-owned).  Synchronous. */
int fe_quadrature_points(const fe_hierarchy* h, double* xyz);

/* b = the load vector of f by quadrature (FE_RHS_QUAD_F): f_qp holds f at the
 * points of fe_quadrature_points ([n_cells][FE_QUAD_POINTS]); b (n_dofs) gets
 * b_i = sum_K sum_q w_q |det J_K| f(x_Kq) phi_i(xi_q) on interior rows and 0 on
 * the boundary.  FP64 accumulation; host or device pointers. */
int fe_load_vector_quadrature(const fe_hierarchy* h, const double* f_qp, double* b, void* stream);

/* Solve A u = b on the finest level by PCG (Jacobi or GMG V-cycle), by full
 * multigrid (FE_PC_FMG), or by FP64 iterative refinement around a
 * reduced-precision GMG-PCG.  rhs: FE_RHS_LOAD, FE_RHS_NODAL_F or
 * FE_RHS_QUAD_F (see above).
 * bc_values: Dirichlet data u = g on the boundary (Sec. 2, Eq. 1: the
 *   boundary condition of the strong form), n_dofs doubles of which only the
 *   boundary entries are read; NULL means g = 0.  The load is eliminated
 *   symmetrically: b_i -= sum_j A_ij g_j over the boundary dofs j for every
 *   interior row i, b_j = g_j on the boundary (with FE_RHS_LOAD the boundary
 *   entries of rhs are then ignored), so u_j = g_j exactly on the boundary.
 * u: in = initial guess (ignored, taken as 0), out = solution.  Synchronises
 * `stream`.  Returns FE_ERR_NO_CONVERGENCE if max_it is reached (u holds the
 * last iterate) and FE_ERR_NAN on a non-finite residual.  opts NULL =
 * defaults; stats may be NULL. */
int fe_solve_poisson(fe_hierarchy* h, const double* rhs, int rhs_kind, const double* bc_values,
                     const fe_solver_opts* opts, double* u, fe_solve_stats* stats, void* stream);

/* Adjoint gradient of J(kappa) = (u - u_d)^T M (u - u_d) = int (u_h - I_h u_d)^2
 * where A(kappa) u = b: solves A u = b (unless u_ckpt != NULL, which is taken
 * as the checkpointed forward solution), then A lambda = -2 M (u - u_d) with
 * lambda_bd = 0, and returns dJ_dkappa[K] = int_K grad(lambda) . grad(u) for
 * every fine cell (n_cells doubles) and J (one double, may be NULL).  u_out
 * (may be NULL) receives u.  rhs as in fe_solve_poisson. */
int fe_adjoint_gradient(fe_hierarchy* h, const double* rhs, int rhs_kind, const double* u_d, const double* u_ckpt,
                        const fe_solver_opts* opts, double* dJ_dkappa, double* J, double* u_out, void* stream);

/* J = (u - u_d)^T M (u - u_d) on the finest level (the objective whose
 * gradient fe_adjoint_gradient returns); J is one double in host memory. */
int fe_objective(const fe_hierarchy* h, const double* u, const double* u_d, double* J, void* stream);

/* ---- batched solves (extension form: many independent problems, one launch) ----
 *
 * A batch holds `nprob` independent Poisson problems, problem p on
 * UnitCubeMesh(N0[p]) refined nrefine[p] times with Lagrange degree[p]
 * (1 or 2); all problems need the same number of levels (2..6).  Host-only
 * arguments; the hierarchies live on the current device. */
int fe_batch_create(int nprob, const int* N0, const int* nrefine, const int* degree, fe_batch** out);
void fe_batch_destroy(fe_batch* batch);

/* The hierarchy of problem p (owned by the batch: do not destroy it).  Use it
 * for fe_set_coefficient (per-problem kappa) and the mesh queries. */
int fe_batch_hierarchy(fe_batch* batch, int p, fe_hierarchy** h);

/* Solve all problems of the batch, FP64 GMG-PCG (2 Chebyshev-Jacobi steps per
 * level, FP64 Cholesky coarse solve), right-hand sides given as nodal values
 * f_nodal[p] (b = M f, Dirichlet rows 0), solutions written to u[p].  All of
 * f_nodal[p] and u[p] must be DEVICE pointers.  One persistent cooperative
 * kernel runs every phase of every iteration for all problems (grid-wide
 * barriers between phases; converged problems drop out), replayed from a
 * captured CUDA graph when opts->use_graph; the first graph solve runs the
 * autotuner (cell-block size, CTAs per SM).  stats: nprob entries (may be
 * NULL).  FE_ERR_TIMEOUT if a grid barrier exceeded opts->wait_timeout_us
 * (the kernel then returns early; the batch stays usable);
 * FE_ERR_NO_CONVERGENCE / FE_ERR_NAN if any problem failed.  Synchronises
 * `stream`. */
int fe_solve_batched(fe_batch* batch, const double* const* f_nodal, double* const* u, const fe_solver_opts* opts,
                     fe_solve_stats* stats, void* stream);

/* The schedule chosen by the autotuner (or the default before tuning). */
int fe_batch_schedule(const fe_batch* batch, int* cell_block, int* dof_block, int* ctas_per_sm);

/* ---- allocation-free entry point (no counterpart in the paper) ----
 *
 * Deterministic FP64 dot product *out = sum_i x[i] y[i] for callers that may
 * not allocate device memory: a host application that owns the whole device
 * memory budget through its own pool, or a latency-critical loop in which
 * cudaMalloc/cudaFree (which can synchronise the device) are not allowed.
 * The call allocates nothing: its partial sums live in a static device array
 * of the library (16384 partials + 2 slots, 128.5 KiB, held by every GPU that
 * loads the library until the process exits).
 *   x, y: DEVICE pointers of the current device to n doubles each (host
 *         pointers and memory of another device are rejected with FE_ERR_ARG,
 *         since staging them would need device memory).  The library cannot
 *         see the length of a buffer: x and y must hold n doubles.
 *   n:    0 <= n <= 67,108,864 (4096 elements per partial sum); larger n is
 *         rejected with FE_ERR_ARG.
 *   out:  one double, device pointer of the current device or host pointer;
 *         a host `out` makes the call synchronise `stream`.
 * The result does not depend on scheduling (fixed summation order).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current.  Under CUDA's default lazy module loading that
 * first lookup also loads the library's device code on that device, which
 * can itself allocate device memory and synchronise: make the first call
 * during set-up, before any stream capture and before the code that must not
 * allocate.
 * Every call shares the one array and overwrites it: calls that overlap on the
 * GPU (several streams, or several host threads) race and must be serialised
 * by the caller. */
int fe_dot_noalloc(const double* x, const double* y, long long n, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FE_GB300_H */
