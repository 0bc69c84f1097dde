"""Plain, slow, FP64 CPU oracle for the finite element Poisson path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: it is used by ``tests/``, by ``__graft_entry__.smoke()``
and by ``bench.py``'s CPU-baseline and reference legs, and by nothing else.
It shares no code with the CUDA library (the only module both use is
``fe_inputs``, which draws seeded random inputs and holds no FE arithmetic).

What it computes, written out from the definitions in the paper:

* the Poisson problem -div(kappa grad u) = f on the unit cube with homogeneous
  (or given) Dirichlet data on all six faces (Section 2, Eq. 1, and the boundary
  conditions of the paper's Poisson script);
* its Galerkin discretisation in continuous Lagrange P1/P2/P3 on a tetrahedral
  ``UnitCubeMesh`` (Section 2, the weak form Eq. 4): the global stiffness
  A_ij = int kappa grad(phi_j) . grad(phi_i) dx and mass M_ij = int phi_j phi_i dx
  are ASSEMBLED into CSR matrices (the paper's PETSc path uses assembled AIJ
  matrices, Section 3 and the telescoping listing), from element matrices
  obtained by quadrature of the physical basis gradients;
* Dirichlet conditions by symmetric elimination (identity rows/columns);
* a geometric multigrid hierarchy of nested meshes (``MeshHierarchy``,
  Section 2 and Section 3) with prolongation = exact interpolation of the coarse
  finite element function at the fine nodes and restriction = its transpose,
  rediscretised coarse operators, Chebyshev smoothing with two iterations per
  level (the level-smoother options of the paper's FMG listing), preconditioned
  by Jacobi or by additive vertex-star patches with exact local solves (the
  paper's PatchPC with star patches), and a direct Cholesky coarse solve
  (Section 3 factorises the coarsest level directly);
* conjugate gradients (Jacobi- or V-cycle-preconditioned), full multigrid as the
  whole solve (the paper's outer solver), the load vector of f by quadrature, the
  L2 error against an analytic solution (Section 2 measures the error against the
  exact solution), and the discrete adjoint gradient dJ/dkappa of
  J = (u-u_d)^T M (u-u_d).

Readings where the paper is silent (each also listed in the design notes):
Kuhn 6-tet split of each cube; level l of the hierarchy is the Kuhn mesh of
N0*2^l cubes per axis; coarse kappa = mean of the 8 child cells; b = M I_h f;
Chebyshev interval [0.1, 1.1] * lambda_max(D^-1 A) with lambda_max estimated by
Lanczos from CG; stopping on the unpreconditioned ||r||_2 <= rtol ||b||_2.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants, brute force and convergence rates.
"""
import ctypes
import os

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# The six Kuhn (Freudenthal) simplices of a cube: tet t visits the cube
# corners origin, origin+e[p0], origin+e[p0]+e[p1], origin+(1,1,1).
KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
# Local P2 edge order inside a tet (pairs of local vertex numbers).
P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
# Parity classes of the P2 lattice in global numbering order: class 0 are the
# mesh vertices, then x-, y-, z-edge midpoints, then xy-, xz-, yz-face
# diagonals, then body diagonals.
PARITY_CLASSES = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1))

# Local P3 node order inside a tet: the 4 vertices, then for each edge (a, b) of
# ``P2_EDGES`` the node at 2/3 lam_a + 1/3 lam_b and then the one at 1/3 lam_a +
# 2/3 lam_b, then the centroid of each face, the face opposite vertex 0, 1, 2, 3.
P3_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))

_UNIT = np.eye(3, dtype=np.int64)


# ---------------------------------------------------------------- mesh ------
class Mesh:
    """Tetrahedral UnitCubeMesh(N, N, N) (Section 2, the paper's Poisson script).

    Vertex (i,j,k) has index i + (N+1)*(j + (N+1)*k) and coordinates (i,j,k)/N.
    Cube (ci,cj,ck) has index q = ci + N*(cj + N*ck); its six Kuhn tets are
    cells 6q..6q+5 in the order of ``KUHN_PERMS``.
    """

    def __init__(self, N):
        self.N = int(N)
        r = np.arange(N + 1)
        k, j, i = np.meshgrid(r, r, r, indexing="ij")
        self.vertex_lattice = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
        self.coords = self.vertex_lattice / float(N)
        rc = np.arange(N)
        ck, cj, ci = np.meshgrid(rc, rc, rc, indexing="ij")
        origin = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
        Q = origin.shape[0]
        lat = np.empty((Q, 6, 4, 3), dtype=np.int64)
        for t, perm in enumerate(KUHN_PERMS):
            p = origin.copy()
            lat[:, t, 0] = p
            p = p + _UNIT[perm[0]]
            lat[:, t, 1] = p
            p = p + _UNIT[perm[1]]
            lat[:, t, 2] = p
            lat[:, t, 3] = origin + 1
        self.cell_vertex_lattice = lat.reshape(Q * 6, 4, 3)
        self.cells = self.vertex_index(self.cell_vertex_lattice.reshape(-1, 3)).reshape(-1, 4)

    def vertex_index(self, L):
        n1 = self.N + 1
        return L[:, 0] + n1 * (L[:, 1] + n1 * L[:, 2])

    @property
    def n_cells(self):
        return self.cells.shape[0]

    @property
    def n_vertices(self):
        return self.coords.shape[0]

    def jacobians(self, sel=slice(None)):
        """J with columns p1-p0, p2-p0, p3-p0 for the selected cells."""
        p = self.coords[self.cells[sel]]
        return (p[:, 1:, :] - p[:, :1, :]).transpose(0, 2, 1)

    def centroids(self):
        return self.coords[self.cells].mean(axis=1)


def dof_count(N, degree):
    """Number of continuous P_k Lagrange dofs on the N^3 Kuhn mesh: (kN+1)^3."""
    return (degree * N + 1) ** 3


def lattice_dof_index(L, N, degree):
    """Global dof number of the lattice points L (m,3) of the (degree*N)-lattice.

    P1 and P3: lexicographic (x fastest) over the (kN+1)^3 lattice.  P2: points
    grouped by the parity class of their lattice coordinates (``PARITY_CLASSES``
    order), lexicographic inside a class over the sub-lattice a = (L - parity)/2
    of extent N+1-parity.
    """
    L = np.asarray(L, dtype=np.int64)
    if degree in (1, 3):
        n1 = degree * N + 1
        return L[:, 0] + n1 * (L[:, 1] + n1 * L[:, 2])
    if degree != 2:
        raise ValueError("degree must be 1, 2 or 3")
    par = L % 2
    code = par[:, 0] + 2 * par[:, 1] + 4 * par[:, 2]
    code_to_class = np.empty(8, dtype=np.int64)
    for c, p in enumerate(PARITY_CLASSES):
        code_to_class[p[0] + 2 * p[1] + 4 * p[2]] = c
    cls = code_to_class[code]
    sizes = N + 1 - np.array(PARITY_CLASSES, dtype=np.int64)
    counts = sizes.prod(axis=1)
    offsets = np.concatenate([[0], np.cumsum(counts)[:-1]])
    a = (L - par) // 2
    s = sizes[cls]
    return offsets[cls] + a[:, 0] + s[:, 0] * (a[:, 1] + s[:, 1] * a[:, 2])


class Space:
    """Continuous Lagrange P1, P2 or P3 on a ``Mesh`` (``FunctionSpace(mesh, "CG", k)``).

    Every P_k node of a Kuhn tet lies on the kN lattice: a node with barycentrics
    (i0, i1, i2, i3)/k sits at sum_v i_v * vertex_v on the N lattice, scaled by k.
    """

    def __init__(self, mesh, degree):
        self.mesh = mesh
        self.degree = int(degree)
        N = mesh.N
        self.n = dof_count(N, degree)
        vl = mesh.cell_vertex_lattice  # (C,4,3) on the N lattice
        if degree == 1:
            lat = vl
        elif degree == 2:
            v2 = 2 * vl
            edges = np.stack([vl[:, a] + vl[:, b] for a, b in P2_EDGES], axis=1)
            lat = np.concatenate([v2, edges], axis=1)  # (C,10,3) on the 2N lattice
        elif degree == 3:
            v3 = 3 * vl
            edges = np.stack([2 * vl[:, a] + vl[:, b] if near_a else vl[:, a] + 2 * vl[:, b]
                              for a, b in P2_EDGES for near_a in (True, False)], axis=1)
            faces = np.stack([vl[:, a] + vl[:, b] + vl[:, c] for a, b, c in P3_FACES], axis=1)
            lat = np.concatenate([v3, edges, faces], axis=1)  # (C,20,3) on the 3N lattice
        else:
            raise ValueError("degree must be 1, 2 or 3")
        self.cell_lattice = lat
        C, nd = lat.shape[:2]
        self.ndof_cell = nd
        self.cell_dofs = lattice_dof_index(lat.reshape(-1, 3), N, degree).reshape(C, nd)
        # dof -> lattice point (inverse of the numbering)
        m = degree * N
        r = np.arange(m + 1)
        k, j, i = np.meshgrid(r, r, r, indexing="ij")
        allL = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
        idx = lattice_dof_index(allL, N, degree)
        self.dof_lattice = np.empty_like(allL)
        self.dof_lattice[idx] = allL
        self.coords = self.dof_lattice / float(m)
        self.boundary = np.any((self.dof_lattice == 0) | (self.dof_lattice == m), axis=1)


# ------------------------------------------------------- reference element --
def tet_quadrature(n):
    """Collapsed-coordinate (conical product) Gauss-Legendre rule on the reference tet.

    xi = u, eta = (1-u) v, zeta = (1-u)(1-v) w with n Gauss points per
    direction; exact for polynomials of total degree <= 2n-3.
    """
    t, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    U, V, W = np.meshgrid(t, t, t, indexing="ij")
    WU, WV, WW = np.meshgrid(w, w, w, indexing="ij")
    xi = np.stack([U.ravel(), ((1 - U) * V).ravel(), ((1 - U) * (1 - V) * W).ravel()], axis=1)
    wt = (WU * WV * WW * (1 - U) ** 2 * (1 - V)).ravel()
    return xi, wt


def ref_basis(degree, xi):
    """Values (m,nd) and reference gradients (m,nd,3) of the P1/P2/P3 basis at points xi (m,3).

    Barycentrics lam = (1-xi-eta-zeta, xi, eta, zeta).  P1: phi_v = lam_v.
    P2: phi_v = lam_v (2 lam_v - 1) for the vertices, phi_ab = 4 lam_a lam_b for
    the edges in ``P2_EDGES`` order.  P3 (node order of ``P3_FACES``' comment):
    phi_v = lam_v (3 lam_v - 1)(3 lam_v - 2) / 2, the edge node nearer a
    phi = 9/2 lam_a lam_b (3 lam_a - 1), the face node of (a, b, c)
    phi = 27 lam_a lam_b lam_c: each is the cubic that is 1 at its node and 0 at
    the other 19 (it vanishes on the planes lam = 0, 1/3, 2/3 through them).
    """
    xi = np.atleast_2d(xi)
    m = xi.shape[0]
    lam = np.stack([1.0 - xi.sum(axis=1), xi[:, 0], xi[:, 1], xi[:, 2]], axis=1)
    dlam = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    if degree == 1:
        return lam, np.broadcast_to(dlam, (m, 4, 3)).copy()
    if degree == 3:
        phi = np.empty((m, 20))
        dphi = np.empty((m, 20, 3))
        for v in range(4):
            L = lam[:, v]
            phi[:, v] = 0.5 * L * (3 * L - 1) * (3 * L - 2)
            dphi[:, v] = (0.5 * (27 * L * L - 18 * L + 2))[:, None] * dlam[v]
        for e, (a, b) in enumerate(P2_EDGES):
            for h, (p, q) in enumerate(((a, b), (b, a))):  # node nearer p
                Lp, Lq = lam[:, p], lam[:, q]
                phi[:, 4 + 2 * e + h] = 4.5 * Lp * Lq * (3 * Lp - 1)
                dphi[:, 4 + 2 * e + h] = 4.5 * ((Lq * (6 * Lp - 1))[:, None] * dlam[p]
                                               + (Lp * (3 * Lp - 1))[:, None] * dlam[q])
        for f, (a, b, c) in enumerate(P3_FACES):
            La, Lb, Lc = lam[:, a], lam[:, b], lam[:, c]
            phi[:, 16 + f] = 27 * La * Lb * Lc
            dphi[:, 16 + f] = 27 * ((Lb * Lc)[:, None] * dlam[a] + (La * Lc)[:, None] * dlam[b]
                                    + (La * Lb)[:, None] * dlam[c])
        return phi, dphi
    phi = np.empty((m, 10))
    dphi = np.empty((m, 10, 3))
    for v in range(4):
        phi[:, v] = lam[:, v] * (2 * lam[:, v] - 1)
        dphi[:, v] = (4 * lam[:, v] - 1)[:, None] * dlam[v]
    for e, (a, b) in enumerate(P2_EDGES):
        phi[:, 4 + e] = 4 * lam[:, a] * lam[:, b]
        dphi[:, 4 + e] = 4 * (lam[:, a][:, None] * dlam[b] + lam[:, b][:, None] * dlam[a])
    return phi, dphi


# ------------------------------------------------------- element matrices ---
def element_stiffness(mesh, degree, kappa=None, sel=slice(None), nq=None):
    """A_K[i,j] = kappa_K * sum_q w_q |det J| (J^-T grad phi_j) . (J^-T grad phi_i).

    The integrand has degree 2(k-1); the n=3 conical rule (exact to degree 3)
    covers P1/P2, n=4 (exact to degree 5) P3.
    """
    xi, w = tet_quadrature(nq if nq is not None else max(3, degree + 1))
    _, dphi = ref_basis(degree, xi)
    J = mesh.jacobians(sel)
    det = np.linalg.det(J)
    JinvT = np.linalg.inv(J).transpose(0, 2, 1)
    grads = np.einsum("cij,qdj->cqdi", JinvT, dphi)
    A = np.einsum("q,cqdi,cqei->cde", w, grads, grads) * np.abs(det)[:, None, None]
    if kappa is not None:
        A *= np.asarray(kappa)[sel][:, None, None]
    return A


def element_mass(mesh, degree, sel=slice(None), nq=None):
    """M_K[i,j] = sum_q w_q |det J| phi_i phi_j (degree 2k: the n=4 rule, exact to
    degree 5, for P1/P2; n=5, exact to degree 7, for P3)."""
    xi, w = tet_quadrature(nq if nq is not None else max(4, degree + 2))
    phi, _ = ref_basis(degree, xi)
    det = np.abs(np.linalg.det(mesh.jacobians(sel)))
    ref = np.einsum("q,qd,qe->de", w, phi, phi)
    return det[:, None, None] * ref[None]


def _assemble(space, elem_fn, chunk=1 << 16):
    C = space.mesh.n_cells
    nd = space.ndof_cell
    out = sp.csr_matrix((space.n, space.n))
    for s in range(0, C, chunk):
        sel = slice(s, min(C, s + chunk))
        Ae = elem_fn(sel)
        cd = space.cell_dofs[sel]
        rows = np.repeat(cd, nd, axis=1).ravel()
        cols = np.tile(cd, (1, nd)).ravel()
        out = out + sp.coo_matrix((Ae.ravel(), (rows, cols)), shape=(space.n, space.n)).tocsr()
    out.sum_duplicates()
    return out


def assemble_stiffness(space, kappa=None):
    """Global (unconstrained) stiffness matrix in CSR."""
    return _assemble(space, lambda sel: element_stiffness(space.mesh, space.degree, kappa, sel))


def assemble_mass(space):
    """Global consistent mass matrix in CSR."""
    return _assemble(space, lambda sel: element_mass(space.mesh, space.degree, sel))


def dirichlet_eliminate(A, boundary):
    """Zero the boundary rows and columns of A and put 1 on their diagonal."""
    keep = sp.diags((~boundary).astype(np.float64))
    return (keep @ A @ keep + sp.diags(boundary.astype(np.float64))).tocsr()


def apply_rows(space, kappa, x, rows):
    """Rows ``rows`` of y = A_bc x, computed cell by cell (for large meshes).

    Only the cells that touch a requested row are visited; boundary rows give
    y_i = x_i and boundary columns are dropped, as in ``dirichlet_eliminate``.
    """
    rows = np.asarray(rows, dtype=np.int64)
    want = np.zeros(space.n, dtype=bool)
    want[rows] = True
    cells = np.nonzero(want[space.cell_dofs].any(axis=1))[0]
    xb = np.where(space.boundary, 0.0, x)
    y = np.zeros(space.n)
    for s in range(0, cells.size, 1 << 15):
        sel = cells[s:s + (1 << 15)]
        Ae = element_stiffness(space.mesh, space.degree, kappa, sel)
        cd = space.cell_dofs[sel]
        np.add.at(y, cd, np.einsum("cde,ce->cd", Ae, xb[cd]))
    y = np.where(space.boundary, x, y)
    return y[rows]


def apply_rows_mass(space, x, rows):
    """Rows ``rows`` of y = M x (consistent mass, all dofs), computed cell by cell."""
    rows = np.asarray(rows, dtype=np.int64)
    want = np.zeros(space.n, dtype=bool)
    want[rows] = True
    cells = np.nonzero(want[space.cell_dofs].any(axis=1))[0]
    y = np.zeros(space.n)
    for s in range(0, cells.size, 1 << 15):
        sel = cells[s:s + (1 << 15)]
        Me = element_mass(space.mesh, space.degree, sel)
        cd = space.cell_dofs[sel]
        np.add.at(y, cd, np.einsum("cde,ce->cd", Me, x[cd]))
    return y[rows]


# ---------------------------------------------------------------- level -----
class Level:
    """One level of the hierarchy: space, kappa, assembled A (with BCs), diagonal."""

    def __init__(self, N, degree, kappa=None):
        self.mesh = Mesh(N)
        self.space = Space(self.mesh, degree)
        self.kappa = None if kappa is None else np.asarray(kappa, dtype=np.float64)
        self.A_free = assemble_stiffness(self.space, self.kappa)
        self.A = dirichlet_eliminate(self.A_free, self.space.boundary)
        self.diag = self.A.diagonal().copy()
        self._M = None

    @property
    def n(self):
        return self.space.n

    @property
    def M(self):
        if self._M is None:
            self._M = assemble_mass(self.space)
        return self._M


def locate_in_mesh(mesh, pts, tol=1e-12):
    """For each point, a containing cell of ``mesh`` and its reference coordinates.

    The cube is found from the coordinates; the six tets of that cube are tried
    in order and the first with all barycentrics >= -tol is taken.
    """
    N = mesh.N
    cube = np.minimum(np.floor(pts * N + tol).astype(np.int64), N - 1)
    cube = np.maximum(cube, 0)
    q = cube[:, 0] + N * (cube[:, 1] + N * cube[:, 2])
    cell = np.full(pts.shape[0], -1, dtype=np.int64)
    ref = np.zeros_like(pts)
    for t in range(6):
        c = 6 * q + t
        J = mesh.jacobians(c)
        p0 = mesh.coords[mesh.cells[c, 0]]
        xi = np.linalg.solve(J, (pts - p0)[:, :, None])[:, :, 0]
        lam0 = 1.0 - xi.sum(axis=1)
        inside = (xi.min(axis=1) >= -tol) & (lam0 >= -tol) & (cell < 0)
        cell[inside] = c[inside]
        ref[inside] = xi[inside]
    if np.any(cell < 0):
        raise RuntimeError("point location failed")
    return cell, ref


def prolongation(coarse, fine):
    """Sparse P (n_fine x n_coarse): row i holds the coarse basis functions at fine node i."""
    cell, ref = locate_in_mesh(coarse.mesh, fine.space.coords)
    phi, _ = ref_basis(coarse.space.degree, ref)
    cols = coarse.space.cell_dofs[cell]
    rows = np.repeat(np.arange(fine.n), phi.shape[1])
    vals = phi.ravel()
    keep = np.abs(vals) > 1e-14
    P = sp.coo_matrix((vals[keep], (rows[keep], cols.ravel()[keep])), shape=(fine.n, coarse.n)).tocsr()
    P.sum_duplicates()
    return P


def coarsen_kappa(coarse_mesh, fine_mesh, kappa_fine):
    """Coarse cell kappa = arithmetic mean of the fine cells whose centroid it contains."""
    parent, _ = locate_in_mesh(coarse_mesh, fine_mesh.centroids())
    s = np.bincount(parent, weights=kappa_fine, minlength=coarse_mesh.n_cells)
    c = np.bincount(parent, minlength=coarse_mesh.n_cells)
    return s / c


# ---------------------------------------------------------- products -----
# The solves' CSR products go through csr_omp.c (the textbook row-by-row
# product with the rows split over OpenMP threads) when it has been built by
# oracle/build_oracle.py, else through scipy's product (one thread).  Both sum
# every row in column order.
THREADS = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
_CSR_LIB = []


def _csr_lib():
    if not _CSR_LIB:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liboracle_csr.so")
        lib = None
        if os.path.exists(path):
            lib = ctypes.CDLL(path)
            lib.oracle_csr_matvec.restype = None
            lib.oracle_csr_matvec.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.c_int]
        _CSR_LIB.append(lib)
    return _CSR_LIB[0]


def matvec(A, x, threads=None):
    """y = A x for a CSR matrix A (the solves' operator products)."""
    lib = _csr_lib()
    x = np.ascontiguousarray(x, dtype=np.float64)
    if lib is None or not sp.isspmatrix_csr(A) or A.indices.dtype != np.int32 or x.ndim != 1:
        return A @ x
    ip = getattr(A, "_oracle_indptr64", None)
    if ip is None:
        ip = np.ascontiguousarray(A.indptr, dtype=np.int64)
        A._oracle_indptr64 = ip
    idx = np.ascontiguousarray(A.indices)
    dat = np.ascontiguousarray(A.data, dtype=np.float64)
    y = np.empty(A.shape[0])
    lib.oracle_csr_matvec(A.shape[0], ip.ctypes.data, idx.ctypes.data, dat.ctypes.data, x.ctypes.data, y.ctypes.data,
                          int(threads or THREADS))
    return y


# ----------------------------------------------------------- Krylov -------
def pcg(apply_A, b, apply_M, rtol, maxit, x0=None):
    """Preconditioned conjugate gradients; stops on ||r||_2 <= rtol ||b||_2.

    Returns (x, iterations, history of ||r||/||b||, Lanczos coefficients).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x)
    bnorm = np.linalg.norm(b)
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0]
    alphas, betas = [], []
    it = 0
    while hist[-1] > rtol and it < maxit:
        q = apply_A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        alphas.append(alpha)
        if hist[-1] <= rtol:
            break
        z = apply_M(r)
        rz_new = r @ z
        beta = rz_new / rz
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    return x, it, hist, (alphas, betas)


def lanczos_lambda_max(alphas, betas):
    """Largest eigenvalue of the Lanczos tridiagonal built from CG coefficients."""
    k = len(alphas)
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = np.sqrt(betas[i]) / alphas[i]
    return float(np.linalg.eigvalsh(T)[-1])


def estimate_lambda_max(A, diag, n_steps=20, seed=0, prec=None):
    """lambda_max(M^-1 A) estimated from n_steps of PCG on a seeded random rhs (M = D, Jacobi, unless
    ``prec`` applies another M^-1)."""
    b = np.random.default_rng(seed).uniform(-1, 1, A.shape[0])
    _, _, _, (al, be) = pcg(lambda v: A @ v, b, prec if prec is not None else (lambda v: v / diag),
                            rtol=0.0, maxit=n_steps)
    return lanczos_lambda_max(al, be)


def chebyshev(apply_A, diag, b, x, lo, hi, steps, prec=None):
    """Chebyshev semi-iteration for A x = b preconditioned by M^-1 on [lo, hi] (M = D, Jacobi, unless
    ``prec`` applies another M^-1, e.g. the vertex-star patch preconditioner).

    theta = (hi+lo)/2, delta = (hi-lo)/2; d_0 = M^-1 r_0 / theta; then
    rho_k = 1/(2 theta/delta - rho_{k-1}),
    d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) M^-1 r_k; x_{k+1} = x_k + d_k.
    """
    if prec is None:
        prec = lambda v: v / diag  # noqa: E731
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = x.copy()
    r = b - apply_A(x)
    d = prec(r) / theta
    for k in range(steps):
        x += d
        if k == steps - 1:
            break
        r = b - apply_A(x)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * prec(r)
        rho = rho_new
    return x


# ------------------------------------------------- vertex-star patches -----
def ref_node_barycentrics(degree):
    """Barycentric coordinates (nd, 4) of the local Lagrange nodes in the local dof order of ``Space``."""
    I4 = np.eye(4)
    if degree == 1:
        return I4.copy()
    if degree == 2:
        return np.concatenate([I4, [(I4[a] + I4[b]) / 2 for a, b in P2_EDGES]])
    edge = [(2 * I4[a] + I4[b]) / 3 if near_a else (I4[a] + 2 * I4[b]) / 3 for a, b in P2_EDGES for near_a in (True, False)]
    face = [(I4[a] + I4[b] + I4[c]) / 3 for a, b, c in P3_FACES]
    return np.concatenate([I4, edge, face])


def star_patches(level):
    """Vertex-star patches (the paper's PatchPC with star construction around vertices, Section 3): for each mesh
    vertex v, the dofs of the open star of v -- the mesh entities whose closure contains v, i.e. the nodes of the
    cells around v whose barycentric coordinate for v is positive -- without the Dirichlet dofs.  Returns a list
    of sorted dof arrays, one per vertex (empty ones dropped)."""
    space, mesh = level.space, level.mesh
    bary = ref_node_barycentrics(space.degree)
    groups = [[] for _ in range(mesh.n_vertices)]
    for a in range(4):
        local = np.nonzero(bary[:, a] > 0)[0]
        for K in range(mesh.n_cells):
            groups[mesh.cells[K, a]].append(space.cell_dofs[K, local])
    out = []
    for g in groups:
        d = np.unique(np.concatenate(g)) if g else np.empty(0, dtype=np.int64)
        d = d[~space.boundary[d]]
        if d.size:
            out.append(d)
    return out


class PatchPreconditioner:
    """Additive Schwarz over the vertex-star patches with exact local solves (PatchPC's default additive
    combination and direct sub-solver): M^-1 r = sum_p R_p^T (R_p A R_p^T)^-1 R_p r on the free dofs, and
    M^-1 r = r on the Dirichlet dofs (their rows are the identity, as for Jacobi)."""

    def __init__(self, level):
        self.level = level
        self.patches = star_patches(level)
        A = level.A_free
        self.bd = level.space.boundary
        self.by_size = {}
        for p in self.patches:
            self.by_size.setdefault(p.size, []).append(p)
        self.blocks = []
        for size, ps in self.by_size.items():
            idx = np.stack(ps)  # (P, size)
            Ap = np.stack([A[p][:, p].toarray() for p in ps])
            self.blocks.append((idx, np.linalg.inv(Ap)))

    def __call__(self, r):
        z = np.zeros_like(r)
        for idx, Ainv in self.blocks:
            np.add.at(z, idx, np.einsum("pij,pj->pi", Ainv, r[idx]))
        z[self.bd] = r[self.bd]
        return z


# -------------------------------------------------------- multigrid -------
class Hierarchy:
    """Nested levels UnitCubeMesh(N0 * 2^l), l = 0..nrefine (``MeshHierarchy``)."""

    def __init__(self, N0, nrefine, degree, kappa_fine=None, cheb_steps=2,
                 cheb_lo=0.1, cheb_hi=1.1, eig_steps=20, smoother="jacobi"):
        """smoother: "jacobi" (Chebyshev preconditioned by D^-1) or "patch" (by the vertex-star patches, the
        paper's PatchPC choice)."""
        self.degree = degree
        Ns = [N0 * 2 ** l for l in range(nrefine + 1)]
        kappas = [None] * len(Ns)
        if kappa_fine is not None:
            kappas[-1] = np.asarray(kappa_fine, dtype=np.float64)
            for l in range(len(Ns) - 2, -1, -1):
                kappas[l] = coarsen_kappa(Mesh(Ns[l]), Mesh(Ns[l + 1]), kappas[l + 1])
        self.levels = [Level(N, degree, k) for N, k in zip(Ns, kappas)]
        self.P = [None] + [prolongation(self.levels[l - 1], self.levels[l]) for l in range(1, len(Ns))]
        self.cheb_steps = cheb_steps
        self.prec = [PatchPreconditioner(L) if smoother == "patch" and l > 0 else None
                     for l, L in enumerate(self.levels)]
        self.lmax = [estimate_lambda_max(L.A, L.diag, eig_steps, prec=P) for L, P in zip(self.levels, self.prec)]
        self.cheb_lo, self.cheb_hi = cheb_lo, cheb_hi
        c = self.levels[0]
        self.coarse_interior = np.nonzero(~c.space.boundary)[0]
        Aii = c.A[self.coarse_interior][:, self.coarse_interior].toarray()
        self.coarse_chol = sla.cho_factor(Aii, lower=True)

    @property
    def fine(self):
        return self.levels[-1]

    def coarse_solve(self, b):
        """Direct solve with the Cholesky factor of the interior coarse matrix; x_bd = b_bd."""
        x = b.copy()
        x[self.coarse_interior] = sla.cho_solve(self.coarse_chol, b[self.coarse_interior])
        return x

    def smooth(self, l, b, x):
        L = self.levels[l]
        lm = self.lmax[l]
        return chebyshev(lambda v: matvec(L.A, v), L.diag, b, x, self.cheb_lo * lm, self.cheb_hi * lm, self.cheb_steps,
                         prec=self.prec[l])

    def vcycle(self, b, l=None):
        """One V-cycle: pre-smooth from 0, restrict the residual, recurse, prolong, post-smooth."""
        if l is None:
            l = len(self.levels) - 1
        if l == 0:
            return self.coarse_solve(b)
        L = self.levels[l]
        x = self.smooth(l, b, np.zeros_like(b))
        r = b - matvec(L.A, x)
        rc = self.P[l].T @ r
        rc[self.levels[l - 1].space.boundary] = 0.0
        x = x + self.P[l] @ self.vcycle(rc, l - 1)
        return self.smooth(l, b, x)

    def fmg(self, b, cycles=1):
        """Full multigrid as the whole solve (the paper's outer solver, Section 3: full
        multigrid with a direct coarse solve): the right-hand side restricted to every
        level (boundary entries zero), the coarsest level solved directly, then on each
        finer level the interpolated coarser solution corrected by ``cycles`` V-cycles
        (x += V(b_l - A_l x), i.e. a V-cycle started from x)."""
        nl = len(self.levels)
        bs = [None] * nl
        bs[-1] = np.asarray(b, dtype=np.float64)
        for l in range(nl - 1, 0, -1):
            rc = self.P[l].T @ bs[l]
            rc[self.levels[l - 1].space.boundary] = 0.0
            bs[l - 1] = rc
        x = self.coarse_solve(bs[0])
        for l in range(1, nl):
            x = self.P[l] @ x
            A = self.levels[l].A
            for _ in range(cycles):
                x = x + self.vcycle(bs[l] - matvec(A, x), l)
        return x


QUAD_N = 3  # Gauss points per direction of the quadrature load vector: 27 per tet, exact to degree 3


def quadrature_points(mesh, n=QUAD_N):
    """Physical points x = p0 + J xi of the conical-product rule on every cell: (C, n^3, 3)."""
    xi, _ = tet_quadrature(n)
    J = mesh.jacobians()
    p0 = mesh.coords[mesh.cells[:, 0]]
    return p0[:, None, :] + np.einsum("cab,qb->cqa", J, xi)


def load_vector_quadrature(level, f_qp, n=QUAD_N):
    """b_i = sum_K sum_q w_q |det J_K| f(x_Kq) phi_i(xi_q): the linear form of f v dx (Section 2)
    by quadrature with f given at the points of ``quadrature_points``; b = 0 on the boundary."""
    xi, w = tet_quadrature(n)
    phi, _ = ref_basis(level.space.degree, xi)
    det = np.abs(np.linalg.det(level.space.mesh.jacobians()))
    be = np.einsum("q,c,cq,qd->cd", w, det, np.asarray(f_qp, dtype=np.float64), phi)
    b = np.zeros(level.n)
    np.add.at(b, level.space.cell_dofs, be)
    b[level.space.boundary] = 0.0
    return b


def load_vector(level, f_nodal, bc_values=None):
    """b = M I_h f on interior rows, minus A_ib g_b; b_bd = g_bd (symmetric elimination)."""
    b = level.M @ f_nodal
    bd = level.space.boundary
    if bc_values is None:
        b[bd] = 0.0
        return b
    g = np.where(bd, bc_values, 0.0)
    b = b - level.A_free @ g
    b[bd] = bc_values[bd]
    return b


def solve(hier_or_level, b, rtol=1e-10, maxit=2000, precond="gmg", x0=None):
    """Solve A_bc u = b by PCG with a GMG V-cycle ("gmg") or Jacobi ("jacobi")."""
    if isinstance(hier_or_level, Hierarchy):
        L = hier_or_level.fine
        M = hier_or_level.vcycle if precond == "gmg" else (lambda v: v / L.diag)
    else:
        L = hier_or_level
        M = lambda v: v / L.diag
    x, it, hist, _ = pcg(lambda v: matvec(L.A, v), b, M, rtol, maxit, x0)
    return x, it, hist


def direct_solve(level, b):
    """Sparse direct solve of A_bc u = b (reference for small meshes)."""
    import scipy.sparse.linalg as spla
    return spla.spsolve(level.A.tocsc(), b)


# ------------------------------------------------------------- errors -----
def l2_error(space, u_h, u_exact, nq=None, chunk=1 << 15):
    """||u_h - u||_{L2} by the conical-product rule with nq points per direction (default max(6, k + 4): exact to
    degree 2 nq - 3 >= 2k + 4 for P_k, beyond the degree 2k of (u_h)^2)."""
    if nq is None:
        nq = max(6, space.degree + 4)
    xi, w = tet_quadrature(nq)
    phi, _ = ref_basis(space.degree, xi)
    mesh = space.mesh
    tot = 0.0
    for s in range(0, mesh.n_cells, chunk):
        sel = slice(s, min(mesh.n_cells, s + chunk))
        J = mesh.jacobians(sel)
        det = np.abs(np.linalg.det(J))
        p0 = mesh.coords[mesh.cells[sel, 0]]
        xq = p0[:, None, :] + np.einsum("cij,qj->cqi", J, xi)
        uq = np.einsum("qd,cd->cq", phi, u_h[space.cell_dofs[sel]])
        ue = u_exact(xq.reshape(-1, 3)).reshape(uq.shape)
        tot += np.sum(det[:, None] * w[None, :] * (uq - ue) ** 2)
    return np.sqrt(tot)


# ------------------------------------------------------------ adjoint -----
def objective(level, u, u_d):
    """J = (u - u_d)^T M (u - u_d) = int (u_h - I_h u_d)^2 dx with the exact mass matrix."""
    e = u - u_d
    return float(e @ (level.M @ e))


def adjoint_gradient(hier, b, u_d, rtol=1e-13, maxit=2000):
    """dJ/dkappa_K = int_K grad(lambda) . grad(u) with A lambda = -2 M (u - u_d), lambda_bd = 0.

    Returns (J, gradient per fine cell, u, lambda).
    """
    L = hier.fine
    u, _, _ = solve(hier, b, rtol, maxit)
    e = u - u_d
    J = float(e @ (L.M @ e))
    rhs = -2.0 * (L.M @ e)
    rhs[L.space.boundary] = 0.0
    lam, _, _ = solve(hier, rhs, rtol, maxit)
    unit = element_stiffness(L.mesh, L.space.degree, None)
    cd = L.space.cell_dofs
    g = np.einsum("cd,cde,ce->c", lam[cd], unit, u[cd])
    return J, g, u, lam
