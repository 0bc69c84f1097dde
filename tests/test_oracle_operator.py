"""Pins of the oracle's stiffness/mass matrices, Dirichlet elimination and transfers.

Closed forms used: the assembled P1 Kuhn stiffness equals h times the 7-point
finite-difference Laplacian, hence D^-1 A has the known cosine spectrum;
element matrices are symmetric with zero row sums and permute with their
vertices; P reproduces polynomials of the element degree; P^T A_f P = A_c.
"""
import itertools

import numpy as np
import pytest

from oracle import fe_oracle as O
import fe_inputs as I


def _perm_local_dofs(k, pi):
    """Local dof permutation induced by relabelling tet vertices by pi."""
    if k == 1:
        return list(pi)
    out = list(pi)
    if k == 2:
        for a, b in O.P2_EDGES:
            pa, pb = sorted((pi[a], pi[b]))
            out.append(4 + O.P2_EDGES.index((pa, pb)))
        return out
    for a, b in O.P2_EDGES:
        for near in (a, b):  # P3: the node nearer `near` on edge (a, b)
            pa, pb = sorted((pi[a], pi[b]))
            out.append(4 + 2 * O.P2_EDGES.index((pa, pb)) + (0 if pi[near] == pa else 1))
    out += [16 + pi[f] for f in range(4)]  # face f is the face opposite vertex f
    return out


@pytest.mark.parametrize("k", [1, 2, 3])
def test_element_stiffness_invariants(k):
    m = O.Mesh(2)
    kap = I.grf_kappa(m.centroids(), seed=3)
    A = O.element_stiffness(m, k, kap)
    assert np.allclose(A, A.transpose(0, 2, 1), atol=1e-15)
    assert np.abs(A.sum(axis=2)).max() < 1e-13
    ev = np.linalg.eigvalsh(A)
    assert ev[:, 0].min() > -1e-13 and (ev[:, 1] > 1e-6).all()  # kernel = constants only
    # relabelling the vertices of a tet permutes its element matrix
    for pi in itertools.permutations(range(4)):
        if pi == (0, 1, 2, 3):
            continue
        m2 = O.Mesh(2)
        inv = np.argsort(pi)
        m2.cells = m.cells[:, inv]
        A2 = O.element_stiffness(m2, k, kap)
        perm = _perm_local_dofs(k, inv)
        assert np.allclose(A2, A[:, perm][:, :, perm], atol=1e-14)


@pytest.mark.parametrize("N", [3, 4])
def test_p1_stiffness_is_h_times_7_point_laplacian(N):
    L = O.Level(N, 1)
    A = L.A_free.toarray()
    h = 1.0 / N
    lat = L.space.dof_lattice
    interior = np.nonzero(~L.space.boundary)[0]
    for i in interior:
        row = A[i]
        assert abs(row[i] - 6 * h) < 1e-14
        for j in np.nonzero(np.abs(row) > 1e-14)[0]:
            if j == i:
                continue
            d = np.abs(lat[j] - lat[i])
            assert d.sum() == 1 and abs(row[j] + h) < 1e-14


def test_p1_jacobi_spectrum_closed_form():
    N = 6
    L = O.Level(N, 1)
    inter = ~L.space.boundary
    A = L.A.toarray()[np.ix_(inter, inter)]
    d = np.diag(A)
    ev = np.sort(np.linalg.eigvalsh(A / np.sqrt(np.outer(d, d))))
    h = 1.0 / N
    j = np.arange(1, N)
    expect = np.sort([1 - (np.cos(a * np.pi * h) + np.cos(b * np.pi * h) + np.cos(c * np.pi * h)) / 3
                      for a in j for b in j for c in j])
    assert np.allclose(ev, expect, atol=1e-13)
    # and the Lanczos estimate used for the Chebyshev interval reaches 1 + cos(pi h)
    assert abs(O.estimate_lambda_max(L.A, L.diag, 30) - (1 + np.cos(np.pi * h))) < 1e-8


@pytest.mark.parametrize("k", [1, 2, 3])
def test_global_matrix_invariants(k):
    L = O.Level(3, k, I.grf_kappa(O.Mesh(3).centroids()))
    A = L.A_free
    assert abs(A - A.T).max() < 1e-14
    assert np.abs(A @ np.ones(L.n)).max() < 1e-12
    Abc = L.A.toarray()
    assert np.linalg.eigvalsh(Abc).min() > 0
    bd = L.space.boundary
    assert np.allclose(Abc[bd][:, bd], np.eye(bd.sum()))
    assert np.abs(Abc[bd][:, ~bd]).max() == 0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_mass_matrix(k):
    L = O.Level(3, k)
    M = L.M
    one = np.ones(L.n)
    assert abs(one @ (M @ one) - 1.0) < 1e-13  # |Omega| = 1
    x = L.space.coords
    # int x dx = 1/2, int x*y dx = 1/4 (x, y in the P1 and P2 spaces)
    assert abs(one @ (M @ x[:, 0]) - 0.5) < 1e-13
    assert abs(x[:, 0] @ (M @ x[:, 1]) - 0.25) < 1e-13
    assert abs(M - M.T).max() < 1e-16


@pytest.mark.parametrize("k", [1, 2, 3])
def test_apply_rows_matches_assembled(k):
    L = O.Level(4, k, I.grf_kappa(O.Mesh(4).centroids()))
    x = I.random_vector(L.n, 5)
    rows = np.random.default_rng(1).choice(L.n, 40, replace=False)
    assert np.allclose(O.apply_rows(L.space, L.kappa, x, rows), (L.A @ x)[rows], atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_apply_rows_mass_matches_assembled(k):
    L = O.Level(4, k)
    x = I.random_vector(L.n, 6)
    rows = np.random.default_rng(2).choice(L.n, 40, replace=False)
    assert np.allclose(O.apply_rows_mass(L.space, x, rows), (L.M @ x)[rows], atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_prolongation_reproduces_polynomials(k):
    c, f = O.Level(2, k), O.Level(4, k)
    P = O.prolongation(c, f)
    assert np.allclose(P @ np.ones(c.n), 1.0, atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(3):
        a = rng.normal(size=20)

        def p(X):
            x, y, z = X[:, 0], X[:, 1], X[:, 2]
            val = a[0] + a[1] * x + a[2] * y + a[3] * z
            if k >= 2:
                val = val + a[4] * x * x + a[5] * y * y + a[6] * z * z + a[7] * x * y + a[8] * x * z + a[9] * y * z
            if k >= 3:
                val = val + (a[10] * x ** 3 + a[11] * y ** 3 + a[12] * z ** 3 + a[13] * x * x * y + a[14] * x * x * z
                             + a[15] * y * y * x + a[16] * y * y * z + a[17] * z * z * x + a[18] * z * z * y
                             + a[19] * x * y * z)
            return val

        assert np.allclose(P @ p(c.space.coords), p(f.space.coords), atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_galerkin_identity(k):
    c, f = O.Level(2, k), O.Level(4, k)
    P = O.prolongation(c, f)
    G = (P.T @ f.A_free @ P).toarray()
    assert np.abs(G - c.A_free.toarray()).max() < 1e-13
    # with the boundary eliminated, on the interior block
    ic, fi = ~c.space.boundary, ~f.space.boundary
    Pi = P[fi][:, ic]
    Gi = (Pi.T @ f.A[fi][:, fi] @ Pi).toarray()
    assert np.abs(Gi - c.A.toarray()[np.ix_(ic, ic)]).max() < 1e-13


def _integer_parents(Nc):
    """Parent coarse cell of every cell of the 2 Nc mesh from integer lattice coordinates alone: with the fine
    tet's vertex lattice coordinates v_0..v_3 (fine lattice), its centroid is s / 8 in coarse cube units, s = sum
    v_i; the coarse cube is q = s // 8 per axis and, with l = s - 8 q, the coarse Kuhn tet is the permutation
    (p0, p1, p2) with l[p0] > l[p1] > l[p2] (a fine centroid is strictly inside one coarse tet)."""
    fine = O.Mesh(2 * Nc)
    s = fine.cell_vertex_lattice.sum(axis=1)
    q = s // 8
    loc = s - 8 * q
    order = tuple(map(tuple, np.argsort(-loc, axis=1, kind="stable")))
    assert np.all(np.diff(-np.sort(-loc, axis=1), axis=1) < 0)  # strict: no centroid on a coarse face
    t = np.array([O.KUHN_PERMS.index(o) for o in order])
    return 6 * (q[:, 0] + Nc * (q[:, 1] + Nc * q[:, 2])) + t


@pytest.mark.parametrize("Nc", [1, 2, 3])
def test_coarsen_kappa(Nc):
    """Pinned without the oracle's point location: parents from integer lattice arithmetic; 8 children per coarse
    cell; a kappa constant on each coarse cell comes back exactly; a random kappa gives the mean of the 8 children
    of each coarse cell."""
    c, f = O.Mesh(Nc), O.Mesh(2 * Nc)
    parent = _integer_parents(Nc)
    assert np.all(np.bincount(parent, minlength=c.n_cells) == 8)
    K = 1.0 + np.arange(c.n_cells) * 0.25
    assert np.array_equal(O.coarsen_kappa(c, f, K[parent]), K)
    kf = np.random.default_rng(Nc).lognormal(size=f.n_cells)
    want = np.array([kf[parent == p].sum() / 8 for p in range(c.n_cells)])
    assert np.allclose(O.coarsen_kappa(c, f, kf), want, rtol=1e-15, atol=0)


# ---------------------------------------------------- quadrature load vector
@pytest.mark.parametrize("k", [1, 2, 3])
def test_quadrature_load_vector_exact_cases(k):
    """The 27-point rule is exact to degree 3: for f = 1 (P_k x f of degree <= 3) and, for P1/P2, f linear the
    quadrature load vector equals M I_h f on the interior rows (I_h f = f).  For P3 x linear (degree 4) the
    64-point rule of the same family (exact to degree 5) does.  The points lie inside their cells (barycentric
    coordinates in [0, 1])."""
    L = O.Level(3, k)
    P = O.quadrature_points(L.space.mesh)
    assert P.shape == (L.space.mesh.n_cells, 27, 3)
    inside = L.space.mesh.coords[L.space.mesh.cells].min(axis=1)[:, None, :] <= P + 1e-15
    assert inside.all()
    X = L.space.coords
    lin_n = O.QUAD_N if k <= 2 else 4
    for f, fx, n in ((lambda p: np.ones(p.shape[:-1]), np.ones(len(X)), O.QUAD_N),
                     (lambda p: 0.3 + 2 * p[..., 0] - p[..., 1] + 0.5 * p[..., 2],
                      0.3 + 2 * X[:, 0] - X[:, 1] + 0.5 * X[:, 2], lin_n)):
        b = O.load_vector_quadrature(L, f(O.quadrature_points(L.space.mesh, n)), n)
        assert np.allclose(b, O.load_vector(L, fx), rtol=0, atol=1e-15)
    if k == 3:
        # the 27-point rule is not exact for P3 x linear: the pin above really needs the finer rule
        b27 = O.load_vector_quadrature(L, 0.3 + 2 * P[..., 0] - P[..., 1] + 0.5 * P[..., 2])
        assert np.abs(b27 - O.load_vector(L, 0.3 + 2 * X[:, 0] - X[:, 1] + 0.5 * X[:, 2])).max() > 1e-10


@pytest.mark.parametrize("k", [2, 3])
def test_quadrature_load_vector_converges(k):
    """Solving with the quadrature load vector of the sin-product f converges at the P_k rate h^(k+1) in L2."""
    errs = []
    for N in (4, 8):
        L = O.Level(N, k)
        b = O.load_vector_quadrature(L, I.sin_product_rhs(O.quadrature_points(L.space.mesh).reshape(-1, 3)).reshape(-1, 27))
        errs.append(O.l2_error(L.space, O.direct_solve(L, b), I.sin_product))
    assert k + 0.6 <= np.log2(errs[0] / errs[1]) <= k + 1.4, errs


def test_p3_energies_of_polynomials():
    """P3 stiffness and mass reproduce exact integrals of polynomials in the space (unit cube, kappa = 1):
    |grad x^3|^2 -> 9/5, |grad (x^2 y)|^2 -> 4/9 + 1/5, (x^3)^2 -> 1/7, x^3 * 1 -> 1/4, (xyz)^2 -> 1/27."""
    L = O.Level(2, 3)
    X = L.space.coords
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    A, M = L.A_free, L.M
    u = x ** 3
    assert abs(u @ (A @ u) - 9 / 5) < 1e-12
    v = x * x * y  # grad = (2xy, x^2, 0): int 4 x^2 y^2 + x^4 = 4/9 + 1/5
    assert abs(v @ (A @ v) - (4 / 9 + 1 / 5)) < 1e-12
    assert abs(u @ (M @ u) - 1 / 7) < 1e-13
    assert abs(np.ones(L.n) @ (M @ u) - 1 / 4) < 1e-13
    w = x * y * z
    assert abs(w @ (M @ w) - 1 / 27) < 1e-13


@pytest.mark.parametrize("threads", [1, 3])
def test_oracle_threaded_csr_product(threads):
    """The solves' CSR product (rows split over threads) against a dense product of the same matrix, on a matrix
    with empty rows, a ragged row-length mix and more rows than threads; it must also equal scipy's product."""
    import scipy.sparse as sp
    rng = np.random.default_rng(7)
    n = 1001
    A = sp.random(n, 733, density=0.01, format="csr", random_state=rng)
    A = A.multiply(np.where(np.arange(n) % 17 == 0, 0.0, 1.0)[:, None]).tocsr()  # empty rows
    x = rng.uniform(-1, 1, 733)
    y = O.matvec(A, x, threads=threads)
    dense = A.toarray() @ x
    assert np.allclose(y, dense, rtol=0, atol=1e-14 * np.abs(A).toarray().sum(axis=1).max())
    assert np.array_equal(y[::17], np.zeros_like(y[::17]))
    assert np.allclose(y, A @ x, rtol=1e-15, atol=1e-15)
    xt = rng.uniform(-1, 1, n)  # a transposed (CSC) operand takes scipy's product
    assert np.allclose(O.matvec(A.T, xt), A.toarray().T @ xt, rtol=0, atol=1e-13)
