"""Pins of the oracle's solvers: brute force, patch tests, convergence rates,
the Chebyshev polynomial identity, the coarse Cholesky solve and the adjoint.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fe_oracle as O
import fe_inputs as I


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("N", [2, 4])
def test_brute_force_dense_solve(k, N):
    h = O.Hierarchy(max(1, N // 2), 1, k)
    L = h.fine
    b = O.load_vector(L, I.sin_product_rhs(L.space.coords))
    dense = np.linalg.solve(L.A.toarray(), b)
    for pc in ("gmg", "jacobi"):
        u, it, hist = O.solve(h, b, rtol=1e-14, precond=pc)
        assert np.linalg.norm(u - dense) <= 1e-12 * np.linalg.norm(dense)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_patch_test_exact(k):
    """Linear (P1) / quadratic (P2) / cubic (P3) solutions with matching Dirichlet data are nodally exact."""
    h = O.Hierarchy(2, 1, k)
    L = h.fine
    X = L.space.coords
    if k == 1:
        u = 1 + 2 * X[:, 0] - 3 * X[:, 1] + 0.5 * X[:, 2]
        f = np.zeros(L.n)
    elif k == 3:
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        u = x ** 3 - 2 * y * y * z + x * y * z + 0.5 * z ** 3 - x * x + 1
        f = -(6 * x - 4 * z + 3 * z - 2)  # -Laplace(u), linear: its P3 interpolant is exact
    else:
        u = X[:, 0] ** 2 + 2 * X[:, 1] ** 2 - X[:, 2] ** 2 + X[:, 0] * X[:, 1] - X[:, 1] * X[:, 2] + 3 * X[:, 0]
        f = np.full(L.n, -4.0)  # -Laplace(u)
    b = O.load_vector(L, f, bc_values=u)
    uh, it, hist = O.solve(h, b, rtol=1e-14)
    assert np.abs(uh - u).max() < 1e-12


@pytest.mark.parametrize("k,Ns,order", [(1, (8, 16), 2.0), (2, (8, 16), 3.0), (3, (4, 8), 4.0)])
def test_convergence_rates(k, Ns, order):
    errs = []
    for N in Ns:
        h = O.Hierarchy(N // 4, 2, k)
        L = h.fine
        b = O.load_vector(L, I.sin_product_rhs(L.space.coords))
        u, it, hist = O.solve(h, b, rtol=1e-12)
        errs.append(O.l2_error(L.space, u, I.sin_product))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.15, (errs, rate)


def test_paper_manufactured_pair():
    """The paper's printed f is -Laplace of its printed u (Section 2, Eqs. 2-3)."""
    rng = np.random.default_rng(0)
    X = rng.uniform(0.05, 0.95, size=(20, 3))
    h = 1e-4
    lap = np.zeros(20)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        lap += (I.paper_solution(X + e) - 2 * I.paper_solution(X) + I.paper_solution(X - e)) / h ** 2
    assert np.allclose(-lap, I.paper_rhs(X), rtol=1e-5, atol=1e-5)


def test_paper_problem_p3_converges_at_h4():
    """The paper's Poisson problem as it states it (Section 2, Eqs. 2-3: its u and f, P3 as in its script): the
    discrete solution's L2 error falls at the P3 rate h^4 (N = 4 -> 8)."""
    errs = []
    for N in (4, 8):
        L = O.Level(N, 3)
        X = L.space.coords
        u = O.direct_solve(L, O.load_vector(L, I.paper_rhs(X)))
        errs.append(O.l2_error(L.space, u, I.paper_solution))
    assert 3.6 <= np.log2(errs[0] / errs[1]) <= 4.4, errs


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_chebyshev_polynomial_identity(steps):
    """x_k - x* = p_k(D^-1 A)(x_0 - x*), p_k(t) = T_k((theta-t)/delta) / T_k(theta/delta)."""
    L = O.Level(2, 2, I.grf_kappa(O.Mesh(2).centroids()))
    A = L.A.toarray()
    d = L.diag
    rng = np.random.default_rng(1)
    b, x0 = rng.normal(size=L.n), rng.normal(size=L.n)
    xs = np.linalg.solve(A, b)
    lo, hi = 0.3, 2.1
    xk = O.chebyshev(lambda v: A @ v, d, b, x0, lo, hi, steps)
    # D^-1 A = D^-1/2 S D^1/2 with S symmetric
    Dh = np.sqrt(d)
    S = A / np.outer(Dh, Dh)
    lam, V = np.linalg.eigh(S)
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    Tk = np.polynomial.chebyshev.Chebyshev.basis(steps)
    pk = Tk((theta - lam) / delta) / Tk(theta / delta)
    e0 = Dh * (x0 - xs)
    ek = (V @ (pk * (V.T @ e0))) / Dh
    assert np.allclose(xk - xs, ek, atol=1e-11)


def test_coarse_cholesky_solve():
    h = O.Hierarchy(3, 1, 2)
    c = h.levels[0]
    b = np.random.default_rng(2).normal(size=c.n)
    x = h.coarse_solve(b)
    assert np.linalg.norm(c.A @ x - b) < 1e-12 * np.linalg.norm(b)


def test_gmg_pcg_is_mesh_independent():
    its = []
    for nref in (1, 2, 3):
        h = O.Hierarchy(2, nref, 2)
        L = h.fine
        b = O.load_vector(L, I.sin_product_rhs(L.space.coords))
        _, it, _ = O.solve(h, b, rtol=1e-8)
        its.append(it)
    assert max(its) <= 12 and its[-1] - its[0] <= 3, its


@pytest.mark.parametrize("k,smoother", [(1, "jacobi"), (2, "jacobi"), (2, "patch"), (3, "jacobi"), (3, "patch")])
def test_vcycle_is_a_symmetric_positive_definite_contraction(k, smoother):
    """The V-cycle as a map b -> x is linear, symmetric and positive definite on the interior dofs (the same
    Chebyshev polynomial before and after the coarse correction, a symmetric smoother preconditioner, restriction =
    prolongation transposed), which CG needs of its preconditioner; its error propagation I - V A contracts in the
    energy norm.  A dropped post-smoothing, a restriction that is not P^T or a wrong coarse correction breaks one
    of these."""
    kap = I.grf_kappa(O.Mesh(4).centroids(), seed=3)
    h = O.Hierarchy(2, 1, k, kap, smoother=smoother)
    L = h.fine
    bd = L.space.boundary
    rng = np.random.default_rng(11)
    u, w = rng.normal(size=L.n), rng.normal(size=L.n)
    u[bd] = w[bd] = 0.0
    Vu, Vw = h.vcycle(u), h.vcycle(w)
    assert np.abs(h.vcycle(2 * u - w) - (2 * Vu - Vw)).max() <= 1e-12 * np.abs(Vu).max()
    assert abs(w @ Vu - u @ Vw) <= 1e-12 * np.linalg.norm(w) * np.linalg.norm(Vu)
    assert u @ Vu > 0 and w @ Vw > 0
    # energy-norm contraction factor of I - V A by power iteration on the interior
    e = rng.normal(size=L.n)
    e[bd] = 0.0
    rho = 0.0
    for _ in range(12):
        en = e - h.vcycle(L.A @ e)
        rho = np.sqrt((en @ (L.A @ en)) / (e @ (L.A @ e)))
        e = en / np.sqrt(en @ (L.A @ en))
    assert rho < 0.5, rho  # measured 0.28-0.44 (P3 with Jacobi the weakest)


def _J_direct(N, k, kappa, f_fn, ud_fn):
    L = O.Level(N, k, kappa)
    b = O.load_vector(L, f_fn(L.space.coords))
    u = spla.spsolve(L.A.tocsc(), b)
    return O.objective(L, u, ud_fn(L.space.coords))


@pytest.mark.parametrize("k", [1, 2])
def test_adjoint_gradient_vs_central_differences(k):
    N = 2
    mesh = O.Mesh(N)
    kappa = I.grf_kappa(mesh.centroids(), seed=7)
    f_fn = lambda X: np.ones(X.shape[0])
    h = O.Hierarchy(1, 1, k, kappa)
    L = h.fine
    b = O.load_vector(L, f_fn(L.space.coords))
    ud = I.target_field(L.space.coords)
    J, g, u, lam = O.adjoint_gradient(h, b, ud)
    assert abs(J - _J_direct(N, k, kappa, f_fn, I.target_field)) < 1e-12 * abs(J)
    cells = np.random.default_rng(0).choice(mesh.n_cells, 12, replace=False)
    for c in cells:
        eps = 1e-5 * kappa[c]
        kp, km = kappa.copy(), kappa.copy()
        kp[c] += eps
        km[c] -= eps
        fd = (_J_direct(N, k, kp, f_fn, I.target_field) - _J_direct(N, k, km, f_fn, I.target_field)) / (2 * eps)
        assert abs(fd - g[c]) <= 1e-6 * np.abs(g).max(), (c, fd, g[c])


def test_adjoint_taylor_remainder_is_second_order():
    N = 4
    mesh = O.Mesh(N)
    kappa = I.grf_kappa(mesh.centroids(), seed=9)
    f_fn = lambda X: np.ones(X.shape[0])
    h = O.Hierarchy(2, 1, 1, kappa)
    L = h.fine
    J, g, u, lam = O.adjoint_gradient(h, O.load_vector(L, f_fn(L.space.coords)), I.target_field(L.space.coords))
    dk = np.random.default_rng(3).normal(size=mesh.n_cells) * kappa
    rem = []
    for t in (1e-2, 5e-3):
        rem.append(abs(_J_direct(N, 1, kappa + t * dk, f_fn, I.target_field) - J - t * (g @ dk)))
    assert 3.0 < rem[0] / rem[1] < 5.0  # O(t^2): halving t divides the remainder by ~4


# ------------------------------------------------------------ full multigrid
def test_fmg_single_level_is_the_direct_solve():
    """With one level FMG is the coarse Cholesky solve: the exact discrete solution."""
    H = O.Hierarchy(3, 0, 2)
    L = H.fine
    b = O.load_vector(L, I.sin_product_rhs(L.space.coords))
    assert np.allclose(H.fmg(b), O.direct_solve(L, b), rtol=0, atol=1e-13)


def test_fmg_cycles_converge_to_discrete_solution():
    """Many V-cycles per level make FMG a converged multigrid iteration: the discrete solution."""
    H = O.Hierarchy(2, 2, 2)
    L = H.fine
    b = O.load_vector(L, I.sin_product_rhs(L.space.coords))
    uh = O.direct_solve(L, b)
    assert np.linalg.norm(H.fmg(b, cycles=25) - uh) <= 1e-11 * np.linalg.norm(uh)


def test_fmg_reaches_discretisation_accuracy():
    """One FMG cycle already solves to the order of the discretisation error (the property
    that makes a single F-cycle a complete solve): its L2 error against the exact solution is
    within 2x that of the exact discrete solution (within 10% with two V-cycles per level)
    and converges at the discretisation's O(h^3) rate for P2."""
    errs = []
    for N0 in (2, 4):
        H = O.Hierarchy(N0, 2, 2)
        L = H.fine
        X = L.space.coords
        b = O.load_vector(L, I.sin_product_rhs(X))
        eh = O.l2_error(L.space, O.direct_solve(L, b), I.sin_product)
        e1 = O.l2_error(L.space, H.fmg(b), I.sin_product)
        e2 = O.l2_error(L.space, H.fmg(b, cycles=2), I.sin_product)
        assert eh < e1 <= 2.0 * eh and e2 <= 1.1 * eh, (e1, e2, eh)
        errs.append(e1)
    assert 2.6 <= np.log2(errs[0] / errs[1]) <= 3.4, errs
