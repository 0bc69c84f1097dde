"""Parity of the extension forms: mixed-precision refinement and the adjoint gradient.

Mixed precision (FP32 inner GMG-PCG inside FP64 iterative refinement) must
reach the same 1e-8 FP64 residual and agree with the FP64 oracle solution to
1e-6 relative L2.  The adjoint gradient dJ/dkappa must match the oracle's
assembled adjoint to 1e-8 relative and central finite differences to 1e-6 of
max |dJ/dkappa|; at the full adjoint size (P1 96^3) it must pass the Taylor
test (second-order remainder).
"""
import numpy as np
import pytest

import fe_inputs as I
from oracle import fe_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def fe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08012_gb300 import build
    build.build()
    import paper_2104_08012_gb300 as fe
    fe.load()
    return fe


def dt(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


# ------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("k,N0,nref", [(2, 4, 2), (1, 4, 3)])
@pytest.mark.parametrize("coef", ["one", "grf"])
def test_mixed_precision_refinement(fe, k, N0, nref, coef):
    with fe.Hierarchy(N0, nref, k) as h:
        kappa = None if coef == "one" else I.grf_kappa(h.cell_centroids(), seed=12)
        h.set_coefficient(None if kappa is None else dt(kappa))
        L = O.Level(N0 * 2 ** nref, k, kappa)
        f = I.sin_product_rhs(L.space.coords)
        b = O.load_vector(L, f)
        ue = O.direct_solve(L, b)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        st = h.solve(dt(f), u, rtol=1e-8, precision=fe.FE_PREC_MIXED_F32)
        uh = host(u)
        # the FP64 residual is recomputed by the oracle, not taken from the library
        assert np.linalg.norm(L.A @ uh - b) <= 1.0001e-8 * np.linalg.norm(b)
        assert st.rel_residual <= 1e-8 and st.outer_iterations >= 2
        rel = np.linalg.norm(uh - ue) / np.linalg.norm(ue)
        assert rel <= 1e-6, rel
        u64 = torch.empty_like(u)
        st64 = h.solve(dt(f), u64, rtol=1e-8)
        assert np.linalg.norm(uh - host(u64)) <= 1e-6 * np.linalg.norm(ue)
        # far fewer FP64 operator applications than the FP64 solve
        assert st.fine_applies_f64 < st64.fine_applies_f64


def test_mixed_precision_reaches_tight_tolerance(fe):
    """Refinement converges past FP32 accuracy: rtol 1e-12 in FP64."""
    with fe.Hierarchy(4, 2, 2) as h:
        L = O.Level(16, 2)
        f = I.sin_product_rhs(L.space.coords)
        b = O.load_vector(L, f)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.solve(dt(f), u, rtol=1e-12, precision=fe.FE_PREC_MIXED_F32)
        assert np.linalg.norm(L.A @ host(u) - b) <= 1.001e-12 * np.linalg.norm(b)


# ------------------------------------------------------------------- adjoint
def _setup_adjoint(fe, N0, nref, k, seed=21):
    h = fe.Hierarchy(N0, nref, k)
    big = h.n_cells() > 100000
    kappa = I.grf_kappa(h.cell_centroids(), seed=seed, device=DEV if big else None)
    X = h.dof_coordinates()
    f = np.ones(h.n_dofs())
    ud = I.target_field(X)
    return h, kappa, f, ud


@pytest.mark.parametrize("k", [1, 2])
def test_adjoint_matches_oracle_assembled_adjoint(fe, k):
    h, kappa, f, ud = _setup_adjoint(fe, 2, 2, k)
    with h:
        h.set_coefficient(dt(kappa))
        g = torch.empty(h.n_cells(), dtype=torch.float64, device=DEV)
        J = h.adjoint_gradient(dt(f), dt(ud), g, rtol=1e-13)
        oh = O.Hierarchy(2, 2, k, kappa)
        L = oh.fine
        Jo, go, _, _ = O.adjoint_gradient(oh, O.load_vector(L, f), ud)
        assert abs(J - Jo) <= 1e-10 * abs(Jo)
        assert np.linalg.norm(host(g) - go) <= 1e-8 * np.linalg.norm(go)


def test_adjoint_vs_central_differences_8cubed(fe):
    """P1 on 8^3: the adjoint gradient against central finite differences of J on every one of the 3072 cells.

    Step eps_K = 1e-4 kappa_K: the truncation error of the central difference is about (eps/kappa)^2 / 6 = 2e-9
    relative, and J's rounding (both solves in native FP64 to rtol 1e-14) divided by eps stays below the floor.
    Per cell: |FD - g_K| <= 1e-6 |g_K| + 1e-7 max|g|, i.e. 1e-6 relative wherever |g_K| >= 10% of max|g|, and an
    absolute 1e-7 max|g| for the cells whose gradient is smaller than that."""
    h, kappa, f, ud = _setup_adjoint(fe, 2, 2, 1)
    with h:
        h.set_f64_mode(fe.FE_F64_NATIVE)
        fd_f, fd_ud = dt(f), dt(ud)
        h.set_coefficient(dt(kappa))
        g = torch.empty(h.n_cells(), dtype=torch.float64, device=DEV)
        h.adjoint_gradient(fd_f, fd_ud, g, rtol=1e-14, max_it=400)
        g = host(g)
        u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        kap = dt(kappa)

        def J(c, e):
            kap[c] = kappa[c] + e
            h.set_coefficient(kap)
            kap[c] = kappa[c]
            h.solve(fd_f, u, rtol=1e-14, max_it=400)
            return h.objective(u, fd_ud)

        fd = np.empty(h.n_cells())
        for c in range(h.n_cells()):
            eps = 1e-4 * kappa[c]
            fd[c] = (J(c, eps) - J(c, -eps)) / (2 * eps)
        tol = 1e-6 * np.abs(g) + 1e-7 * np.abs(g).max()
        bad = np.nonzero(np.abs(fd - g) > tol)[0]
        assert bad.size == 0, (bad.size, bad[:5], fd[bad[:5]], g[bad[:5]])
        big = np.abs(g) >= 0.1 * np.abs(g).max()
        assert np.all(np.abs(fd - g)[big] <= 2e-6 * np.abs(g)[big])


def test_autograd_function(fe):
    from paper_2104_08012_gb300.autograd import poisson_objective
    h, kappa, f, ud = _setup_adjoint(fe, 2, 1, 2)
    with h:
        kap = dt(kappa).requires_grad_(True)
        J = poisson_objective(kap, h, dt(f), dt(ud))
        J.backward()
        g = torch.empty(h.n_cells(), dtype=torch.float64, device=DEV)
        h.set_coefficient(dt(kappa))
        J2 = h.adjoint_gradient(dt(f), dt(ud), g, rtol=1e-12)
        assert abs(J.item() - J2) <= 1e-10 * abs(J2)
        assert torch.allclose(kap.grad, g, rtol=1e-8, atol=1e-12 * g.abs().max().item())


def test_adjoint_full_size_taylor(fe):
    """P1 UnitCubeMesh 96^3 (5,308,416 cells), 4 levels from 12^3: Taylor remainder is O(t^2)."""
    h, kappa, f, ud = _setup_adjoint(fe, 12, 3, 1)
    with h:
        assert h.n_cells() == 5308416
        fd_f, fd_ud = dt(f), dt(ud)
        h.set_coefficient(dt(kappa))
        g = torch.empty(h.n_cells(), dtype=torch.float64, device=DEV)
        J0 = h.adjoint_gradient(fd_f, fd_ud, g, rtol=1e-12)
        g = host(g)
        dk = np.random.default_rng(5).normal(size=h.n_cells()) * kappa
        u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        rem = []
        for t in (1e-2, 5e-3):
            h.set_coefficient(dt(kappa + t * dk))
            h.solve(fd_f, u, rtol=1e-12)
            rem.append(abs(h.objective(u, fd_ud) - J0 - t * (g @ dk)))
        assert 3.0 < rem[0] / rem[1] < 5.0, rem


# ------------------------------------------------------- bf16 tensor cores
@pytest.mark.parametrize("k,N", [(1, 3), (1, 8), (1, 16), (2, 3), (2, 8), (2, 16), (3, 3), (3, 6)])
@pytest.mark.parametrize("form", ["uniform", "per_cell"])
def test_apply_bf16_tensor_core(fe, k, N, form):
    """tcgen05 GEMM-form apply: each dof split into two bf16 terms, tables exact (two bf16 terms where needed,
    P3), FP32 accumulation; the one-table form (G = c M, N = 16 / 16 / 32 columns) and the six-table form
    (N = 32 / 64 / 128 columns).

    Rowwise bound 5e-5 |A||x| (the two-term bf16 split keeps 16 bits, 2^-17
    relative, plus FP32 sums); N=3 gives 162 cells, i.e. one partial 128-cell tile.
    """
    with fe.Hierarchy(N, 0, k) as h:
        if form == "per_cell":
            h.set_geometry_form(fe.FE_GEOMETRY_PER_CELL)
        kappa = I.grf_kappa(h.cell_centroids(), seed=N + 40)
        h.set_coefficient(dt(kappa))
        L = O.Level(N, k, kappa)
        x = I.random_vector(L.n, 50 + N).astype(np.float32)
        y = torch.empty(L.n, dtype=torch.float32, device=DEV)
        h.apply_operator(dt(x, torch.float32), y, dtype=fe.FE_BF16)
        y32 = torch.empty(L.n, dtype=torch.float32, device=DEV)
        h.apply_operator(dt(x, torch.float32), y32, dtype=fe.FE_F32)
        torch.cuda.synchronize()
        xd = x.astype(np.float64)
        scale = abs(L.A) @ np.abs(xd)
        got = host(y)
        err = np.abs(got - L.A @ xd)
        assert np.all(err <= 5e-5 * scale), np.max(err / scale)
        # interior rows are exactly the GEMM of the two-term bf16 split of the dofs
        # (up to FP32 accumulation); Dirichlet rows copy the FP32 x (identity rows)
        xt = torch.from_numpy(x)
        hi = xt.to(torch.bfloat16).to(torch.float32)
        lo = (xt - hi).to(torch.bfloat16).to(torch.float32)
        xb = hi.double().numpy() + lo.double().numpy()
        inter = ~L.space.boundary
        err_b = np.abs(got - L.A @ xb)[inter]
        sb = (abs(L.A) @ np.abs(xb))[inter]
        assert np.all(err_b <= 2e-5 * sb), np.max(err_b / sb)
        assert np.array_equal(got[~inter], x[~inter].astype(np.float64))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_geometry_forms_agree(fe, k):
    """Every operator path with one geometric value per cell (G = c M) against the six stored factors: FP64 in
    float pairs (per tet and, for P1, per cube), native FP64 and FP32, rowwise at their parity tolerances, and a
    GMG-PCG solve."""
    with fe.Hierarchy(4, 1, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=k)
        h.set_coefficient(dt(kappa))
        L = O.Level(8, k, kappa)
        x = I.random_vector(L.n, 7)
        scale = abs(L.A) @ np.abs(x)
        out = {}
        for form in (fe.FE_GEOMETRY_AUTO, fe.FE_GEOMETRY_PER_CELL):
            h.set_geometry_form(form)
            for mode in (fe.FE_F64_DOUBLE_FLOAT, fe.FE_F64_DOUBLE_FLOAT_TET, fe.FE_F64_NATIVE):
                h.set_f64_mode(mode)
                y = torch.empty(L.n, dtype=torch.float64, device=DEV)
                h.apply_operator(dt(x), y)
                out[form, mode] = host(y)
            h.set_f64_mode(fe.FE_F64_DOUBLE_FLOAT)
            y32 = torch.empty(L.n, dtype=torch.float32, device=DEV)
            h.apply_operator(dt(x, torch.float32), y32, dtype=fe.FE_F32)
            out[form, "f32"] = host(y32)
            u = torch.empty(L.n, dtype=torch.float64, device=DEV)
            st = h.solve(dt(I.sin_product_rhs(h.dof_coordinates())), u, rtol=1e-12)
            out[form, "solve"] = (host(u), st.iterations)
        ref = L.A @ x
        for mode in (fe.FE_F64_DOUBLE_FLOAT, fe.FE_F64_DOUBLE_FLOAT_TET, fe.FE_F64_NATIVE):
            for form in (fe.FE_GEOMETRY_AUTO, fe.FE_GEOMETRY_PER_CELL):
                assert np.all(np.abs(out[form, mode] - ref) <= 1e-13 * scale), (form, mode)
        for form in (fe.FE_GEOMETRY_AUTO, fe.FE_GEOMETRY_PER_CELL):
            assert np.all(np.abs(out[form, "f32"] - ref) <= 1e-5 * scale), form
        ua, ia = out[fe.FE_GEOMETRY_AUTO, "solve"]
        ub, ib = out[fe.FE_GEOMETRY_PER_CELL, "solve"]
        assert ia == ib and np.linalg.norm(ua - ub) <= 1e-11 * np.linalg.norm(ub)


def test_mixed_bf16_refinement(fe):
    with fe.Hierarchy(4, 2, 2) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=13)
        h.set_coefficient(dt(kappa))
        L = O.Level(16, 2, kappa)
        f = I.sin_product_rhs(L.space.coords)
        b = O.load_vector(L, f)
        ue = O.direct_solve(L, b)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        st = h.solve(dt(f), u, rtol=1e-8, precision=fe.FE_PREC_MIXED_BF16)
        uh = host(u)
        assert np.linalg.norm(L.A @ uh - b) <= 1.0001e-8 * np.linalg.norm(b)
        assert np.linalg.norm(uh - ue) <= 1e-6 * np.linalg.norm(ue)
        assert st.outer_iterations >= 2


# --------------------------------------------- the paper's manufactured problem
def test_paper_manufactured_problem_converges():
    """The paper's own problem (Section 2, Eqs. 2-3: u = sin(pi x) tan(pi x/4) sin(pi y) sin(2 pi z),
    f as printed) solved by GPU GMG-PCG on P2 hierarchies: the L2 error (oracle's conical-product
    rule) converges at the P2 rate O(h^3) and FMG with two V-cycles per level stays within 2x of it."""
    import paper_2104_08012_gb300 as fe
    from paper_2104_08012_gb300 import build
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    errs = []
    for N0 in (2, 4, 8):
        with fe.Hierarchy(N0, 2, 2) as h:
            X = h.dof_coordinates()
            f = torch.from_numpy(I.paper_rhs(X)).to(DEV)
            u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
            h.solve(f, u, rtol=1e-11)
            space = O.Space(O.Mesh(4 * N0), 2)
            e = O.l2_error(space, host(u), I.paper_solution)
            h.solve(f, u, precond=fe.FE_PC_FMG, max_it=2)
            e_fmg = O.l2_error(space, host(u), I.paper_solution)
            assert e_fmg <= 2.0 * e, (N0, e_fmg, e)
            errs.append(e)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 2.6) & (rates < 3.4)), (errs, rates)
