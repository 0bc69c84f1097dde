"""P3 elements (the paper's degree) on the GPU against the FP64 CPU oracle.

Same bars as the P1/P2 parity tests: FP64 applications rowwise within 1e-13 of
|A||x|, FP32 within 1e-5, transfers within 1e-14, FP64 solutions within a
relative L2 error of 1e-10 (both sides to rtol 1e-13), the mixed-precision
solution within 1e-6 of the direct solve.
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


def assert_rowwise(got, ref, scale, tol, what):
    err = np.abs(got - ref)
    bound = tol * np.maximum(scale, 1e-300)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"{what}: {bad.size} rows off, worst {np.max(err / bound):.3g}x tol at {bad[:5]}"


@pytest.mark.parametrize("N", [1, 2, 3])
def test_p3_mesh_queries(fe, N):
    with fe.Hierarchy(N, 0, 3) as h:
        s = O.Space(O.Mesh(N), 3)
        assert h.n_dofs() == s.n == (3 * N + 1) ** 3 and h.n_cells() == 6 * N ** 3
        assert np.array_equal(h.dof_coordinates(), s.coords)
        assert np.array_equal(h.boundary_mask(), s.boundary)
        assert np.allclose(h.cell_centroids(), s.mesh.centroids(), atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 5])
@pytest.mark.parametrize("coef", ["one", "grf"])
@pytest.mark.parametrize("mode", ["double_float", "native"])
def test_p3_apply_f64_and_f32(fe, N, coef, mode):
    """FP64 operator in float pairs (default) and in FP64 FMAs, and the FP32 operator."""
    with fe.Hierarchy(N, 0, 3) as h:
        h.set_f64_mode(fe.FE_F64_NATIVE if mode == "native" else fe.FE_F64_DOUBLE_FLOAT)
        kappa = None if coef == "one" else I.grf_kappa(h.cell_centroids(), seed=N)
        h.set_coefficient(None if kappa is None else dt(kappa))
        L = O.Level(N, 3, kappa)
        x = I.random_vector(L.n, 30 + N)
        y = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.apply_operator(dt(x), y)
        y32 = torch.empty(L.n, dtype=torch.float32, device=DEV)
        x32 = x.astype(np.float32)
        h.apply_operator(dt(x32, torch.float32), y32, dtype=fe.FE_F32)
        torch.cuda.synchronize()
        assert_rowwise(host(y), L.A @ x, abs(L.A) @ np.abs(x), 1e-13, "P3 fp64 apply")
        xd = x32.astype(np.float64)
        assert_rowwise(host(y32), L.A @ xd, abs(L.A) @ np.abs(xd), 1e-5, "P3 fp32 apply")


@pytest.mark.parametrize("mode", ["double_float", "native"])
def test_p3_mass_and_diagonal(fe, mode):
    """P3 mass in float pairs (integer reference matrix, default) and in FP64; the diagonal."""
    N = 3
    with fe.Hierarchy(N, 0, 3) as h:
        h.set_f64_mode(fe.FE_F64_NATIVE if mode == "native" else fe.FE_F64_DOUBLE_FLOAT)
        kappa = I.grf_kappa(h.cell_centroids(), seed=5)
        h.set_coefficient(dt(kappa))
        L = O.Level(N, 3, kappa)
        x = I.random_vector(L.n, 8)
        y = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.apply_mass(dt(x), y)
        d = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.diagonal(d)
        torch.cuda.synchronize()
        assert_rowwise(host(y), L.M @ x, abs(L.M) @ np.abs(x), 1e-13, "P3 mass")
        assert_rowwise(host(d), L.diag, np.abs(L.diag), 1e-13, "P3 diagonal")


@pytest.mark.parametrize("N0", [1, 2, 3])
def test_p3_prolong_restrict(fe, N0):
    with fe.Hierarchy(N0, 1, 3) as h:
        c, f = O.Level(N0, 3), O.Level(2 * N0, 3)
        P = O.prolongation(c, f)
        xc = I.random_vector(c.n, 1)
        xf = torch.empty(f.n, dtype=torch.float64, device=DEV)
        h.prolong(dt(xc), xf, 1)
        rf = I.random_vector(f.n, 2)
        rc = torch.empty(c.n, dtype=torch.float64, device=DEV)
        h.restrict(dt(rf), rc, 1)
        rc0 = torch.empty(c.n, dtype=torch.float64, device=DEV)
        h.restrict(dt(rf), rc0, 1, zero_boundary=True)
        torch.cuda.synchronize()
        assert_rowwise(host(xf), P @ xc, abs(P) @ np.abs(xc), 1e-14, "P3 prolong")
        ref = P.T @ rf
        assert_rowwise(host(rc), ref, abs(P.T) @ np.abs(rf), 1e-14, "P3 restrict")
        ref[c.space.boundary] = 0
        assert_rowwise(host(rc0), ref, abs(P.T) @ np.abs(rf), 1e-14, "P3 restrict (zero bd)")


def test_p3_coarse_cholesky(fe):
    with fe.Hierarchy(2, 1, 3) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=2)
        h.set_coefficient(dt(kappa))
        oh = O.Hierarchy(2, 1, 3, kappa)
        c = oh.levels[0]
        b = I.random_vector(c.n, 9)
        x = torch.empty(c.n, dtype=torch.float64, device=DEV)
        h.coarse_solve(dt(b), x)
        torch.cuda.synchronize()
        ref = np.linalg.solve(c.A.toarray(), b)
        assert np.linalg.norm(host(x) - ref) <= 1e-11 * np.linalg.norm(ref)


def test_p3_smoother_and_vcycle(fe):
    with fe.Hierarchy(2, 2, 3) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=4)
        h.set_coefficient(dt(kappa))
        oh = O.Hierarchy(2, 2, 3, kappa)
        oh.lmax = [h.lambda_max(l) for l in range(3)]  # same Chebyshev intervals
        L = oh.fine
        b = I.random_vector(L.n, 5)
        b[L.space.boundary] = 0
        x0 = I.random_vector(L.n, 6)
        xs = dt(x0)
        h.smooth(dt(b), xs, steps=2, lo=0.1, hi=1.1)
        x = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.vcycle(dt(b), x)
        torch.cuda.synchronize()
        lm = oh.lmax[2]
        ref_s = O.chebyshev(lambda v: L.A @ v, L.diag, b, x0, 0.1 * lm, 1.1 * lm, 2)
        assert np.linalg.norm(host(xs) - ref_s) <= 1e-12 * np.linalg.norm(ref_s)
        ref = oh.vcycle(b)
        assert np.linalg.norm(host(x) - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("N0,nref,mode", [(1, 2, "double_float"), (2, 1, "native"), (2, 2, "double_float"),
                                          (2, 2, "native")])
def test_p3_gmg_pcg_solution_parity(fe, N0, nref, mode):
    with fe.Hierarchy(N0, nref, 3) as h:
        h.set_f64_mode(fe.FE_F64_NATIVE if mode == "native" else fe.FE_F64_DOUBLE_FLOAT)
        kappa = I.grf_kappa(h.cell_centroids(), seed=6)
        h.set_coefficient(dt(kappa))
        L = O.Level(N0 * 2 ** nref, 3, kappa)
        f = I.sin_product_rhs(L.space.coords)
        b = O.load_vector(L, f)
        ue = O.direct_solve(L, b)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        st = h.solve(dt(f), u, rtol=1e-13)
        assert np.linalg.norm(host(u) - ue) <= 1e-10 * np.linalg.norm(ue)
        assert st.iterations <= 40
        st2 = h.solve(f, np.empty(L.n), rtol=1e-13)  # host pointers (end-to-end path)
        assert st2.iterations == st.iterations


def test_p3_mixed_precision_and_fmg(fe):
    with fe.Hierarchy(2, 2, 3) as h:
        L = O.Level(8, 3)
        f = I.sin_product_rhs(L.space.coords)
        b = O.load_vector(L, f)
        ue = O.direct_solve(L, b)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        st = h.solve(dt(f), u, rtol=1e-8, precision=fe.FE_PREC_MIXED_F32)
        uh = host(u)
        assert np.linalg.norm(L.A @ uh - b) <= 1.0001e-8 * np.linalg.norm(b)
        assert st.outer_iterations >= 2
        assert np.linalg.norm(uh - ue) <= 1e-6 * np.linalg.norm(ue)
        # full multigrid as the whole solve: each V-cycle in defect form reduces the error
        errs = []
        for cycles in (1, 2, 3):
            st = h.solve(dt(f), u, precond=fe.FE_PC_FMG, max_it=cycles)
            errs.append(np.linalg.norm(host(u) - ue))
        assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1], errs


def test_p3_full_size_sampled_rows(fe):
    """The P3 benchmark mesh (UnitCubeMesh 32^3, 912,673 dofs): sampled rows of the FP64 and FP32 operators
    against the oracle's row-by-row element sums."""
    N = 32
    with fe.Hierarchy(4, 3, 3) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=9)
        h.set_coefficient(dt(kappa))
        space = O.Space(O.Mesh(N), 3)
        x = I.random_vector(space.n, 3)
        y = torch.empty(space.n, dtype=torch.float64, device=DEV)
        h.apply_operator(dt(x), y)
        y32 = torch.empty(space.n, dtype=torch.float32, device=DEV)
        h.apply_operator(dt(x, torch.float32), y32, dtype=fe.FE_F32)
        torch.cuda.synchronize()
        rows = np.random.default_rng(4).choice(space.n, 300, replace=False)
        ref = O.apply_rows(space, kappa, x, rows)
        # a global bound at this size (row-wise |A||x| bounds are in the small-mesh tests above)
        assert np.abs(host(y)[rows] - ref).max() <= 1e-12 * np.abs(ref).max()
        x32 = x.astype(np.float32).astype(np.float64)
        ref32 = O.apply_rows(space, kappa, x32, rows)
        assert np.abs(host(y32)[rows] - ref32).max() <= 1e-4 * np.abs(ref32).max()


def test_p3_batched_is_unsupported(fe):
    with pytest.raises(fe.FeError) as e:
        fe.Batch([(2, 1, 3)])
    assert e.value.code == fe.FE_ERR_UNSUPPORTED


def test_p3_mixed_bf16_tensor_core_solve(fe):
    """FP64 iterative refinement around the GMG-PCG whose smoother applies the P3 operator on the tensor cores
    (K = 20 -> 32): reaches the FP64 solution at rtol 1e-10."""
    with fe.Hierarchy(2, 2, 3) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=9)
        h.set_coefficient(dt(kappa))
        f = dt(I.sin_product_rhs(h.dof_coordinates()))
        u64 = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        ub = torch.empty_like(u64)
        h.solve(f, u64, rtol=1e-12)
        st = h.solve(f, ub, rtol=1e-10, precision=fe.FE_PREC_MIXED_BF16, max_it=40)
        assert st.rel_residual <= 1e-10
        assert (torch.linalg.norm(ub - u64) / torch.linalg.norm(u64)).item() <= 1e-8
