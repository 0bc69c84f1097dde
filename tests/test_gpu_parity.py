"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 operator/mass/diagonal/transfer/smoother applications are
compared elementwise against |A||x| (the rounding-error scale of each row) with
a factor 1e-13; FP32 applications at 1e-5 of that scale; FP64 solutions at a
relative L2 error of 1e-10 with both sides solved to rtol 1e-13.
"""
import numpy as np
import pytest

import fe_inputs as I
from oracle import fe_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08012_gb300 import build
    build.build()
    import paper_2104_08012_gb300 as fe
    fe.load()
    return fe


DEV = "cuda"


def dt(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def assert_rowwise(got, ref, scale, tol, what):
    err = np.abs(got - ref)
    bound = tol * np.maximum(scale, 1e-300)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"{what}: {bad.size} rows off, worst {np.max(err / bound):.3g}x tol at {bad[:5]}"


# ------------------------------------------------------------------ mesh
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("N", [1, 3, 4])
def test_mesh_queries_match_oracle(fe, k, N):
    with fe.Hierarchy(N, 0, k) as h:
        s = O.Space(O.Mesh(N), k)
        assert h.n_dofs() == s.n and h.n_cells() == 6 * N ** 3
        assert np.array_equal(h.dof_coordinates(), s.coords)
        assert np.array_equal(h.boundary_mask(), s.boundary)
        assert np.allclose(h.cell_centroids(), s.mesh.centroids(), atol=1e-15)


# ------------------------------------------------------------ operator
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("coef", ["one", "grf", "grf_per_pair"])
@pytest.mark.parametrize("mode", ["native", "double_float", "double_float_tet", "double_float_cube",
                                  "double_float_pair"])
def test_apply_f64(fe, k, N, coef, mode):
    """FP64 operator in both arithmetics: FP64 FMAs and float-pair (~48-bit) on the FP32 pipes
    (per cube, per tet, and two tets per thread in packed FP32x2 instructions).  In the default mode the P2
    operator is the solver's: pre-split input, fixed-point limbs, one tet per unit under a coefficient that varies
    from tet to tet ("grf"), the two tets that share a face as one unit where they have the same coefficient ("one",
    and "grf_per_pair": the value of the pair's first tet on both)."""
    with fe.Hierarchy(N, 0, k) as h:
        h.set_f64_mode({"native": fe.FE_F64_NATIVE, "double_float": fe.FE_F64_DOUBLE_FLOAT,
                        "double_float_cube": fe.FE_F64_DOUBLE_FLOAT_CUBE,
                        "double_float_tet": fe.FE_F64_DOUBLE_FLOAT_TET,
                        "double_float_pair": fe.FE_F64_DOUBLE_FLOAT_PAIR}[mode])
        kappa = None if coef == "one" else I.grf_kappa(h.cell_centroids(), seed=N)
        if coef == "grf_per_pair":
            kappa[1::2] = kappa[0::2]
        h.set_coefficient(None if kappa is None else dt(kappa))
        L = O.Level(N, k, kappa)
        x = I.random_vector(L.n, 10 + N)
        y = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.apply_operator(dt(x), y)
        torch.cuda.synchronize()
        scale = abs(L.A) @ np.abs(x)
        assert_rowwise(host(y), L.A @ x, scale, 1e-13, "fp64 apply")


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("N,variable_kappa", [(6, True), (17, True), (12, False)])
def test_apply_f32(fe, k, N, variable_kappa):
    """FP32 apply (one thread per cube, 256 per block): meshes whose cube counts leave a
    ragged last block (N=6, N=17) and a constant coefficient (N=12)."""
    with fe.Hierarchy(N, 0, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=3) if variable_kappa else np.ones(6 * N ** 3)
        if variable_kappa:
            h.set_coefficient(dt(kappa))
        L = O.Level(N, k, kappa)
        x = I.random_vector(L.n, 4).astype(np.float32)
        y = torch.empty(L.n, dtype=torch.float32, device=DEV)
        h.apply_operator(dt(x, torch.float32), y, dtype=fe.FE_F32)
        torch.cuda.synchronize()
        xd = x.astype(np.float64)
        assert_rowwise(host(y), L.A @ xd, abs(L.A) @ np.abs(xd), 1e-5, "fp32 apply")


@pytest.mark.parametrize("scale", [1e-300, 1e-250, 1e-30, 1e-8, 1.0, 1e8, 1e30, 1e250, 1e300])
@pytest.mark.parametrize("mode", ["double_float", "double_float_cube", "double_float_tet", "double_float_pair"])
def test_double_float_value_range(fe, scale, mode):
    """The float-pair split/widen keep FP64-class accuracy from 1e-300 to 1e300 (each tet's dofs are scaled by a
    power of two first; contributions below the normal FP64 range widen to subnormal doubles), with exact zeros
    and sign changes, and NaN dofs propagate."""
    with fe.Hierarchy(3, 0, 2) as h:
        h.set_f64_mode({"double_float": fe.FE_F64_DOUBLE_FLOAT, "double_float_cube": fe.FE_F64_DOUBLE_FLOAT_CUBE,
                        "double_float_tet": fe.FE_F64_DOUBLE_FLOAT_TET,
                        "double_float_pair": fe.FE_F64_DOUBLE_FLOAT_PAIR}[mode])
        L = O.Level(3, 2)
        x = I.random_vector(L.n, 77) * scale
        x[::7] = 0.0
        x[3::17] = -np.abs(x[3::17])
        y = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.apply_operator(dt(x), y)
        torch.cuda.synchronize()
        assert_rowwise(host(y), L.A @ x, abs(L.A) @ np.abs(x), 1e-13, "double-float value range")
        xn = x.copy()
        xn[np.nonzero(~L.space.boundary)[0][0]] = np.nan
        h.apply_operator(dt(xn), y)
        assert torch.isnan(y).any()


@pytest.mark.parametrize("scale", [1.0, 1e-40, 1e40, 1e-100, 1e100])
def test_presplit_inputs_match_in_kernel_split(fe, scale):
    """Inside the solver the P2 float-pair operator gathers its input as float pairs written by the kernel that
    produced it (Chebyshev update, prolongation, CG direction); dofs outside [2^-64, 2^64) are markers and their
    tets split the FP64 values themselves.  The V-cycle and the CG solution equal those of the mode that always
    splits inside the operator (FE_F64_DOUBLE_FLOAT_TET) up to the order of the atomic additions, at every scale
    and with a right-hand side whose entries span 2^-100 .. 2^100 (tets of both kinds in one launch)."""
    with fe.Hierarchy(4, 2, 2) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=8)
        h.set_coefficient(dt(kappa))
        n = h.n_dofs()
        f = I.random_vector(n, 3) * scale
        g = f.copy()
        g[::11] *= 2.0 ** 100 if scale <= 1.0 else 2.0 ** -100
        out = {}
        for mode in (fe.FE_F64_DOUBLE_FLOAT, fe.FE_F64_DOUBLE_FLOAT_TET):
            h.set_f64_mode(mode)
            v = torch.empty(n, dtype=torch.float64, device=DEV)
            h.vcycle(dt(f), v)
            u = torch.empty(n, dtype=torch.float64, device=DEV)
            st = h.solve(dt(f), u, rhs_kind=fe.FE_RHS_LOAD, rtol=1e-12)
            w = torch.empty(n, dtype=torch.float64, device=DEV)
            h.solve(dt(g), w, rhs_kind=fe.FE_RHS_LOAD, rtol=1e-12)
            out[mode] = (host(v), host(u), host(w), st.iterations)
        a, b = out[fe.FE_F64_DOUBLE_FLOAT], out[fe.FE_F64_DOUBLE_FLOAT_TET]
        assert np.abs(a[0] - b[0]).max() <= 1e-13 * np.abs(b[0]).max()
        assert np.linalg.norm(a[1] - b[1]) <= 1e-11 * np.linalg.norm(b[1]) and a[3] == b[3]
        assert np.linalg.norm(a[2] - b[2]) <= 1e-11 * np.linalg.norm(b[2])


def test_paired_float_pair_kernel_matches_per_tet(fe):
    """The packed two-tets-per-thread kernel evaluates the element with the six stored geometric factors per cell,
    the per-tet kernel with one factor per cell times the matrix M shared by every Kuhn tet; both are the same
    operator in float-pair arithmetic, so they agree to the FP64 rounding scale of each row."""
    with fe.Hierarchy(12, 0, 2) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=5)
        h.set_coefficient(dt(kappa))
        L = O.Level(12, 2, kappa)
        xh = I.random_vector(h.n_dofs(), 21)
        x = dt(xh)
        ys = {}
        for mode in (fe.FE_F64_DOUBLE_FLOAT_TET, fe.FE_F64_DOUBLE_FLOAT_PAIR):
            h.set_f64_mode(mode)
            ys[mode] = torch.empty_like(x)
            h.apply_operator(x, ys[mode])
        torch.cuda.synchronize()
        scale = abs(L.A) @ np.abs(xh)
        assert_rowwise(host(ys[fe.FE_F64_DOUBLE_FLOAT_TET]), host(ys[fe.FE_F64_DOUBLE_FLOAT_PAIR]), scale, 2e-14,
                       "per-tet vs paired kernels")


def test_apply_host_pointers_match_device(fe):
    with fe.Hierarchy(4, 0, 2) as h:
        x = I.random_vector(h.n_dofs(), 7)
        y_host = np.empty_like(x)
        h.apply_operator(x, y_host)  # numpy in, numpy out: staged through the library
        y_dev = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        h.apply_operator(dt(x), y_dev)
        torch.cuda.synchronize()
        L = O.Level(4, 2)
        assert_rowwise(y_host, L.A @ x, abs(L.A) @ np.abs(x), 1e-13, "host-pointer apply")
        assert_rowwise(host(y_dev), y_host, abs(L.A) @ np.abs(x), 1e-13, "host vs device")


@pytest.mark.parametrize("k", [1, 2])
def test_mass_and_diagonal(fe, k):
    N = 4
    with fe.Hierarchy(N, 0, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=5)
        h.set_coefficient(dt(kappa))
        L = O.Level(N, k, kappa)
        x = I.random_vector(L.n, 8)
        y = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.apply_mass(dt(x), y)
        d = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.diagonal(d)
        torch.cuda.synchronize()
        assert_rowwise(host(y), L.M @ x, abs(L.M) @ np.abs(x), 1e-13, "mass")
        assert_rowwise(host(d), L.diag, np.abs(L.diag), 1e-13, "diagonal")


# ------------------------------------------------------------ transfers
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("N0", [1, 2, 3])
def test_prolong_restrict(fe, k, N0):
    """Prolongation rows are sums of at most m = 2 (P1) or 10 (P2) weighted coarse values.  Each side's sum is
    within (m - 1) u sum |w x| of the exact one (u = 2^-53), and the oracle's weights (basis values at reference
    coordinates found by a linear solve) are within about u |w| of the exact dyadic weights the library uses, so the
    two results differ by at most about 4 m u of the row scale |P| |x|: 8.9e-16 (P1), 4.4e-15 (P2)."""
    m = 2 if k == 1 else 10
    with fe.Hierarchy(N0, 1, k) as h:
        c, f = O.Level(N0, k), O.Level(2 * N0, k)
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
        assert_rowwise(host(xf), P @ xc, abs(P) @ np.abs(xc), 4 * m * 2.0 ** -53, "prolong")
        ref = P.T @ rf
        assert_rowwise(host(rc), ref, abs(P.T) @ np.abs(rf), 1e-14, "restrict")
        ref[c.space.boundary] = 0
        assert_rowwise(host(rc0), ref, abs(P.T) @ np.abs(rf), 1e-14, "restrict (zero bd)")


def test_transfers_p2_full_size(fe):
    """On large P2 levels the prolongation runs per coarse cube with compile-time weights (k_prolong_cube); the level
    pair 32^3 -> 64^3 of the benchmark hierarchy against the oracle's P and P^T row by row, prolongation with and
    without accumulation, restriction with and without zeroed boundary rows, at the FP64 bounds of
    test_prolong_restrict."""
    import types
    with fe.Hierarchy(8, 3, 2) as h:
        sc, sf = O.Space(O.Mesh(32), 2), O.Space(O.Mesh(64), 2)
        c = types.SimpleNamespace(mesh=sc.mesh, space=sc, n=sc.n)
        f = types.SimpleNamespace(mesh=sf.mesh, space=sf, n=sf.n)
        P = O.prolongation(c, f)
        xc = I.random_vector(c.n, 31)
        x0 = I.random_vector(f.n, 32)
        xf = torch.empty(f.n, dtype=torch.float64, device=DEV)
        h.prolong(dt(xc), xf, 3)
        xa = dt(x0)
        h.prolong(dt(xc), xa, 3, accumulate=True)
        torch.cuda.synchronize()
        rf = I.random_vector(f.n, 33)
        rc = torch.empty(c.n, dtype=torch.float64, device=DEV)
        h.restrict(dt(rf), rc, 3)
        rc0 = torch.empty(c.n, dtype=torch.float64, device=DEV)
        h.restrict(dt(rf), rc0, 3, zero_boundary=True)
        torch.cuda.synchronize()
        tol = 4 * 10 * 2.0 ** -53
        assert_rowwise(host(xf), P @ xc, abs(P) @ np.abs(xc), tol, "prolong (per cube)")
        assert_rowwise(host(xa), x0 + P @ xc, np.abs(x0) + abs(P) @ np.abs(xc), tol, "prolong (per cube, accumulate)")
        ref = P.T @ rf
        assert_rowwise(host(rc), ref, abs(P.T) @ np.abs(rf), 1e-14, "restrict (full size)")
        ref[sc.boundary] = 0
        assert_rowwise(host(rc0), ref, abs(P.T) @ np.abs(rf), 1e-14, "restrict (full size, zero bd)")


# ------------------------------------------------------------ smoother
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_chebyshev_smoother(fe, k, steps):
    N = 4
    with fe.Hierarchy(N, 0, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=11)
        h.set_coefficient(dt(kappa))
        L = O.Level(N, k, kappa)
        lm = h.lambda_max()
        b, x0 = I.random_vector(L.n, 3), I.random_vector(L.n, 4)
        x = dt(x0)
        h.smooth(dt(b), x, steps=steps, lo=0.1, hi=1.1)
        torch.cuda.synchronize()
        ref = O.chebyshev(lambda v: L.A @ v, L.diag, b, x0, 0.1 * lm, 1.1 * lm, steps)
        assert np.linalg.norm(host(x) - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("mode", ["df", "df_tet", "df_cube", "f32"])
def test_fused_smoother(fe, k, mode):
    """Smoothing with the Chebyshev update fused into the operator launch (per-dof countdowns) against the
    oracle's Chebyshev iteration and against the unfused kernels, on a fine and a coarse level, applied twice in a
    row (the countdowns must be restored for the second call)."""
    f64_mode = {"df": fe.FE_F64_DOUBLE_FLOAT, "df_tet": fe.FE_F64_DOUBLE_FLOAT_TET,
                "df_cube": fe.FE_F64_DOUBLE_FLOAT_CUBE, "f32": fe.FE_F64_DOUBLE_FLOAT}[mode]
    dtype, tdt = (fe.FE_F32, torch.float32) if mode == "f32" else (fe.FE_F64, torch.float64)
    tol = 1e-5 if mode == "f32" else 1e-12
    with fe.Hierarchy(3, 1, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=12)
        h.set_coefficient(dt(kappa))
        h.set_f64_mode(f64_mode)
        oh = O.Hierarchy(3, 1, k, kappa)
        for lev in (1, 0):
            L = oh.levels[lev]
            lm = h.lambda_max(lev)
            b, x0 = I.random_vector(L.n, 30 + lev), I.random_vector(L.n, 40 + lev)
            ref = x0
            for _ in range(2):
                ref = O.chebyshev(lambda v: L.A @ v, L.diag, b, ref, 0.1 * lm, 1.1 * lm, 3)
            got = {}
            for fused in (True, False):
                h.set_smoother_fusion(fused)
                x = dt(x0, tdt)
                for _ in range(2):
                    h.smooth(dt(b, tdt), x, level=lev, steps=3, lo=0.1, hi=1.1, dtype=dtype)
                torch.cuda.synchronize()
                got[fused] = host(x)
                err = np.linalg.norm(got[fused] - ref) / np.linalg.norm(ref)
                assert err <= tol, (lev, fused, err)
            h.set_smoother_fusion(True)
            assert np.linalg.norm(got[True] - got[False]) <= tol * np.linalg.norm(ref)


def test_lambda_max_p1_closed_form(fe):
    """Lanczos estimate of lambda_max(D^-1 A) for P1 against 1 + cos(pi h) (Kuhn P1 = h x 7-point)."""
    for N in (4, 8, 16):
        with fe.Hierarchy(N, 0, 1) as h:
            lm = h.lambda_max()
            exact = 1 + np.cos(np.pi / N)
            assert exact * (1 - 2e-2) <= lm <= exact * (1 + 1e-12), (N, lm, exact)


# --------------------------------------------------------- coarse solve
@pytest.mark.parametrize("k,N0", [(1, 4), (2, 2), (2, 4)])
def test_coarse_cholesky(fe, k, N0):
    with fe.Hierarchy(N0, 1, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=2)
        h.set_coefficient(dt(kappa))
        oh = O.Hierarchy(N0, 1, k, kappa)
        c = oh.levels[0]
        b = I.random_vector(c.n, 9)
        x = torch.empty(c.n, dtype=torch.float64, device=DEV)
        h.coarse_solve(dt(b), x)
        torch.cuda.synchronize()
        ref = np.linalg.solve(c.A.toarray(), b)
        assert np.linalg.norm(host(x) - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("k,N0", [(1, 4), (2, 2), (2, 4), (3, 2), (3, 4)])
def test_coarse_blocked_matches_oracle(fe, k, N0):
    """The blocked band factor (diagonal-block inverses and sub-diagonal blocks of B = bandwidth rows, the
    interior unknowns padded with identity rows to a multiple of B: P2 4^3 has 343 unknowns in 4 blocks of 114,
    P3 4^3 1331 in 4 blocks of 399) against the oracle's Cholesky solve of the same coarse level, and against the
    dense inverse factor; then a whole GMG-PCG solve through it against the oracle's solution."""
    with fe.Hierarchy(N0, 1, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=4)
        h.set_coefficient(dt(kappa))
        oh = O.Hierarchy(N0, 1, k, kappa)
        c = oh.levels[0]
        b = I.random_vector(c.n, 12)
        ref = oh.coarse_solve(b)
        out = {}
        for mode in (fe.FE_COARSE_BLOCKED, fe.FE_COARSE_DENSE):
            h.set_coarse_solver(mode)
            info = h.coarse_info()
            assert info["blocked"] == (mode == fe.FE_COARSE_BLOCKED) and info["n_interior"] == (k * N0 - 1) ** 3
            x = torch.empty(c.n, dtype=torch.float64, device=DEV)
            h.coarse_solve(dt(b), x)
            out[mode] = host(x)
            assert np.linalg.norm(out[mode] - ref) <= 1e-11 * np.linalg.norm(ref), mode
        assert np.linalg.norm(out[fe.FE_COARSE_BLOCKED] - out[fe.FE_COARSE_DENSE]) <= 1e-12 * np.linalg.norm(ref)
        h.set_coarse_solver(fe.FE_COARSE_BLOCKED)
        f = I.sin_product_rhs(h.dof_coordinates())
        L = oh.fine
        uo = O.direct_solve(L, O.load_vector(L, f))
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.solve(dt(f), u, rtol=1e-13, max_it=500)
        assert np.linalg.norm(host(u) - uo) <= 1e-10 * np.linalg.norm(uo)


def test_dense_coarse_solve_after_a_smaller_coarse_level(fe):
    """The one-launch dense coarse solve keeps its shared-memory limit when a hierarchy with a smaller coarse level is
    set up after it (the limit is a process-wide attribute of the kernel): P2 8^3 (3375 interior unknowns, 76 KB of
    shared memory per block), then P1 12^3 (1331 unknowns, 60 KB), then the first hierarchy's coarse solve against the
    oracle's and a whole solve to 1e-10."""
    with fe.Hierarchy(8, 1, 2) as big:
        oh = O.Hierarchy(8, 1, 2)
        c = oh.levels[0]
        b = I.random_vector(c.n, 13)
        ref = oh.coarse_solve(b)
        with fe.Hierarchy(12, 1, 1) as small:
            assert small.coarse_info()["n_interior"] == 11 ** 3 and not small.coarse_info()["blocked"]
            x = torch.empty(c.n, dtype=torch.float64, device=DEV)
            big.coarse_solve(dt(b), x)
            torch.cuda.synchronize()
            assert np.linalg.norm(host(x) - ref) <= 1e-11 * np.linalg.norm(ref)
            f = dt(I.sin_product_rhs(big.dof_coordinates()))
            u = torch.empty_like(f)
            st = big.solve(f, u, rtol=1e-10, max_it=100)
            assert st.rel_residual <= 1e-10 and st.iterations <= 15


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("coef", ["grf", "grf_per_pair", "one"])
def test_vcycle_matches_oracle(fe, k, coef):
    """One V-cycle against the oracle's; at P2 the operator units are single tets ("grf"), pairs of tets on the
    fine level ("grf_per_pair"; below it, single tets wherever the coarsened coefficient differs between the tets
    of a pair), or pairs on every level ("one")."""
    with fe.Hierarchy(2, 2, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=4)
        if coef == "grf_per_pair":
            kappa[1::2] = kappa[0::2]
        elif coef == "one":
            kappa[:] = 1.0
        h.set_coefficient(dt(kappa))
        oh = O.Hierarchy(2, 2, k, kappa)
        oh.lmax = [h.lambda_max(l) for l in range(3)]  # same Chebyshev intervals
        b = I.random_vector(oh.fine.n, 5)
        b[oh.fine.space.boundary] = 0
        x = torch.empty(oh.fine.n, dtype=torch.float64, device=DEV)
        h.vcycle(dt(b), x)
        torch.cuda.synchronize()
        ref = oh.vcycle(b)
        assert np.linalg.norm(host(x) - ref) <= 1e-11 * np.linalg.norm(ref)


# ---------------------------------------------------- quadrature load vector
@pytest.mark.parametrize("k", [1, 2, 3])
def test_quadrature_load_vector(fe, k):
    """fe_quadrature_points and fe_load_vector_quadrature against the oracle (points to 1e-15,
    load vector rowwise 1e-13), and a solve with FE_RHS_QUAD_F equals a solve with the assembled
    load vector passed as FE_RHS_LOAD."""
    with fe.Hierarchy(2, 1, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=8)
        h.set_coefficient(dt(kappa))
        L = O.Level(4, k, kappa)
        P = h.quadrature_points()
        Pref = O.quadrature_points(L.space.mesh)
        assert np.abs(P - Pref).max() <= 1e-15
        fq = I.sin_product_rhs(P.reshape(-1, 3)).reshape(P.shape[:2])
        ref = O.load_vector_quadrature(L, fq)
        b = torch.empty(L.n, dtype=torch.float64, device=DEV)
        h.load_vector_quadrature(dt(fq), b)
        torch.cuda.synchronize()
        # rowwise scale sum_K sum_q w_q |det J| |f| |phi_i| (P2 vertex functions change sign)
        xi, w = O.tet_quadrature(O.QUAD_N)
        phi, _ = O.ref_basis(k, xi)
        det = np.abs(np.linalg.det(L.space.mesh.jacobians()))
        scale = np.zeros(L.n)
        np.add.at(scale, L.space.cell_dofs, np.einsum("q,c,cq,qd->cd", w, det, np.abs(fq), np.abs(phi)))
        scale[L.space.boundary] = 1.0
        assert np.all(np.abs(host(b) - ref) <= 1e-13 * scale), np.max(np.abs(host(b) - ref) / scale)
        u1 = torch.empty_like(b)
        u2 = torch.empty_like(b)
        h.solve(dt(fq), u1, rhs_kind=fe.FE_RHS_QUAD_F, rtol=1e-12)
        h.solve(b, u2, rhs_kind=fe.FE_RHS_LOAD, rtol=1e-12)
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(u1 - u2)) <= 1e-11 * float(torch.linalg.norm(u2))
        # host pointers in and out (staged through the library's buffers) give the same results
        bh = np.empty(L.n)
        h.load_vector_quadrature(np.ascontiguousarray(fq), bh)
        assert np.all(np.abs(bh - host(b)) <= 1e-13 * scale)  # atomics: summation order may differ
        uh = np.empty(L.n)
        h.solve(np.ascontiguousarray(fq), uh, rhs_kind=fe.FE_RHS_QUAD_F, rtol=1e-12)
        assert np.linalg.norm(uh - host(u2)) <= 1e-11 * np.linalg.norm(host(u2))


# ---------------------------------------------------------- full multigrid
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("cycles", [1, 2])
def test_fmg_matches_oracle(fe, k, cycles):
    """Full multigrid as the whole solve (FE_PC_FMG) against the oracle's FMG with the same
    Chebyshev intervals; the reported residual is that of the returned solution; the captured
    graph and direct launches agree."""
    with fe.Hierarchy(2, 2, k) as h:
        kappa = I.grf_kappa(h.cell_centroids(), seed=6)
        h.set_coefficient(dt(kappa))
        oh = O.Hierarchy(2, 2, k, kappa)
        oh.lmax = [h.lambda_max(l) for l in range(3)]
        L = oh.fine
        f = I.sin_product_rhs(L.space.coords)
        b = O.load_vector(L, f)
        ref = oh.fmg(b, cycles=cycles)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        st = h.solve(dt(f), u, precond=fe.FE_PC_FMG, max_it=cycles)
        u2 = torch.empty_like(u)
        h.solve(dt(f), u2, precond=fe.FE_PC_FMG, max_it=cycles, use_graph=0)
        torch.cuda.synchronize()
        got = host(u)
        assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
        assert np.linalg.norm(host(u2) - got) <= 1e-13 * np.linalg.norm(got)
        rel = np.linalg.norm(b - L.A @ got) / np.linalg.norm(b)
        assert st.iterations == cycles and abs(st.rel_residual - rel) <= 1e-6 * rel


def test_fmg_full_size_accuracy_and_options(fe):
    """FMG on P2 64^3 (4 levels): every extra V-cycle per level cuts the residual and the algebraic error
    (distance to the discrete solution, a CG solve to 1e-12) at least 2x; with 4 V-cycles per level the
    algebraic error is below half the discretisation error at the nodes; invalid FMG options are refused."""
    with fe.Hierarchy(8, 3, 2) as h:
        X = h.dof_coordinates()
        f = dt(I.sin_product_rhs(X))
        ue = I.sin_product(X)
        u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        h.solve(f, u, rtol=1e-12)
        uh = host(u)
        rms = lambda v: float(np.sqrt(np.mean(v * v)))
        res, alg = [], []
        for c in (1, 2, 3, 4):
            st = h.solve(f, u, precond=fe.FE_PC_FMG, max_it=c)
            res.append(st.rel_residual)
            alg.append(rms(host(u) - uh))
        assert all(res[i + 1] <= 0.5 * res[i] and alg[i + 1] <= 0.5 * alg[i] for i in range(3)), (res, alg)
        assert alg[-1] <= 0.5 * rms(uh - ue), (alg, rms(uh - ue))
        for bad in (dict(max_it=0), dict(precision=fe.FE_PREC_MIXED_F32)):
            with pytest.raises(fe.FeError) as e:
                h.solve(f, u, precond=fe.FE_PC_FMG, **{**dict(max_it=1), **bad})
            assert e.value.code == fe.FE_ERR_ARG


# ---------------------------------------------------------------- solves
def test_config0_jacobi_pcg(fe):
    """P1 on UnitCubeMesh 8^3 (3072 cells, 729 vertices), Jacobi-PCG to rtol 1e-10."""
    with fe.Hierarchy(8, 0, 1) as h:
        assert h.n_cells() == 3072 and h.n_dofs() == 729
        L = O.Level(8, 1)
        f = I.sin_product_rhs(L.space.coords)
        b = O.load_vector(L, f)
        ue = O.direct_solve(L, b)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        st = h.solve(dt(f), u, precond=fe.FE_PC_JACOBI, rtol=1e-10)
        uh = host(u)
        assert st.rel_residual <= 1e-10
        assert np.linalg.norm(L.A @ uh - b) <= 1.01e-10 * np.linalg.norm(b)
        _, it_orc, _ = O.solve(L, b, rtol=1e-10, precond="jacobi")
        assert abs(st.iterations - it_orc) <= 1
        st = h.solve(dt(f), u, precond=fe.FE_PC_JACOBI, rtol=1e-13)
        assert np.linalg.norm(host(u) - ue) <= 1e-10 * np.linalg.norm(ue)
        # the discrete solution converges to the sin product at O(h^2)
        assert O.l2_error(L.space, host(u), I.sin_product) < 0.05


@pytest.mark.parametrize("k,N0,nref", [(1, 2, 2), (2, 2, 2), (2, 3, 1)])
@pytest.mark.parametrize("mode", ["native", "double_float"])
def test_gmg_pcg_solution_parity(fe, k, N0, nref, mode):
    with fe.Hierarchy(N0, nref, k) as h:
        h.set_f64_mode(fe.FE_F64_NATIVE if mode == "native" else fe.FE_F64_DOUBLE_FLOAT)
        kappa = I.grf_kappa(h.cell_centroids(), seed=6)
        h.set_coefficient(dt(kappa))
        L = O.Level(N0 * 2 ** nref, k, kappa)
        f = I.sin_product_rhs(L.space.coords)
        b = O.load_vector(L, f)
        ue = O.direct_solve(L, b)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        st = h.solve(dt(f), u, rtol=1e-13)
        assert np.linalg.norm(host(u) - ue) <= 1e-10 * np.linalg.norm(ue)
        assert st.iterations <= 30
        st2 = h.solve(f, np.empty(L.n), rtol=1e-13)  # host pointers (end-to-end path)
        assert st2.iterations == st.iterations


def test_gmg_pcg_localized_rhs_parity(fe):
    """A right-hand side nonzero in one corner region only: the first smoothing steps leave most tets with all-zero
    dofs, which the pre-split P2 operator skips, and the rest of the cube mixes zero and nonzero dofs within tets.
    The solution must still match the oracle's direct solve (P2, 3 levels, rtol 1e-13)."""
    k, N0, nref = 2, 2, 2
    with fe.Hierarchy(N0, nref, k) as h:
        L = O.Level(N0 * 2 ** nref, k)
        X = L.space.coords
        f = np.where((X[:, 0] < 0.3) & (X[:, 1] < 0.3) & (X[:, 2] < 0.3), 1.0 + X[:, 0], 0.0)
        b = O.load_vector(L, f)
        ue = O.direct_solve(L, b)
        u = torch.empty(L.n, dtype=torch.float64, device=DEV)
        st = h.solve(dt(f), u, rtol=1e-13)
        assert np.linalg.norm(host(u) - ue) <= 1e-10 * np.linalg.norm(ue)
        assert st.iterations <= 30


def test_gmg_iterations_mesh_independent(fe):
    its = []
    for nref in (1, 2, 3):
        with fe.Hierarchy(4, nref, 2) as h:
            f = dt(I.sin_product_rhs(h.dof_coordinates()))
            u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
            its.append(h.solve(f, u, rtol=1e-8).iterations)
    assert max(its) <= 15 and its[-1] - its[0] <= 3, its


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("cheb_steps", [2, 3])
def test_graph_cg_loop_matches_host_loop(fe, k, cheb_steps):
    """The device-side CG loop (conditional graph node) runs the same kernels as the host-driven loop: the same
    iteration count and the same solution up to the order of the operator's atomic additions; the launch counter
    sees the loop's kernels (the graph path adds one parameter kernel, one loop test before the loop and one per
    further iteration)."""
    with fe.Hierarchy(4, 2, k) as h:
        f = dt(I.sin_product_rhs(h.dof_coordinates()))
        u1 = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        u2 = torch.empty_like(u1)
        h.solve(f, u1, rtol=1e-10, cheb_steps=cheb_steps)  # builds the loop graph
        n0 = fe.fe_kernel_launches()
        s1 = h.solve(f, u1, rtol=1e-10, cheb_steps=cheb_steps)
        n1 = fe.fe_kernel_launches()
        s2 = h.solve(f, u2, rtol=1e-10, cheb_steps=cheb_steps, profile=1)  # host-driven loop
        n2 = fe.fe_kernel_launches()
        torch.cuda.synchronize()
        assert s1.iterations == s2.iterations > 1
        assert s1.rel_residual <= 1e-10 and s2.rel_residual <= 1e-10
        assert abs(s1.rel_residual - s2.rel_residual) <= 1e-6 * s2.rel_residual
        assert float(torch.linalg.norm(u1 - u2)) <= 1e-12 * float(torch.linalg.norm(u2))
        assert (n1 - n0) == (n2 - n1) + s1.iterations + 1


def test_graph_cg_loop_limits(fe):
    """Iteration limit and non-finite residuals end the device-side loop with the host loop's status codes."""
    with fe.Hierarchy(4, 1, 2) as h:
        f = dt(I.sin_product_rhs(h.dof_coordinates()))
        u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        for it in (1, 2, 3):
            for prof in (0, 1):
                with pytest.raises(fe.FeError) as e:
                    h.solve(f, u, rtol=1e-14, max_it=it, profile=prof)
                assert e.value.code == fe.FE_ERR_NO_CONVERGENCE
        st = h.solve(f, u, rtol=1e-8, max_it=50)
        assert st.iterations < 50 and st.rel_residual <= 1e-8
        nanf = f.clone()
        nanf[7] = float("inf")
        with pytest.raises(fe.FeError) as e:
            h.solve(nanf, u, rtol=1e-8)
        assert e.value.code == fe.FE_ERR_NAN


def test_solver_errors(fe):
    with fe.Hierarchy(4, 1, 1) as h:
        f = dt(I.sin_product_rhs(h.dof_coordinates()))
        u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        with pytest.raises(fe.FeError) as e:
            h.solve(f, u, rtol=1e-12, max_it=1)
        assert e.value.code == fe.FE_ERR_NO_CONVERGENCE
        with pytest.raises(fe.FeError) as e:
            h.apply_operator(u, u)
        assert e.value.code == fe.FE_ERR_ARG
        with pytest.raises(fe.FeError) as e:
            h.set_coefficient(dt(-np.ones(h.n_cells())))
        assert e.value.code == fe.FE_ERR_ARG
        nanf = f.clone()
        nanf[5] = float("nan")
        with pytest.raises(fe.FeError) as e:
            h.solve(nanf, u, rtol=1e-8)
        assert e.value.code == fe.FE_ERR_NAN

