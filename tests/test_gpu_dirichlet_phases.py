"""Inhomogeneous Dirichlet data through fe_solve_poisson's bc_values, and the per-phase, per-level timers of a
profiled solve.

Dirichlet data (Sec. 2, Eq. 1: u = g on the boundary): the library eliminates g symmetrically (b_i -= A_ij g_j on
interior rows, b_j = g_j on the boundary), as the oracle's ``load_vector(..., bc_values)`` does.  Pinned two ways:
against the oracle's direct solve of the same elimination (FP64, relative L2 1e-10 at rtol 1e-13), and by the patch
test -- a polynomial u of the element degree with f = -Laplace(u) and g = u on the boundary is reproduced at every
node (the Galerkin solution is u itself), up to the solve's rtol times the condition number.
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


def dt(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def boundary_data(X):
    """A smooth, non-polynomial g(x, y, z) for the parity cases."""
    return np.exp(X[:, 0]) * np.cos(2 * X[:, 1]) + X[:, 2] ** 2


@pytest.mark.parametrize("k,N0,nref", [(1, 2, 2), (2, 2, 1), (3, 2, 1)])
@pytest.mark.parametrize("coef", ["one", "grf"])
def test_dirichlet_data_matches_oracle(fe, k, N0, nref, coef):
    with fe.Hierarchy(N0, nref, k) as h:
        kappa = None if coef == "one" else I.grf_kappa(h.cell_centroids(), seed=17)
        if kappa is not None:
            h.set_coefficient(dt(kappa))
        X = h.dof_coordinates()
        f = I.sin_product_rhs(X)
        g = boundary_data(X)
        L = O.Level(N0 << nref, k, kappa)
        ref = O.direct_solve(L, O.load_vector(L, f, bc_values=g))
        u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        h.solve(dt(f), u, bc_values=dt(g), rtol=1e-13, max_it=2000)
        got = u.cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
        bd = L.space.boundary
        assert np.array_equal(got[bd], g[bd])  # boundary values are set, not solved for
        # host pointers for the data and the load given as an assembled vector (FE_RHS_LOAD: its boundary
        # entries are replaced by g)
        b_load = L.M @ f
        b_load[bd] = 123.0
        u2 = np.empty(h.n_dofs())
        h.solve(b_load, u2, rhs_kind=fe.FE_RHS_LOAD, bc_values=g, rtol=1e-13, max_it=2000)
        assert np.linalg.norm(u2 - ref) <= 1e-10 * np.linalg.norm(ref)


PATCH = {
    # degree: (u, f = -Laplace(u))
    1: (lambda X: 1.0 + 2.0 * X[:, 0] - X[:, 1] + 3.0 * X[:, 2], lambda X: np.zeros(len(X))),
    2: (lambda X: X[:, 0] ** 2 + X[:, 1] * X[:, 2] - 2.0 * X[:, 2] ** 2 + X[:, 0],
        lambda X: np.full(len(X), 2.0)),
    3: (lambda X: X[:, 0] ** 3 + X[:, 0] * X[:, 1] * X[:, 2] - 2.0 * X[:, 1] ** 2 * X[:, 2] + X[:, 2],
        lambda X: -6.0 * X[:, 0] + 4.0 * X[:, 2]),
}


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("precond", ["gmg", "fmg"])
def test_dirichlet_patch_test(fe, k, precond):
    """u of degree k is in the discrete space and f = -Laplace(u) has degree <= k, so b = M I_h f is the exact
    load and the discrete solution is u at every node."""
    ue_fn, f_fn = PATCH[k]
    with fe.Hierarchy(2, 2, k) as h:
        X = h.dof_coordinates()
        ue = ue_fn(X)
        u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        if precond == "gmg":
            h.solve(dt(f_fn(X)), u, bc_values=dt(ue), rtol=1e-13, max_it=2000)
        else:  # full multigrid with enough cycles per level to reach the discrete solution
            h.solve(dt(f_fn(X)), u, bc_values=dt(ue), precond=fe.FE_PC_FMG, max_it=30)
        err = np.abs(u.cpu().numpy() - ue).max()
        assert err <= 1e-10 * np.abs(ue).max(), err


def test_dirichlet_mixed_precision(fe):
    """The refinement solve takes the same eliminated load: it reaches the FP64 solution with data g."""
    with fe.Hierarchy(4, 2, 2) as h:
        X = h.dof_coordinates()
        f, g = I.sin_product_rhs(X), boundary_data(X)
        u64 = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        u32 = torch.empty_like(u64)
        h.solve(dt(f), u64, bc_values=dt(g), rtol=1e-12)
        st = h.solve(dt(f), u32, bc_values=dt(g), rtol=1e-10, precision=fe.FE_PREC_MIXED_F32, max_it=30)
        assert st.rel_residual <= 1e-10
        assert (torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64)).item() <= 1e-8


# ------------------------------------------------------------------ phase timers
@pytest.mark.parametrize("k", [1, 2])
def test_phase_timers(fe, k):
    """opts.profile brackets every phase of every level with events: smoothing, residual applications and
    transfers on levels >= 1, the direct solve on level 0 only, CG's own applications and vector work on the
    finest level; their sum is the solve's device time (below the host wall time)."""
    with fe.Hierarchy(2, 3, k) as h:
        f = dt(I.sin_product_rhs(h.dof_coordinates()))
        u = torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV)
        st = h.solve(f, u, rtol=1e-8, profile=1)
        nl = h.nlev
        assert st.levels_timed == nl
        P = np.array([list(r) for r in st.phase_ms])
        assert P.shape == (fe.FE_NUM_PHASES, fe.FE_MAX_LEVELS)
        assert np.all(P >= 0) and np.all(P[:, nl:] == 0)
        assert P[fe.FE_PHASE_COARSE, 0] > 0 and np.all(P[fe.FE_PHASE_COARSE, 1:] == 0)
        for ph in (fe.FE_PHASE_SMOOTH, fe.FE_PHASE_TRANSFER):
            assert P[ph, 0] == 0 and np.all(P[ph, 1:nl] > 0), (ph, P[ph])
        assert np.all(P[fe.FE_PHASE_APPLY, 1:nl] > 0)
        assert P[fe.FE_PHASE_BLAS1, nl - 1] > 0
        # CG's own applications are part of the finest level's APPLY time
        assert P[fe.FE_PHASE_APPLY, nl - 1] >= st.apply_ms * (1 - 1e-6)
        assert 0 < P.sum() <= st.solve_ms
        # without profiling nothing is timed
        st0 = h.solve(f, u, rtol=1e-8)
        assert st0.levels_timed == 0 and all(v == 0 for row in st0.phase_ms for v in row)
        # full multigrid: transfers, coarse solve and per-level V-cycles are timed too
        stf = h.solve(f, u, precond=fe.FE_PC_FMG, max_it=1, profile=1)
        Pf = np.array([list(r) for r in stf.phase_ms])
        assert Pf[fe.FE_PHASE_COARSE, 0] > 0 and np.all(Pf[fe.FE_PHASE_TRANSFER, 1:nl] > 0)
