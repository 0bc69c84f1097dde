"""The batched persistent solver (one cooperative launch for many problems).

Each problem of a batch must match the single-problem FP64 GMG-PCG solver and
the oracle's direct solve (1e-10 relative L2 at rtol 1e-13); a deliberately
tiny barrier time limit must end the kernel with FE_ERR_TIMEOUT and leave the
batch usable; the full workload (64 problems, P1/P2, 16^3..48^3, GRF kappa)
must reach the 1e-8 residual on every problem, checked independently on
sampled rows by the oracle.
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
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, torch.float64)


SMALL = [(1, 2, 1), (2, 2, 2), (1, 2, 2), (3, 2, 1), (2, 2, 1), (3, 2, 2)]  # (N0, nrefine, degree)


def _setup(fe, sizes, seed0=100):
    B = fe.Batch(sizes)
    kappas, fs, us = [], [], []
    for p, h in enumerate(B.problems):
        big = h.n_cells() > 100000
        kap = I.grf_kappa(h.cell_centroids(), seed=seed0 + p, device=DEV if big else None)
        h.set_coefficient(dt(kap))
        kappas.append(kap)
        fs.append(torch.ones(h.n_dofs(), dtype=torch.float64, device=DEV))
        us.append(torch.empty(h.n_dofs(), dtype=torch.float64, device=DEV))
    return B, kappas, fs, us


def test_batched_matches_single_and_oracle(fe):
    B, kappas, fs, us = _setup(fe, SMALL)
    with B:
        stats = B.solve(fs, us, rtol=1e-13, max_it=200)
        for p, (h, (N0, nref, k)) in enumerate(zip(B.problems, SMALL)):
            L = O.Level(N0 * 2 ** nref, k, kappas[p])
            b = O.load_vector(L, np.ones(L.n))
            ue = O.direct_solve(L, b)
            ub = us[p].cpu().numpy()
            assert np.linalg.norm(ub - ue) <= 1e-10 * np.linalg.norm(ue), p
            u1 = torch.empty_like(us[p])
            st1 = h.solve(fs[p], u1, rtol=1e-13, max_it=200)
            assert abs(stats[p].iterations - st1.iterations) <= 1, (p, stats[p].iterations, st1.iterations)
            assert stats[p].rel_residual <= 1e-13
        # a second solve reuses the captured graph and gives the same answers
        us2 = [torch.empty_like(u) for u in us]
        B.solve(fs, us2, rtol=1e-13, max_it=200)
        for a, b2 in zip(us, us2):
            assert torch.allclose(a, b2, rtol=0, atol=1e-12 * a.abs().max().item())


def test_batched_barrier_timeout_is_reported(fe):
    B, kappas, fs, us = _setup(fe, SMALL[:3])
    with B:
        with pytest.raises(fe.FeError) as e:
            B.solve(fs, us, rtol=1e-10, wait_timeout_us=1, use_graph=0)
        assert e.value.code == fe.FE_ERR_TIMEOUT
        st = B.solve(fs, us, rtol=1e-10)  # the context and the batch stay usable
        assert all(s.rel_residual <= 1e-10 for s in st)


def test_batched_full_workload(fe):
    """64 problems, sizes drawn from {16,...,48} (multiples of 8), half P1 half P2, 4 levels, rtol 1e-8."""
    table = I.batched_problem_table()
    sizes = [(N // 8, 3, k) for N, k in table]
    B, kappas, fs, us = _setup(fe, sizes)
    with B:
        stats = B.solve(fs, us, rtol=1e-8)
        assert all(s.rel_residual <= 1e-8 for s in stats)
        assert max(s.iterations for s in stats) <= 30
        # independent residual check on sampled rows of three problems (oracle, cell by cell):
        # |b_i - (A u)_i| <= ||b - A u||_2 <= 1e-8 ||b||_2 with b = M 1 (Dirichlet rows 0)
        rng = np.random.default_rng(0)
        for p in (0, 17, 63):
            N, k = table[p]
            space = O.Space(O.Mesh(N), k)
            u = us[p].cpu().numpy()
            rows = rng.choice(space.n, 200, replace=False)
            b = np.where(space.boundary[rows], 0.0, O.apply_rows_mass(space, np.ones(space.n), rows))
            Au = O.apply_rows(space, kappas[p], u, rows)
            assert np.abs(Au - b).max() <= 1.01e-8 * stats[p].bnorm


def test_batched_phase_clock(fe):
    """opts.profile: block 0 of the persistent launch charges the wall time between grid barriers to
    (phase, level); the same solution and iteration counts as the unprofiled launch."""
    B, kappas, fs, us = _setup(fe, SMALL[:4])
    with B:
        st0 = B.solve(fs, us, rtol=1e-10)
        ref = [u.clone() for u in us]
        st = B.solve(fs, us, rtol=1e-10, profile=1)
        nl = B.problems[0].nlev
        for s0, s1, a, b in zip(st0, st, ref, us):
            assert s0.iterations == s1.iterations
            assert torch.allclose(a, b, rtol=0, atol=1e-12 * a.abs().max().item())
        P = np.array([list(r) for r in st[0].phase_ms])
        assert st[0].levels_timed == nl and np.all(P >= 0) and np.all(P[:, nl:] == 0)
        assert P[fe.FE_PHASE_COARSE, 0] > 0 and np.all(P[fe.FE_PHASE_COARSE, 1:] == 0)
        assert np.all(P[fe.FE_PHASE_SMOOTH, 1:nl] > 0) and np.all(P[fe.FE_PHASE_TRANSFER, 1:nl] > 0)
        assert P[fe.FE_PHASE_APPLY, nl - 1] > 0 and P[fe.FE_PHASE_BLAS1, nl - 1] > 0
        assert P.sum() <= st[0].solve_ms
        assert all(np.array_equal(P, np.array([list(r) for r in s.phase_ms])) for s in st)
