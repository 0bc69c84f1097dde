"""Pins of the oracle's vertex-star patch preconditioner (the paper's PatchPC with star patches around
vertices, Section 3), CPU only.

What fixes it independently of its own code: for P1 a vertex star holds one dof, so additive Schwarz is Jacobi;
the Kuhn mesh gives every interior vertex 14 edges, so an interior P2 patch holds 15 dofs and every free dof is
covered once per vertex of its entity; the local matrix of a patch is the element matrices of the star's cells
summed over the patch dofs (a different construction from the submatrix of the global matrix); additive
Schwarz with exact local solves is SPD with 1 <= lambda_max(M^-1 A) <= the colouring number of the patch
coupling graph.
"""
import numpy as np
import pytest

from oracle import fe_oracle as O
import fe_inputs as I


def test_p1_star_patches_are_jacobi():
    L = O.Level(3, 1, I.grf_kappa(O.Mesh(3).centroids(), seed=1))
    M = O.PatchPreconditioner(L)
    r = I.random_vector(L.n, 2)
    assert all(p.size == 1 for p in M.patches)
    assert np.allclose(M(r), r / L.diag, rtol=1e-14, atol=0)


@pytest.mark.parametrize("k,sizes", [(2, (15,)), (3, (1 + 28 + 36,))])
def test_patch_topology(k, sizes):
    """Interior-vertex patches: P2 = vertex + 14 edge midpoints; P3 = vertex + 2 x 14 edge dofs + 36 face dofs
    (the Kuhn mesh has 36 faces around an interior vertex).  Coverage of a free dof = the number of vertices of
    its entity (1 vertex, 2 edge, 3 face)."""
    N = 4
    L = O.Level(N, k)
    pats = O.star_patches(L)
    sp = L.space
    interior_v = [v for v in range(L.mesh.n_vertices)
                  if np.all((L.mesh.coords[v] > 0) & (L.mesh.coords[v] < 1))]
    # the patch of an interior vertex contains its own dof; find it by the vertex's dof
    vdof = sp.cell_dofs[:, :4].ravel()
    vid = L.mesh.cells.ravel()
    dof_of_vertex = np.empty(L.mesh.n_vertices, dtype=np.int64)
    dof_of_vertex[vid] = vdof
    by_vertex_dof = {}
    for p in pats:
        for d in p:
            by_vertex_dof.setdefault(d, []).append(p)
    for v in interior_v[:20]:
        owners = [p for p in by_vertex_dof[dof_of_vertex[v]]]
        assert len(owners) == 1 and owners[0].size in sizes
    cover = np.zeros(L.n, dtype=np.int64)
    for p in pats:
        cover[p] += 1
    free = ~sp.boundary
    # the vertices of a dof's entity are the nonzero barycentrics of its node
    bary = O.ref_node_barycentrics(k)
    nverts = np.zeros(L.n, dtype=np.int64)
    nverts[sp.cell_dofs.ravel()] = np.tile((bary > 0).sum(axis=1), L.mesh.n_cells)
    assert np.array_equal(cover[free], nverts[free])
    assert set(np.unique(cover[free])) == set(range(1, k + 1))


@pytest.mark.parametrize("k", [2, 3])
def test_patch_matrix_is_the_star_element_sum(k):
    N = 2
    kap = I.grf_kappa(O.Mesh(N).centroids(), seed=4)
    L = O.Level(N, k, kap)
    Ae = O.element_stiffness(L.mesh, k, kap)
    bary = O.ref_node_barycentrics(k)
    M = O.PatchPreconditioner(L)
    for v in range(L.mesh.n_vertices):
        cells, locals_ = np.nonzero(L.mesh.cells == v)
        if cells.size == 0:
            continue
        dofs = set()
        for K, a in zip(cells, locals_):
            dofs |= set(L.space.cell_dofs[K, bary[:, a] > 0].tolist())
        dofs = np.array(sorted(d for d in dofs if not L.space.boundary[d]))
        if dofs.size == 0:
            continue
        pos = {d: i for i, d in enumerate(dofs)}
        Ap = np.zeros((dofs.size, dofs.size))
        for K in cells:
            cd = L.space.cell_dofs[K]
            for i in range(cd.size):
                for j in range(cd.size):
                    if cd[i] in pos and cd[j] in pos:
                        Ap[pos[cd[i]], pos[cd[j]]] += Ae[K, i, j]
        assert any(p.size == dofs.size and np.array_equal(p, dofs) for p in M.patches)
        assert np.allclose(Ap, L.A_free[dofs][:, dofs].toarray(), atol=1e-14)


@pytest.mark.parametrize("k", [2, 3])
def test_additive_schwarz_spd_and_spectral_bound(k):
    L = O.Level(2, k, I.grf_kappa(O.Mesh(2).centroids(), seed=7))
    M = O.PatchPreconditioner(L)
    free = np.nonzero(~L.space.boundary)[0]
    n = free.size
    E = np.zeros((L.n, n))
    E[free, np.arange(n)] = 1.0
    Minv = np.stack([M(E[:, j]) for j in range(n)], axis=1)[free]
    assert np.allclose(Minv, Minv.T, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0
    Af = L.A[free][:, free].toarray()
    ev = np.linalg.eigvals(Minv @ Af).real
    # additive Schwarz: lambda_max <= the number of colours of the patch coupling graph <= the largest number of
    # patches coupled to one patch (itself included); exact local solves give lambda_max >= 1
    B = (abs(L.A_free) > 0).astype(np.int64)
    R = np.zeros((len(M.patches), L.n), dtype=np.int64)
    for q, p in enumerate(M.patches):
        R[q, p] = 1
    coupled = ((R @ B.toarray() @ R.T) > 0).sum(axis=1).max()
    assert 1 - 1e-10 <= ev.max() <= coupled + 1e-10
    # the Lanczos estimate used for the Chebyshev interval sees the same largest eigenvalue
    assert abs(O.estimate_lambda_max(L.A, L.diag, 40, prec=M) - ev.max()) < 1e-6 * ev.max()


def test_patch_smoothing_beats_jacobi_in_gmg_pcg():
    N0, nref, k = 2, 2, 2
    errs = {}
    for sm in ("jacobi", "patch"):
        h = O.Hierarchy(N0, nref, k, smoother=sm)
        L = h.fine
        b = O.load_vector(L, I.sin_product_rhs(L.space.coords))
        u, it, hist = O.solve(h, b, rtol=1e-10)
        errs[sm] = it
        assert np.linalg.norm(L.A @ u - b) <= 1e-10 * np.linalg.norm(b)
    assert errs["patch"] < errs["jacobi"], errs


def test_patch_smoothed_full_multigrid_reaches_discretisation_error():
    """The paper's solver (full multigrid, Chebyshev(2) preconditioned by vertex-star patches, direct coarse solve)
    on P3: two V-cycles per level leave an error within 1.2x of the discretisation error (max nodal, against the
    analytic solution); with Jacobi smoothing it stays several times above it."""
    L = O.Level(8, 3)
    X = L.space.coords
    b = O.load_vector(L, I.sin_product_rhs(X))
    e_h = np.abs(O.direct_solve(L, b) - I.sin_product(X)).max()
    err = {}
    for sm in ("patch", "jacobi"):
        h = O.Hierarchy(2, 2, 3, smoother=sm)
        err[sm] = np.abs(h.fmg(b, cycles=2) - I.sin_product(X)).max()
    assert err["patch"] <= 1.2 * e_h, (err, e_h)
    assert err["jacobi"] >= 3 * e_h, (err, e_h)
