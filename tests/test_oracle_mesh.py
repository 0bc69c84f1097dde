"""Pins of the oracle's mesh, numbering and quadrature (CPU only).

The mesh, space and numbering follow the paper's UnitCubeMesh / FunctionSpace
(Section 2); the DOF-count identities reproduce the counts quoted in Section 3.
"""
import math
import os

import numpy as np
import pytest

from oracle import fe_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_dof_counts.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()[:2]
            out[k] = int(v)
    return out


def test_config0_sizes():
    m = O.Mesh(8)
    assert m.n_cells == 3072 and m.n_vertices == 729


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_volumes_and_orientation(N):
    m = O.Mesh(N)
    det = np.linalg.det(m.jacobians())
    assert np.allclose(np.abs(det), 1.0 / N ** 3, rtol=0, atol=1e-15)
    assert abs(np.abs(det).sum() / 6.0 - 1.0) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_unique_dofs_match_lattice_count(N, k):
    s = O.Space(O.Mesh(N), k)
    assert np.unique(s.cell_dofs).size == (k * N + 1) ** 3 == s.n
    # numbering is a bijection of the lattice
    assert np.array_equal(np.sort(O.lattice_dof_index(s.dof_lattice, N, k)), np.arange(s.n))
    # boundary dofs: (kN+1)^3 - (kN-1)^3
    assert s.boundary.sum() == (k * N + 1) ** 3 - (k * N - 1) ** 3


def test_p2_vertex_dofs_first():
    m = O.Mesh(3)
    s = O.Space(m, 2)
    assert np.allclose(s.coords[: m.n_vertices], m.coords)
    assert np.array_equal(s.cell_dofs[:, :4], m.cells)


def test_p2_edge_dofs_are_midpoints():
    m = O.Mesh(2)
    s = O.Space(m, 2)
    for e, (a, b) in enumerate(O.P2_EDGES):
        mid = 0.5 * (m.coords[m.cells[:, a]] + m.coords[m.cells[:, b]])
        assert np.allclose(s.coords[s.cell_dofs[:, 4 + e]], mid)


def test_paper_dof_counts():
    g = _golden()
    n = O.dof_count(128, 3)  # degree 3 on the twice-refined 32^3 mesh
    assert abs(n - g["total_dofs_approx"]) / g["total_dofs_approx"] < 0.01
    assert round(n / 512) == g["dofs_per_core_512"]
    n1 = O.dof_count(64, 3)  # MG level 1
    assert abs(n1 / 512 - g["level1_dofs_per_proc_512"]) / g["level1_dofs_per_proc_512"] < 0.01


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_quadrature_exact_on_monomials(n):
    xi, w = O.tet_quadrature(n)
    maxdeg = 2 * n - 3
    for a in range(maxdeg + 1):
        for b in range(maxdeg + 1 - a):
            for c in range(maxdeg + 1 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                assert abs(got - exact) < 1e-15, (a, b, c)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_basis_is_nodal_and_partition_of_unity(k):
    nodes = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    if k == 2:
        nodes = np.concatenate([nodes, [(nodes[a] + nodes[b]) / 2 for a, b in O.P2_EDGES]])
    if k == 3:  # edge nodes at 1/3 and 2/3 (nearer a first), then the face centroids
        edge = [(2 * nodes[a] + nodes[b]) / 3 if h == 0 else (nodes[a] + 2 * nodes[b]) / 3
                for a, b in O.P2_EDGES for h in (0, 1)]
        face = [(nodes[a] + nodes[b] + nodes[c]) / 3 for a, b, c in O.P3_FACES]
        nodes = np.concatenate([nodes, edge, face])
    phi, dphi = O.ref_basis(k, nodes)
    assert np.allclose(phi, np.eye(len(nodes)), atol=1e-15)
    pts = np.random.default_rng(0).dirichlet(np.ones(4), 50)[:, 1:]
    phi, dphi = O.ref_basis(k, pts)
    assert np.allclose(phi.sum(axis=1), 1.0)
    assert np.allclose(dphi.sum(axis=1), 0.0)
    # reference gradients against central differences of the basis values
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (O.ref_basis(k, pts + e)[0] - O.ref_basis(k, pts - e)[0]) / (2 * h)
        assert np.allclose(fd, dphi[:, :, a], atol=1e-8)


def test_p3_nodes_on_the_3n_lattice():
    """P3 (the paper's degree): vertex dofs sit at the mesh vertices, edge dofs at the thirds of the edges
    (nearer the first vertex first), face dofs at the face centroids."""
    m = O.Mesh(2)
    s = O.Space(m, 3)
    assert s.ndof_cell == 20
    P = m.coords[m.cells]  # (C,4,3)
    assert np.allclose(s.coords[s.cell_dofs[:, :4]], P)
    for e, (a, b) in enumerate(O.P2_EDGES):
        assert np.allclose(s.coords[s.cell_dofs[:, 4 + 2 * e]], (2 * P[:, a] + P[:, b]) / 3)
        assert np.allclose(s.coords[s.cell_dofs[:, 5 + 2 * e]], (P[:, a] + 2 * P[:, b]) / 3)
    for f, (a, b, c) in enumerate(O.P3_FACES):
        assert np.allclose(s.coords[s.cell_dofs[:, 16 + f]], (P[:, a] + P[:, b] + P[:, c]) / 3)
