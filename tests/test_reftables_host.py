"""The library's reference-element tables (fe_reftables.h, host code) against the oracle, CPU only.

The library tabulates on the host, and uploads to constant memory: the P1/P2 reference mass matrices (closed-form
barycentric monomial integrals), the P3 reference stiffness coefficients and mass matrix (its own P3 basis and a
5-point conical Gauss rule), and the 27-point rule of the quadrature load vector with the P1/P2/P3 basis values at
its points.  Here they are compiled for the host (g++) and compared with the oracle's basis (``ref_basis``) and rule
(``tet_quadrature``), and with properties fixed by the mathematics: the mass matrix sums to the reference volume 1/6,
stiffness rows sum to zero (constants have no gradient), the P3 entries are integers over 3360 (stiffness) and
26880 (mass) as the float-pair kernels assume, and the Gauss-Legendre nodes are numpy's.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fe_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("reftables") / "reftables_host")
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2104_08012_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "host", "reftables_host.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    t = {}
    for line in out.splitlines():
        name, *vals = line.split()
        t[name] = np.array([float(v) for v in vals])
    return t


def ref_mass(k):
    xi, w = O.tet_quadrature(5)  # exact to degree 7
    phi, _ = O.ref_basis(k, xi)
    return np.einsum("q,qi,qj->ij", w, phi, phi)


@pytest.mark.parametrize("k,name", [(1, "m1"), (2, "m2"), (3, "M3")])
def test_reference_mass_matrices(tables, k, name):
    nd = {1: 4, 2: 10, 3: 20}[k]
    M = tables[name].reshape(nd, nd)
    assert np.abs(M - ref_mass(k)).max() <= 1e-15
    assert abs(M.sum() - 1.0 / 6.0) <= 1e-15
    assert np.abs(M - M.T).max() <= 1e-17  # symmetric up to the rounding of the quadrature products


def test_p3_reference_stiffness_coefficients(tables):
    K = tables["K3"].reshape(210, 6)
    xi, w = O.tet_quadrature(5)
    _, d = O.ref_basis(3, xi)  # (q, 20, 3)
    S = np.einsum("q,qia,qjb->abij", w, d, d)
    iu, ju = np.triu_indices(20)
    ref = np.stack([S[0, 0], S[0, 1] + S[1, 0], S[0, 2] + S[2, 0], S[1, 1], S[1, 2] + S[2, 1], S[2, 2]],
                   axis=-1)[iu, ju]
    assert np.abs(K - ref).max() <= 1e-13
    # constants have no gradient: every coefficient's full 20 x 20 matrix has zero row sums
    for c in range(6):
        A = np.zeros((20, 20))
        A[iu, ju] = K[:, c]
        A[ju, iu] = K[:, c]
        assert np.abs(A.sum(axis=1)).max() <= 1e-13


def test_p3_entries_are_small_integers_over_fixed_denominators(tables):
    K = tables["K3"] * 3360
    M = tables["M3"] * 26880
    assert np.abs(K - np.rint(K)).max() < 1e-9 and np.abs(np.rint(K)).max() <= 1944
    assert np.abs(M - np.rint(M)).max() < 1e-9 and np.abs(np.rint(M)).max() <= 432
    # ... so the integers are exact in FP32 (the float-pair mass kernel multiplies by them)
    assert np.array_equal(np.rint(M).astype(np.float32).astype(np.float64), np.rint(M))


def test_load_vector_rule_and_basis_values(tables):
    xi, w = O.tet_quadrature(O.QUAD_N)
    assert np.abs(tables["xi"].reshape(27, 3) - xi).max() <= 1e-16
    assert np.abs(tables["w"] - w).max() <= 1e-15 * w.max()
    for k, name in ((1, "phi1"), (2, "phi2"), (3, "phi3")):
        phi, _ = O.ref_basis(k, xi)
        assert np.abs(tables[name].reshape(27, -1) - phi).max() <= 1e-14, name


def test_gauss_legendre_nodes(tables):
    t, w = np.polynomial.legendre.leggauss(5)  # ascending nodes on [-1, 1]
    order = np.argsort(tables["gl5_t"])
    assert np.abs(tables["gl5_t"][order] - 0.5 * (t + 1)).max() <= 1e-15
    assert np.abs(tables["gl5_w"][order] - 0.5 * w).max() <= 1e-15
