"""The integer P2 stiffness of a Kuhn tet (fe_kuhn.h, compiled for the host) against the oracle, CPU only.

The fixed-point limb operator applies every P2 element of UnitCubeMesh as (kappa h / 120) K120 with one integer
matrix K120 derived in fe_kuhn.h from the basis gradients and the metric M shared by all Kuhn tets.  The oracle
assembles each tet's matrix by quadrature from its own Jacobian, so agreement on all six tet types and at two mesh
sizes pins both the integer matrix and the claim that every Kuhn tet has the same metric.  The properties the
kernel's exactness argument needs (symmetry, divisibility by 4, zero row sums, |K120/4| row sums <= 62) are pinned
here directly as well, and so is the stiffness of two Kuhn tets that share a face (kuhn_pair_k), which the
operator applies as one unit where both tets have the same coefficient.  The compile-time P2 prolongation weights (pro_w8, times 8) are compared entry by entry with
the host stencil tables of fe_stencils.h, which test_transfer_stencils_host.py pins against the oracle's P.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fe_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kuhn_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("kuhn") / "kuhn_host")
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2104_08012_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "kuhn_host.cpp"), "-o", exe])
    return exe


def _matrix(exe, *args):
    out = subprocess.run([exe, *args], capture_output=True, text=True, check=True).stdout
    return np.array([[int(v) for v in line.split()] for line in out.splitlines()], dtype=np.int64)


@pytest.fixture(scope="module")
def k120(kuhn_exe):
    return _matrix(kuhn_exe)


@pytest.fixture(scope="module")
def pair120(kuhn_exe):
    return _matrix(kuhn_exe, "pair")


@pytest.mark.parametrize("N", [1, 2])
def test_k120_is_every_kuhn_element_matrix(k120, N):
    mesh = O.Mesh(N)
    A = O.element_stiffness(mesh, 2)  # (cells, 10, 10), kappa = 1
    h = 1.0 / N
    for c in range(6):  # the six tet types of the first cube
        assert np.allclose(A[c] * 120.0 / h, k120, rtol=0, atol=1e-10), f"tet type {c}"


def test_k120_properties(k120):
    assert np.array_equal(k120, k120.T)
    assert np.all(k120 % 4 == 0)
    K = k120 // 4
    assert np.all(K.sum(axis=1) == 0)
    assert np.abs(K).sum(axis=1).max() == 62
    assert np.count_nonzero(K) == 82


# The second tet's local dofs that are not the first tet's: its vertex 2 and the edges (0,2), (1,2), (2,3).
PAIR_SECOND = (2, 5, 7, 9)


@pytest.mark.parametrize("N", [1, 2])
def test_pair_stiffness_is_two_assembled_kuhn_tets(pair120, N):
    """Cells 6q+2k and 6q+2k+1 (the Kuhn permutations with the same first axis) assembled by the oracle on their
    14 distinct P2 dofs, through the oracle's own global dof numbers, equal the pair matrix (times 120/h), for every
    pair of every cube; this pins both the matrix and which local dofs the two tets share."""
    mesh = O.Mesh(N)
    space = O.Space(mesh, 2)
    A = O.element_stiffness(mesh, 2)
    h = 1.0 / N
    for q in range(N ** 3):
        for k in range(3):
            c1, c2 = 6 * q + 2 * k, 6 * q + 2 * k + 1
            d1, d2 = space.cell_dofs[c1], space.cell_dofs[c2]
            pair_dofs = list(d1) + [d2[j] for j in PAIR_SECOND]
            assert len(set(pair_dofs)) == 14
            pos = {d: n for n, d in enumerate(pair_dofs)}
            M = np.zeros((14, 14))
            for cell, d in ((c1, d1), (c2, d2)):
                for a in range(10):
                    for b in range(10):
                        M[pos[d[a]], pos[d[b]]] += A[cell][a, b]
            assert np.allclose(M * 120.0 / h, pair120, rtol=0, atol=1e-9), (q, k)


def test_pair_stiffness_properties(pair120):
    assert np.array_equal(pair120, pair120.T)
    K = pair120 // 4
    assert np.all(pair120 % 4 == 0) and np.all(K.sum(axis=1) == 0)
    assert np.abs(K).sum(axis=1).max() == 124  # below 127: 127 * 2^17 < 2^24 keeps the limb sums exact
    assert np.count_nonzero(K) == 136


def test_limb_sums_exact_at_the_worst_case(kuhn_exe):
    """The operator's exactness argument, run in FP32 on the host: every row of K and of the pair matrix, summed by
    single-precision FMAs in column order over limbs of the largest magnitude with odd unit counts and the row's signs
    (A_j = +-(2 - 2^-16), B_j = +-(2^-17 + 2^-22 + 2^-33)), equals the exact integer sum; the largest |sum A| is
    124 (2^17 - 1) units of 2^-16, below 2^24.  (With the coefficients' magnitudes raised so that rows exceed 127 the
    same check reports inexact rows.)"""
    inexact, max_a, max_b = (int(v) for v in subprocess.run([kuhn_exe, "limbs"], capture_output=True, text=True,
                                                             check=True).stdout.split())
    assert inexact == 0
    assert max_a == 124 * (2 ** 17 - 1) and max_a < 2 ** 24
    assert max_b < 2 ** 24


def test_prolongation_weights_match_the_stencil_tables(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("kuhnpro") / "kuhn_pro_host")
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2104_08012_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "kuhn_pro_host.cpp"), "-o", exe])
    bad, compared, maxsum = (int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                                               check=True).stdout.split())
    assert bad == 0 and compared == 64 * 27 + 61 * 27
    assert maxsum == 16  # the largest sum of |8 w| over one fine point's stencil

