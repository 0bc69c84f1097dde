"""The library's P3 element formula (gradient at the P2 nodes, fe_p3.cuh) compiled for the host and compared with
the oracle's P3 element stiffness matrices (conical Gauss quadrature of the physical basis gradients) on the tets
of a mesh with a random coefficient; and the operation counts the benchmark's rooflines use, counted from the P2
and P3 element formulas themselves.  CPU only: nvcc compiles the headers as host code."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fe_oracle as O
import fe_inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("p3host") / "p3_element_host")
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2104_08012_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "p3_element_host.cu"), "-o", out])
    return out


def test_p3_gradient_form_matches_oracle_element_matrices(exe):
    m = O.Mesh(2)
    kap = I.grf_kappa(m.centroids(), seed=21)
    A = O.element_stiffness(m, 3, kap)  # (C, 20, 20)
    J = m.jacobians()
    det = np.abs(np.linalg.det(J))
    Jinv = np.linalg.inv(J)
    G = np.einsum("cij,ckj->cik", Jinv, Jinv) * (det * kap)[:, None, None]  # kappa |det J| J^-1 J^-T
    g6 = np.stack([G[:, 0, 0], G[:, 0, 1], G[:, 0, 2], G[:, 1, 1], G[:, 1, 2], G[:, 2, 2]], axis=1)
    u = np.random.default_rng(5).uniform(-1, 1, (m.n_cells, 20))
    lines = "\n".join(" ".join(f"{v:.17g}" for v in np.concatenate([g6[c], u[c]])) for c in range(m.n_cells))
    res = subprocess.run([exe], input=lines + "\n", capture_output=True, text=True, check=True)
    y = np.array([[float(t) for t in line.split()] for line in res.stdout.strip().splitlines()])
    ref = np.einsum("cij,cj->ci", A, u)
    scale = np.einsum("cij,cj->ci", np.abs(A), np.abs(u))
    assert y.shape == ref.shape
    assert np.all(np.abs(y - ref) <= 1e-13 * scale), np.max(np.abs(y - ref) / scale)


def test_p3_operation_count_matches_the_benchmark_constant(tmp_path):
    """The operation count the benchmark's P3 roofline uses (ops per tet) is the formula's own: the element run
    once with a tallying arithmetic type."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path / "p3_opcount_host")
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2104_08012_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "p3_opcount_host.cu"), "-o", out])
    add, mul, fma, neg = map(int, subprocess.run([out], capture_output=True, text=True, check=True).stdout.split())
    import bench
    assert add + mul + fma + neg == bench.OPS_PER_CELL_P3 == 677
    assert (add, mul, fma, neg) == (206, 165, 284, 22)


def test_p2_flop_count_matches_the_benchmark_constant(tmp_path):
    """The FP64 flop count of the P2 element formula that the benchmark's roofline for the native FP64 operator uses
    (151 per tet: additions and multiplications, an FMA counting 2) is the formula's own."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path / "p2_opcount_host")
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2104_08012_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "p2_opcount_host.cu"), "-o", out])
    add, mul, neg = map(int, subprocess.run([out], capture_output=True, text=True, check=True).stdout.split())
    import bench
    assert add + mul == bench.FLOPS_PER_CELL_P2_F64 == 151
    assert (add, mul, neg) == (95, 56, 4)
