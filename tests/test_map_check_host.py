"""The library's cell->dof map check (fe_checks.h, run on every level's maps when FE_DEBUG_CHECKS=1) on maps built
from the oracle's function spaces, CPU only: it accepts the tet and cube maps of P1/P2/P3 spaces in the library's
layout ([nd][Cs] rows, Dirichlet dofs encoded as -1 - j, padded cells) and counts every planted fault: a dof out of
range, a Dirichlet flag on a free dof or a missing one, a dof repeated within a cell."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fe_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("mapcheck") / "map_check_host")
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2104_08012_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "map_check_host.cpp"), "-o", out])
    return out


def count_bad(exe, rows, n, bnd):
    nd, C = rows.shape
    Cs = (C + 127) // 128 * 128
    m = np.zeros((nd, Cs), dtype=np.int64)
    m[:, :C] = rows
    text = f"{nd} {C} {Cs} {n} {len(bnd)}\n" + " ".join(map(str, bnd)) + "\n" + " ".join(map(str, m.ravel())) + "\n"
    return int(subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout)


def library_layout(space, cell_dofs):
    bd = space.boundary
    enc = np.where(bd[cell_dofs], -1 - cell_dofs, cell_dofs)
    return np.ascontiguousarray(enc.T)


def cube_dofs(space, k, N):
    L = np.rint(space.coords * k * N).astype(np.int64)
    idx = np.empty((k * N + 1,) * 3, dtype=np.int64)
    idx[L[:, 0], L[:, 1], L[:, 2]] = np.arange(space.n)
    out = []
    for cz in range(N):
        for cy in range(N):
            for cx in range(N):
                out.append([idx[k * cx + a, k * cy + b, k * cz + c]
                            for c in range(k + 1) for b in range(k + 1) for a in range(k + 1)])
    return np.array(out)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_valid_maps_pass_and_planted_faults_are_counted(exe, k):
    N = 3
    s = O.Space(O.Mesh(N), k)
    bnd = np.nonzero(s.boundary)[0]
    for dofs in (s.cell_dofs, cube_dofs(s, k, N)):
        rows = library_layout(s, dofs)
        assert count_bad(exe, rows, s.n, bnd) == 0
        free = int(np.nonzero(~s.boundary[dofs[0]])[0][0])  # a free dof of cell 0
        bad = rows.copy()
        bad[free, 0] = s.n  # out of range
        assert count_bad(exe, bad, s.n, bnd) == 1
        bad = rows.copy()
        bad[free, 0] = -1 - bad[free, 0]  # a free dof flagged Dirichlet
        assert count_bad(exe, bad, s.n, bnd) == 1
        bad = rows.copy()
        dir_rows = np.nonzero(bad[:, 0] < 0)[0]
        bad[dir_rows[0], 0] = -1 - bad[dir_rows[0], 0]  # a Dirichlet dof left unflagged
        assert count_bad(exe, bad, s.n, bnd) == 1
        bad = rows.copy()
        other = (free + 1) % rows.shape[0]
        bad[other, 5] = bad[free, 5]  # a repeated dof in cell 5 (and possibly a wrong flag on it)
        assert count_bad(exe, bad, s.n, bnd) >= 1
