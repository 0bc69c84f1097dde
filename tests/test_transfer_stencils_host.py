"""The library's transfer stencils (fe_stencils.h, host code) against the oracle's prolongation matrix, CPU only.

The oracle builds P by locating every fine node in the coarse mesh and evaluating the coarse basis there; the
library tabulates, per class of fine lattice point inside a coarse cube, the coarse lattice offsets and weights, and
derives the restriction taps from the same entries.  Here the stencils are compiled for the host (g++), expanded over
a coarse 2^3 mesh and compared with the oracle's P (prolongation) and P^T (restriction) entry by entry, for P1, P2
and P3.  Also pinned: the weights are dyadic with small denominators (so the FP32 copies the kernels use are exact),
and no prolongation class exceeds the entry count the prolongation kernel unrolls.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fe_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NC = 2  # coarse mesh size


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("stencils") / "transfer_stencils_host")
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2104_08012_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "host", "transfer_stencils_host.cpp"), "-o", out])
    return out


def stencils(exe, k):
    res = subprocess.run([exe, str(k)], capture_output=True, text=True, check=True)
    pro, rst = {}, {}
    for line in res.stdout.splitlines():
        kind, q, a, b, c, w = line.split()
        (pro if kind == "p" else rst).setdefault(int(q), []).append(((int(a), int(b), int(c)), float(w)))
    return pro, rst


def lattice_index(space, m):
    """Dof of each integer lattice point of the m-lattice, from the dof coordinates."""
    L = np.rint(space.coords * m).astype(np.int64)
    assert np.allclose(L, space.coords * m, atol=1e-12)
    idx = -np.ones((m + 1,) * 3, dtype=np.int64)
    idx[L[:, 0], L[:, 1], L[:, 2]] = np.arange(space.n)
    assert (idx >= 0).all()
    return L, idx


@pytest.mark.parametrize("k", [1, 2, 3])
def test_stencils_reproduce_oracle_prolongation_and_its_transpose(exe, k):
    pro, rst = stencils(exe, k)
    K2 = 2 * k
    assert sorted(pro) == list(range(K2 ** 3))
    c, f = O.Level(NC, k), O.Level(2 * NC, k)
    P = O.prolongation(c, f).toarray()
    Lf, _ = lattice_index(f.space, 2 * k * NC)
    Lc, cidx = lattice_index(c.space, k * NC)
    _, fidx = lattice_index(f.space, 2 * k * NC)
    # prolongation: fine point 2k B + o takes w * coarse(k B + d)
    Pst = np.zeros_like(P)
    for i, xf in enumerate(Lf):
        B, o = xf // K2, xf % K2
        for d, w in pro.get(int(o[0] + K2 * (o[1] + K2 * o[2])), []):
            cl = k * B + np.array(d)
            assert np.all((cl >= 0) & (cl <= k * NC)), (xf, d)
            Pst[i, cidx[tuple(cl)]] += w
    assert np.abs(Pst - P).max() <= 1e-14
    # restriction: coarse point c takes w * fine(2 c + off) from its class's taps, fine points outside skipped
    R = np.zeros_like(P.T)
    for j, xc in enumerate(Lc):
        m = xc % k
        for off, w in rst.get(int(m[0] + k * (m[1] + k * m[2])), []):
            F = 2 * xc + np.array(off)
            if np.all((F >= 0) & (F <= K2 * NC)):
                R[j, fidx[tuple(F)]] += w
    assert np.array_equal(R, Pst.T)


@pytest.mark.parametrize("k,den,bound", [(1, 2, 2), (2, 8, 10), (3, 16, 20)])
def test_weights_are_dyadic_and_stencils_fit_the_kernel(exe, k, den, bound):
    pro, rst = stencils(exe, k)
    ws = np.array([w for ents in pro.values() for _, w in ents])
    assert np.all(ws != 0)
    assert np.array_equal(ws * den, np.rint(ws * den))
    assert np.array_equal(ws.astype(np.float32).astype(np.float64), ws)
    assert max(len(e) for e in pro.values()) <= bound
    # every entry of a class sums to 1 (constants are interpolated exactly)
    for q, ents in pro.items():
        assert sum(w for _, w in ents) == 1.0, q
    # the restriction taps are the prolongation entries regrouped
    assert sorted(w for ents in rst.values() for _, w in ents) == sorted(ws.tolist())
