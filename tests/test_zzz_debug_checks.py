"""Hierarchies built with FE_DEBUG_CHECKS=1 pass the library's own map checks (fe_checks.h) on the GPU.

The variable is read once per process, so the hierarchies are built in a child process.  Collected last, so that a
failure here cannot hide the other tests.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_checks_accept_the_library_maps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08012_gb300 import build
    build.build()
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import torch, paper_2104_08012_gb300 as fe\n"
        "fe.load()\n"
        "for k in (1, 2, 3):\n"
        "    with fe.Hierarchy(2, 1, k) as h:\n"
        "        x = torch.ones(h.n_dofs(), dtype=torch.float64, device='cuda')\n"
        "        y = torch.empty_like(x)\n"
        "        h.apply_operator(x, y)\n"
        "        torch.cuda.synchronize()\n"
        "print('ok')\n" % ROOT)
    env = dict(os.environ, FE_DEBUG_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]
