"""The oracle and the CUDA path are independent (CPU only): no product source imports, includes or names a module
of ``oracle/``, the oracle imports nothing of the product, and the shared input module imports neither."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2104_08012_gb300")


def sources(folder, exts):
    for dirpath, _, files in os.walk(folder):
        if "__pycache__" in dirpath or "_build" in dirpath:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_product_does_not_use_the_oracle():
    for path in sources(PKG, (".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
        src = open(path).read()
        assert not re.search(r"^\s*(import\s+oracle|from\s+oracle)", src, flags=re.M), path
        assert "fe_oracle" not in src, path
        assert not re.search(r'#include\s+"[^"]*oracle', src), path


def test_oracle_does_not_use_the_product():
    for path in sources(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        src = open(path).read()
        assert "paper_2104_08012_gb300" not in src, path
        assert "csrc" not in src and "libfe_gb300" not in src, path


def test_input_module_is_shared_but_imports_neither():
    src = open(os.path.join(ROOT, "fe_inputs.py")).read()
    assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S)
    assert "paper_2104_08012_gb300" not in src
