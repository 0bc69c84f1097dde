"""The C-ABI library builds, loads and exports every symbol include/fe.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_08012_gb300 import build
    build.build()
    import paper_2104_08012_gb300 as fe
    return fe.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    import paper_2104_08012_gb300 as fe
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        getattr(lib, name)
    assert declared == set(fe.EXPORTED)


def test_calls_without_gpu_fail_loudly(lib):
    import paper_2104_08012_gb300 as fe
    if fe.fe_device_count() > 0:
        pytest.skip("a GPU is present")
    with pytest.raises(fe.FeError) as e:
        fe.Hierarchy(2, 1, 2)
    assert e.value.code == fe.FE_ERR_CUDA


def test_argument_validation(lib):
    import paper_2104_08012_gb300 as fe
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create(2, 3, 4)
    assert e.value.code == fe.FE_ERR_UNSUPPORTED
    with pytest.raises(fe.FeError) as e:
        fe.fe_mesh_create(0)
    assert e.value.code == fe.FE_ERR_ARG
    m = fe.fe_mesh_create(2)
    with pytest.raises(fe.FeError) as e:
        fe.fe_hierarchy_refine(m, 1, 4)
    assert e.value.code == fe.FE_ERR_UNSUPPORTED
    with pytest.raises(fe.FeError) as e:
        fe.fe_hierarchy_refine(m, 9, 1)
    assert e.value.code == fe.FE_ERR_ARG
    fe.fe_mesh_destroy(m)
    assert lib.fe_num_levels(None) == fe.FE_ERR_ARG


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2104_08012_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src), f
