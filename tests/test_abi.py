"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/*.h declares (no compute calls here)."""
from __future__ import annotations

import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__.cuda_build_module().build()
    from paper_1402_4073_gb300 import _native
    return _native


def test_library_exports_every_declared_symbol(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    declared = native.declared_symbols()
    assert "bm_threshold" in declared and "bm_threshold" in native.SIGNATURES
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, f"declared but not exported: {missing}"
    # every declared entry point has a binding signature, and vice versa
    assert sorted(native.SIGNATURES) == declared


def test_strerror_without_gpu(native):
    lib = native.load()
    for code in range(0, -8, -1):
        assert lib.bm_strerror(code)
    assert lib.bm_strerror(-99) == b"unknown status"


def test_package_imports_and_has_no_cpu_fallback(native):
    import paper_1402_4073_gb300 as bm
    assert os.path.samefile(bm.lib._name, native.LIB_PATH)
    src = open(os.path.join(ROOT, "paper_1402_4073_gb300", "__init__.py")).read()
    assert "oracle" not in src and "datagen" not in src


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_1402_4073_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.c" not in text, f


def test_binding_constants_match_header():
    """Every #define of include/bm.h that the binding mirrors has its value."""
    import re

    import paper_1402_4073_gb300 as bm
    text = open(os.path.join(ROOT, "include", "bm.h")).read()
    defs = {m.group(1): int(m.group(2), 0)
            for m in re.finditer(r"#define\s+(BM_\w+)\s+\(?(-?(?:0x[0-9a-fA-F]+|\d+))u?\)?", text)}
    mirrored = {"BM_N_MAX": bm.BM_N_MAX, "BM_WEIGHT_MAX": bm.BM_WEIGHT_MAX,
                "BM_PATH_AUTO": bm.PATH_AUTO, "BM_PATH_DENSE": bm.PATH_DENSE,
                "BM_PATH_SPARSE": bm.PATH_SPARSE, "BM_PATH_RLE": bm.PATH_RLE,
                "BM_POST_NONE": bm.POST_NONE, "BM_POST_AND": bm.POST_AND,
                "BM_POST_OR": bm.POST_OR, "BM_POST_ANDNOT": bm.POST_ANDNOT,
                "BM_EINVAL": bm.BM_EINVAL, "BM_ERANGE": bm.BM_ERANGE}
    for name, value in mirrored.items():
        assert defs.get(name) == value, (name, defs.get(name), value)
