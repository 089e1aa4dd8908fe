"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads without
a GPU, exports every entry point include/rcell.h declares, and the product path
never reaches the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = "".join(open(os.path.join(ROOT, "include", f)).read()
                  for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const\s+char\s*\*)\s*\**\s*(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1902_09171_gb300 import build, rcell
    build.build()
    return rcell.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("rcell_create", "rcell_set_deformation", "rcell_run", "rcell_stress", "fe_step"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_mirrors_the_header():
    from paper_1902_09171_gb300 import rcell, surrogate
    assert sorted(rcell.EXPORTS + surrogate.EXPORTS) == header_functions()
    for name in rcell.EXPORTS:
        assert callable(getattr(rcell, name)), name
    for name in surrogate.EXPORTS:
        assert callable(getattr(surrogate, name)), name


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1902_09171_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, flags=re.M), f
                assert "liboracle" not in src, f
                assert "rcell_oracle" not in src, f


def test_library_built_for_sm103a_only(lib):
    from paper_1902_09171_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path):
    from paper_1902_09171_gb300 import rcell
    saved = rcell._lib
    rcell._lib = None
    try:
        with pytest.raises(RuntimeError):
            rcell.load(str(tmp_path / "absent.so"))
    finally:
        rcell._lib = saved
