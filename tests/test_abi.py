"""CPU checks of the boundary: the library builds and loads, exports every
entry point the header declares, and the oracle and the product path share no
code."""
import ast
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2301_01719_gb300")


@pytest.fixture(scope="module")
def built_lib():
    from paper_2301_01719_gb300 import build

    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")
    return build.build()


@pytest.fixture(scope="module")
def built_checked_lib():
    from paper_2301_01719_gb300 import build

    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")
    return build.build(checked=True)


def test_library_exports_every_header_symbol(built_lib):
    from paper_2301_01719_gb300 import _lib

    names = _lib.header_symbols()
    assert len(names) >= 14
    L = ctypes.CDLL(built_lib)
    missing = [s for s in names if not hasattr(L, s)]
    assert not missing, missing
    # and the binding declares a signature for each of them, with the same name
    assert sorted(_lib.SIGNATURES) == names


def test_checked_library_exports_the_same_symbols(built_checked_lib):
    from paper_2301_01719_gb300 import _lib

    assert os.path.basename(built_checked_lib) == "libradtex_checked.so"
    L = ctypes.CDLL(built_checked_lib)
    missing = [s for s in _lib.header_symbols() if not hasattr(L, s)]
    assert not missing, missing
    L.rt_status_string.restype = ctypes.c_char_p
    L.rt_status_string.argtypes = [ctypes.c_int32]
    assert L.rt_status_string(8) == b"a computed texel address fell outside its object (checked build)"


def test_status_strings(built_lib):
    from paper_2301_01719_gb300 import _lib

    L = _lib.lib()
    for s in range(9):
        assert L.rt_status_string(s) != b"unknown status"
    assert L.rt_status_string(0) == b"ok"


def test_header_cites_the_paper():
    with open(os.path.join(ROOT, "include", "radtex.h")) as fh:
        text = fh.read()
    for needle in ("Eq. 1b", "Eq. 3", "Note after Eq. 3", "Section 2", "Eq. 4a", "Eq. 2c"):
        assert needle in text


def _imports(path):
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def _py_files(d):
    for base, _, files in os.walk(d):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_product_never_imports_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in _imports(f), f
    for f in _py_files(os.path.join(ROOT, "synth")):
        assert not ({"oracle", "paper_2301_01719_gb300"} & _imports(f)), f


def test_oracle_never_imports_the_product():
    for f in _py_files(os.path.join(ROOT, "oracle")):
        assert not ({"paper_2301_01719_gb300", "synth"} & _imports(f)), f
    src = open(os.path.join(ROOT, "oracle", "radtex_oracle.c")).read()
    assert not re.search(r'#include\s+"', src), "the oracle includes no project header"


def test_cuda_sources_include_no_oracle_code():
    for base, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            text = open(os.path.join(base, f)).read()
            assert "oracle" not in text.lower(), f
