"""The C-ABI library builds, loads without a GPU and exports every function
include/gse.h declares; the Python binding names the same set.  No compute
call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gse_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libgse():
    from paper_2411_04686_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libgse):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(libgse, n)]
    assert not missing, missing


def test_binding_lists_the_header(libgse):
    import paper_2411_04686_gb300 as gse
    assert sorted(gse.EXPORTS) == _declared()


def test_strerror_is_pure(libgse):
    libgse.gse_strerror.restype = ctypes.c_char_p
    assert libgse.gse_strerror(0) == b"ok"
    assert b"Inf" in libgse.gse_strerror(-2)


def test_oracle_is_not_linked_into_the_library(libgse):
    assert not hasattr(libgse, "orc_encode")
    for f in os.listdir(os.path.join(ROOT, "paper_2411_04686_gb300", "csrc")):
        txt = open(os.path.join(ROOT, "paper_2411_04686_gb300", "csrc", f)).read()
        assert "oracle" not in txt.lower(), f
