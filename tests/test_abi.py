"""The C-ABI library builds, loads without a GPU and exports every function
include/gse.h declares; the Python binding names the same set, with the same
parameter and return kinds, struct layouts and constants.  No compute call is
made (no GPU needed)."""
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


def _header_src():
    return re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "gse.h")).read(), flags=re.S)


def _c_kind(decl):
    """ctypes kind of one C parameter or return type as gse.h writes it."""
    decl = decl.strip()
    if "*" in decl or re.match(r"(const\s+)?gse_(handle|engine)\b", decl):
        return "ptr"
    base = re.sub(r"\b(const|unsigned)\b", "", decl).split()[0]
    return {"int": "i", "int64_t": "l", "double": "d", "size_t": "L", "void": None}[base]


def _ctypes_kind(t):
    if t is None:
        return None
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    return t._type_


def test_binding_signatures_match_the_header(libgse):
    """Every prototype's parameter kinds (pointer, int, int64_t, double,
    size_t) and return kind equal the ctypes declarations of the binding, so
    no argument is truncated or misread across the ABI."""
    import paper_2411_04686_gb300 as gse
    L = gse.lib()
    protos = re.findall(r"(int|void|size_t|const\s+char\s*\*)\s+(gse_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", _header_src())
    assert sorted(p[1] for p in protos) == _declared()
    for ret, name, params in protos:
        f = getattr(L, name)
        want = [_c_kind(p) for p in params.split(",") if p.strip() and p.strip() != "void"]
        got = [_ctypes_kind(t) for t in f.argtypes]
        assert got == want, (name, got, want)
        want_ret = "ptr" if "char" in ret else _c_kind(ret)
        assert _ctypes_kind(f.restype) == want_ret, (name, f.restype, ret)


def test_struct_layouts_match_the_header(tmp_path):
    """gcc compiles a probe against gse.h that prints each field's offset and
    size; the binding's ctypes structures must agree field by field and in total
    size."""
    import shutil
    import subprocess

    import paper_2411_04686_gb300 as gse
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    structs = {"gse_csr": gse.CSR, "gse_step_policy": gse.StepPolicy, "gse_solve_info": gse.SolveInfo,
               "gse_matrix_info": gse.MatrixInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gse.h"', "int main(void) {"]
    for cname, cls in structs.items():
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f"sizeof((({cname}*)0)->{fname}));")
        lines.append(f'printf("{cname} SIZE 0 %zu\\n", sizeof({cname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    seen = 0
    for line in filter(None, out):
        cname, fname, off, size = line.split()
        cls = structs[cname]
        if fname == "SIZE":
            assert ctypes.sizeof(cls) == int(size), cname
        else:
            d = getattr(cls, fname)
            assert (d.offset, d.size) == (int(off), int(size)), (cname, fname)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def test_binding_constants_match_the_header():
    """Status codes, level selectors, policy flags, schedule and index-place
    constants: the binding's values are the header's #defines."""
    import paper_2411_04686_gb300 as gse
    defs = dict(re.findall(r"#define\s+GSE_([A-Z0-9_]+)\s+(-?\d+)", _header_src()))
    assert len(defs) >= 20
    for name, v in defs.items():
        assert getattr(gse, name) == int(v), name


def test_missing_library_fails_loudly(monkeypatch):
    """Without libgse.so every entry of the binding raises: there is no CPU
    fallback for the GSE path."""
    import paper_2411_04686_gb300 as gse
    import synth
    monkeypatch.setattr(gse, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libgse.so"))
    monkeypatch.setattr(gse, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gse.lib()
    with pytest.raises(RuntimeError):
        gse.GseMatrix.from_csr(synth.poisson2d(4))
