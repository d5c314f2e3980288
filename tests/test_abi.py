"""CPU checks of the C-ABI boundary: the library builds, loads and exports every
function include/pexp.h declares; the binding's structs match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "pexp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pexp_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1509_04567_gb300 import pexp
    return pexp.lib()


def test_library_exports_every_declared_function(lib):
    names = _header_functions()
    assert "pexp_solve_linear" in names and len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_function():
    from paper_1509_04567_gb300 import pexp
    assert sorted(pexp.EXPORTS) == _header_functions()


def test_struct_layouts_match_header_order():
    from paper_1509_04567_gb300 import pexp
    txt = open(os.path.join(ROOT, "include", "pexp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    for cname, pycls in (("pexp_operator", pexp.Operator), ("pexp_options", pexp.Options), ("pexp_report", pexp.Report)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", txt).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            parts = decl.split()
            names = " ".join(parts[1:]).replace(" ", "").split(",")
            fields += [re.sub(r"\[.*\]", "", nm) for nm in names]
        assert [f[0] for f in pycls._fields_] == fields, cname


def test_status_strings_and_defaults_without_gpu(lib):
    from paper_1509_04567_gb300 import pexp
    assert pexp.status_string(0) == "ok"
    assert "invalid" in pexp.status_string(-1)
    o = pexp.make_options({"P": 8, "n_out": 101})
    assert o.P == 8 and o.restart_len == 20 and o.krylov == pexp.KRYLOV_SAI


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.pexp_create(ctypes.byref(h), 0, None)
    assert rc != 0 and not h.value
