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


def _header_defines():
    txt = open(os.path.join(ROOT, "include", "pexp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(PEXP_\w+)\s+(-?\d+)\s*$", txt, re.M)}
    macros = {m.group(1): (m.group(2), m.group(3).strip())
              for m in re.finditer(r"#define\s+(PEXP_\w+)\((\w+)\)\s+(.+)$", txt, re.M)}
    return consts, macros


def test_binding_constants_match_header():
    from paper_1509_04567_gb300 import pexp
    consts, macros = _header_defines()
    for name, value in consts.items():
        short = name[len("PEXP_"):]
        if hasattr(pexp, short):
            assert getattr(pexp, short) == value, name
    for name in ("OK", "ERR_INVALID_ARG", "ERR_NOT_CONVERGED", "ERR_SCRATCH_LIMIT", "DIAG_ORTH", "DIAG_KTIME",
                 "KRYLOV_SAI", "BC_DIRICHLET0", "MIXED", "F32"):
        assert "PEXP_" + name in consts, name
    # kernel-class indices name the entries of KC_NAMES
    for name, value in consts.items():
        if name.startswith("PEXP_KC_") and name != "PEXP_KC_COUNT":
            assert pexp.KC_NAMES[value] == name[len("PEXP_KC_"):].lower(), name
    assert len(pexp.KC_NAMES) == consts["PEXP_KC_COUNT"]
    # the function-like diagnostics macros, evaluated for a few arguments
    for mname, fn in (("PEXP_DIAG_KTIME_CLASS", pexp.DIAG_KTIME_CLASS), ("PEXP_DIAG_KTIME_SAMPLE", pexp.DIAG_KTIME_SAMPLE)):
        arg, body = macros[mname]
        for x in range(8):
            assert eval(re.sub(r"\b%s\b" % arg, str(x), body)) == fn(x), (mname, x)
    # the class and sample fields do not overlap each other or the flag bits
    assert pexp.DIAG_KTIME_CLASS(7) < pexp.DIAG_KTIME_SAMPLE(1)
    assert pexp.DIAG_KTIME_CLASS(0) > (pexp.DIAG_ORTH | pexp.DIAG_KTIME)


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "pexp.h"

int main(void) {
    pexp_options o;
    pexp_report r;
    pexp_operator op;
    pexp_ctx* ctx = NULL;
    memset(&r, 0, sizeof(r));
    memset(&op, 0, sizeof(op));
    pexp_default_options(&o);
    if (o.restart_len != 20 || o.krylov != PEXP_KRYLOV_SAI || o.jacobian != 0 || o.wr_diverge != 3) return 2;
    if (strcmp(pexp_status_string(PEXP_OK), "ok") != 0) return 3;
    if (pexp_solve_linear(ctx, &op, &o, NULL, NULL, PEXP_F64, NULL, PEXP_F64, &r) != PEXP_ERR_INVALID_ARG) return 4;
    printf("%d %d %d %d %d %d\n", o.P, PEXP_DIAG_KTIME | PEXP_DIAG_KTIME_CLASS(PEXP_KC_UPDATE) | PEXP_DIAG_KTIME_SAMPLE(2),
           (int)sizeof(pexp_operator), (int)sizeof(pexp_options), (int)sizeof(pexp_report), (int)sizeof(pexp_problem));
    if (pexp_solve_batched(ctx, 1, NULL, NULL) != PEXP_ERR_INVALID_ARG) return 5;
    return 0;
}
"""


def test_header_is_c99_and_links_from_plain_c(lib, tmp_path):
    """The boundary is a C ABI: a C99 program including only include/pexp.h compiles
    without warnings, links against libpexp.so and calls it (no CUDA call is made:
    the null context is rejected before any)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1509_04567_gb300 import pexp
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(pexp.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-lpexp", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, (run.returncode, run.stderr)
    sizes = [str(ctypes.sizeof(c)) for c in (pexp.Operator, pexp.Options, pexp.Report, pexp.Problem)]
    assert run.stdout.split() == ["1", str(2 | (1 << 11) | (2 << 16))] + sizes


def test_binding_checks_the_series_it_passes():
    """The binding checks, before a solve's pointers go to the library, that y0, G and Y hold
    what a valid solve reads and writes: G has n_out rows, or P (n_samp - 1) + 1 with
    Chebyshev samples; invalid options are left to the library (no buffer check fails)."""
    import numpy as np
    from paper_1509_04567_gb300 import pexp
    op = dict(dim=1, nx=64, ny=1, bc=0, ax=1.0, ay=0.0, nu=1e-2, Lx=1.0, Ly=1.0)
    opts = dict(n_out=9, P=4)
    cheb = dict(n_out=9, P=4, nodes=pexp.NODES_CHEBYSHEV, n_samp=13)
    assert pexp.source_rows(opts) == 9 and pexp.source_rows(cheb) == 49
    y0, Y = np.zeros(64), np.zeros((9, 64))
    pexp._check_series_shapes(op, opts, y0, np.zeros((9, 64)), Y)
    pexp._check_series_shapes(op, cheb, y0, np.zeros((49, 64)), Y)
    pexp._check_series_shapes(op, dict(opts, n_out=1), y0, None, Y)   # invalid: the library says so
    for bad in ((cheb, np.zeros((9, 64)), Y), (opts, np.zeros((9, 32)), Y), (opts, None, np.zeros((8, 64)))):
        with pytest.raises(ValueError):
            pexp._check_series_shapes(op, bad[0], y0, bad[1], bad[2])
    with pytest.raises(ValueError):
        pexp._check_series_shapes(op, opts, np.zeros(63), None, Y)
