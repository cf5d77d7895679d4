"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; the Python binding names the same entry points."""
import ctypes
import glob
import os
import re
import subprocess

import paper_1305_3976_gb300 as ib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ib_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1305_3976_gb300 import _build
    path = _build.build()
    L = ctypes.CDLL(path)
    decl = declared_symbols()
    assert {"ib_create_grid", "ib_add_fiber", "ib_step", "ib_read_fields"} <= decl
    missing = [n for n in sorted(decl) if not hasattr(L, n)]
    assert not missing, missing
    assert decl == set(ib.EXPORTS)


def test_error_strings_without_gpu():
    L = ib.lib()
    assert L.ib_error_string(ib.IB_ERR_ARG) == b"invalid argument"
    assert L.ib_error_string(0) == b"ok"
    assert L.ib_kernel_name(0) == b"interp"
    assert L.ib_kernel_name(4) == b"rhs" and L.ib_kernel_name(11) == b""


def test_argument_errors_need_no_gpu():
    # argument checks run before any CUDA call
    L = ib.lib()
    n = (ctypes.c_int * 3)(4, 8, 8)      # n < 8 is rejected
    rc = L.ib_cyclic_solve_lines(0, 3, n, 0, 1.0, ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert rc == ib.IB_ERR_ARG
    d = ib.ib_grid_desc()
    d.dim = 4
    h = ctypes.c_void_p()
    assert L.ib_create_grid(ctypes.byref(d), ctypes.byref(h)) == ib.IB_ERR_ARG
    assert b"dim" in L.ib_last_error()


def test_bad_scheme_is_rejected_without_gpu():
    L = ib.lib()
    d = ib.ib_grid_desc()
    d.dim, d.H, d.rho, d.mu, d.dt, d.chi = 2, 1.0, 1.0, 0.1, 1e-3, 0.6
    d.n[0] = d.n[1] = d.n[2] = 16
    d.scheme = 7
    h = ctypes.c_void_p()
    assert L.ib_create_grid(ctypes.byref(d), ctypes.byref(h)) == ib.IB_ERR_ARG
    assert b"scheme" in L.ib_last_error()


def test_struct_layout_matches_the_header(tmp_path):
    # offsets and sizes of the two structs as a C compiler lays them out
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "ib_gb300.h"\n'
        "#define F(s, m) printf(#s \" \" #m \" %zu\\n\", offsetof(s, m));\n"
        "int main(void) {\n"
        "  F(ib_grid_desc, dim) F(ib_grid_desc, n) F(ib_grid_desc, H) F(ib_grid_desc, rho)\n"
        "  F(ib_grid_desc, mu) F(ib_grid_desc, dt) F(ib_grid_desc, chi) F(ib_grid_desc, precision)\n"
        "  F(ib_grid_desc, kernel) F(ib_grid_desc, rotate_split) F(ib_grid_desc, stream)\n"
        "  F(ib_grid_desc, scheme)\n"
        "  F(ib_diag, volume) F(ib_diag, div_l2) F(ib_diag, div_max) F(ib_diag, kinetic)\n"
        "  F(ib_diag, elastic) F(ib_diag, step)\n"
        '  printf("ib_grid_desc sizeof %zu\\n", sizeof(ib_grid_desc));\n'
        '  printf("ib_diag sizeof %zu\\n", sizeof(ib_diag));\n'
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        s, m, v = line.split()
        cls = getattr(ib, s)
        if m == "sizeof":
            assert ctypes.sizeof(cls) == int(v), line
        else:
            assert getattr(cls, m).offset == int(v), line
