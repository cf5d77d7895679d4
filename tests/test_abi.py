"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; the Python binding names the same entry points."""
import ctypes
import glob
import os
import re

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
