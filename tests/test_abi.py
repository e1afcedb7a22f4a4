"""The C-ABI library loads and exports every entry point include/wilson.h
declares; host-side argument checks reject bad input before any GPU work.
Runs without a GPU (no compute call is made)."""
import ctypes
import os
import re

from paper_1811_00893_gb300 import wilson

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "wilson.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    # a type, then whitespace or a '*', then the function name and '(' (a
    # function-pointer member such as "int (*f)(...)" is not a declaration)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:\w+\s+)*\w+(?:\s+|\s*\*\s*)(\w+)\s*\(", src, flags=re.M))
                  - {"if", "while", "for", "return", "sizeof"})


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("wilson_dslash", "wilson_mult", "wilson_solve", "wl_gauge_create"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = wilson.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(declared_functions()) <= set(wilson.exported_symbols())


def test_rejects_bad_lattices_without_gpu_work():
    lib = wilson.load()
    g = ctypes.c_void_p()
    for dims, bc in [((3, 4, 4, 4), (1, 1, 1, -1)), ((4, 4, 0, 4), (1, 1, 1, -1)),
                     ((4, 4, 4, 4), (1, 1, 1, -0.5))]:
        lat = wilson.lattice(dims, 0.12, bc)
        rc = lib.wl_gauge_create(ctypes.byref(g), ctypes.byref(lat), ctypes.c_void_p(16), 7, None)
        assert rc == wilson.WL_ERR_ARG
        assert wilson.wl_last_error()


def test_null_handles_rejected():
    lib = wilson.load()
    assert lib.wilson_dslash(None, None, None, 0, 0, 1, 1, None) == wilson.WL_ERR_ARG
    assert lib.wilson_mult(None, None, None, 1, 0, 1, 1, None) == wilson.WL_ERR_ARG
    p = wilson.solve_params()
    info = (wilson.wl_solve_info * 1)()
    assert lib.wilson_solve(None, None, None, 1, ctypes.byref(p), info, None) == wilson.WL_ERR_ARG
    assert lib.wl_field_bytes(None, 1, 1) == 0
