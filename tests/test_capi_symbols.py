"""The C ABI library builds and exports every function include/dg_elliptic.h declares (no GPU calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dg_elliptic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("dg_", "elliptic_")) and n not in ("dg_status",)))


def test_library_exports_every_declared_function():
    import __graft_entry__

    lib_path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 20, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_exactly_the_header():
    from paper_2111_06767_gb300 import _native

    assert sorted(_native.SIGNATURES) == declared_functions()


def test_release_build_has_no_bounds_checks():
    """dg_debug_bounds_check() answers -1 in the release build without touching the GPU."""
    import ctypes

    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2111_06767_gb300", "libdg_elliptic.so"))
    lib.dg_debug_bounds_check.restype = ctypes.c_int32
    assert lib.dg_debug_bounds_check() == -1
