"""The build script (no compilation here): the release and the bounds-checked debug variants differ
only by -DDG_BOUNDS_CHECK and their output paths, and both target sm_103a."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build_module():
    spec = importlib.util.spec_from_file_location("dg_build", os.path.join(ROOT, "paper_2111_06767_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_debug_variant_adds_only_the_bounds_check_define():
    b = _build_module()
    rel, dbg = b._flags(), b._flags(debug=True)
    assert "-DDG_BOUNDS_CHECK" not in rel and "-DDG_BOUNDS_CHECK" in dbg
    assert [f for f in dbg if f != "-DDG_BOUNDS_CHECK"] == rel
    assert any("compute_103a" in f and "sm_103a" in f for f in rel)


def test_debug_variant_builds_apart_from_the_release_library():
    b = _build_module()
    assert b.DEBUG_LIB != b.LIB and b.DEBUG_BUILD != b.BUILD
    assert os.path.basename(b.DEBUG_LIB) == "libdg_elliptic_debug.so"
