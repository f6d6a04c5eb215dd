"""C-ABI checks that need no GPU: the library builds, loads and exports every
function that include/ladder.h declares; geometry validation happens before
any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_2301_12191_gb300 import build as lbuild
from paper_2301_12191_gb300 import ladder as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "ladder.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:LADDER_API\s+)?(?:ladder_status|void|long|const char\s*\*)\s*\*?\s*(\w+)\s*\(",
                                 src, re.M)))


@pytest.fixture(scope="module")
def lib():
    lbuild.build()
    return ctypes.CDLL(lbuild.LIB)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("ladder_init", "analyze_reference", "analyze_dependent", "fetch_decisions",
              "analyze_independent", "ladder_release_frame", "ladder_destroy", "ladder_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in L.SIGNATURES}
    assert set(_declared_functions()) <= bound


def test_header_is_plain_c_and_links(lib, tmp_path):
    """A C99 program includes the header and links against the library."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text('#include "ladder.h"\n'
                   'int main(void) {\n'
                   '    ladder_t *l = 0;\n'
                   '    ladder_subpel_job job = {0};\n'
                   '    (void)job;\n'
                   '    return ladder_frame_bytes(l) == 0 && ladder_set_mv_predictor(l, 0) != LADDER_OK ? 0 : 1;\n'
                   '}\n')
    exe = tmp_path / "abi"
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                           os.path.join(ROOT, "include"), str(src), lbuild.LIB, "-o", str(exe),
                           "-Wl,-rpath," + os.path.dirname(lbuild.LIB)])
    assert os.path.exists(exe)


def test_version_string(lib):
    lib.ladder_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.ladder_version()


@pytest.mark.parametrize("field,value", [
    ("bit_depth", 12), ("ctu_size", 48), ("ref_search_range", 3), ("ref_search_range", 65),
    ("dep_refine_range", 33), ("satd_mode", 2), ("max_frames", 0), ("ref_rung", 2),
    ("dep_depth_lo", 2), ("dep_use_ref_mv", 3), ("n_rungs", 0),
])
def test_invalid_geometry_is_rejected_before_cuda(lib, field, value):
    rungs = (L.Rung * 2)(L.Rung(640, 360), L.Rung(320, 180))
    g = L.Geometry(2, rungs, 1, 8, 64, 16, 4, 0, 1, 1, 0, 2)
    setattr(g, field, value)
    h = ctypes.c_void_p()
    lib.ladder_init.restype = ctypes.c_int
    lib.ladder_init.argtypes = [ctypes.POINTER(L.Geometry), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    assert lib.ladder_init(ctypes.byref(g), None, ctypes.byref(h)) == -1
    assert not h.value


def test_odd_rung_size_rejected(lib):
    rungs = (L.Rung * 1)(L.Rung(641, 360))
    g = L.Geometry(1, rungs, 0, 8, 64, 16, 4, 0, 1, 1, 0, 2)
    h = ctypes.c_void_p()
    lib.ladder_init.restype = ctypes.c_int
    assert lib.ladder_init(ctypes.byref(g), None, ctypes.byref(h)) == -1


def test_null_handles_are_refused_without_touching_a_device():
    """Every entry point that takes a handle refuses NULL with LADDER_E_INVAL
    (and the size queries answer 0) before any CUDA call."""
    lib = L.load()
    E_INVAL = -1
    assert lib.ladder_set_mv_predictor(None, 0) == E_INVAL
    assert lib.ladder_set_parents(None, None) == E_INVAL
    assert lib.ladder_subpel_workspace_bytes(None, 0) == 0
    assert lib.ladder_frame_bytes(None) == 0
    assert lib.ladder_refine_subpel_batch(None, 1, None, None) == E_INVAL
    assert lib.ladder_decide_qps(None, 0, 0, 1, None, None, None) == E_INVAL
    out = ctypes.c_void_p()
    assert lib.ladder_pipeline_create(None, 2, 0, 1024, None, None, None, ctypes.byref(out)) == E_INVAL
    assert lib.ladder_pipeline_submit(None, None, 27, None, None) == E_INVAL
    assert lib.ladder_pipeline_wait(None, 0) == E_INVAL
    lib.ladder_pipeline_destroy(None)
    lib.ladder_destroy(None)


def test_debug_build_compiles_the_bounds_checks_in():
    """libladder_debug.so (the same sources with LADDER_BOUNDS_CHECK=1) says
    so in its version string and exports every symbol the header declares."""
    import ctypes
    from paper_2301_12191_gb300 import build as B
    B.build(debug=True)
    lib = ctypes.CDLL(B.LIB_DEBUG)
    lib.ladder_version.restype = ctypes.c_char_p
    assert b"bounds-checked" in lib.ladder_version()
    rel = ctypes.CDLL(B.LIB)
    rel.ladder_version.restype = ctypes.c_char_p
    assert b"bounds-checked" not in rel.ladder_version()
    for name in _declared_functions():
        getattr(lib, name)
