"""The C ABI library builds, loads and exports every function include/nm.h
declares; host-side argument validation works without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2301_06763_gb300 import build, nm
    build.build()
    return nm.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nm_plan", "nm_plan_ex", "nm_green", "nm_potential", "nm_potential_host",
                     "nm_workspace_bytes", "nm_batch_potential", "nm_get_green_octant",
                     "nm_destroy", "nm_status_string", "nm_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_2301_06763_gb300 import nm
    assert nm.status_string(0) == "NM_OK"
    assert nm.status_string(5) == "NM_EUNSUPPORTED"


@pytest.mark.parametrize("levels,N,dx0,code", [
    (0, 16, 0.1, 1), (17, 16, 0.1, 1), (2, 6, 0.1, 1), (2, 2, 0.1, 1),
    (2, 12, 0.1, 5), (2, 512, 0.1, 5), (2, 16, 0.0, 1), (2, 16, float("nan"), 1),
    (2, 16, -1.0, 1)])
def test_plan_rejects_bad_geometry_before_touching_the_device(lib, levels, N, dx0, code):
    from paper_2301_06763_gb300 import nm
    h = ctypes.c_void_p()
    st = lib.nm_plan(levels, N, dx0, ctypes.byref(h))
    assert st == code
    assert h.value is None
    assert len(nm.last_error()) > 0


def test_null_arguments(lib):
    assert lib.nm_plan_ex(None, None) == 1
    assert lib.nm_potential(None, None, None, None) == 1
    assert lib.nm_acceleration(None, None, None, None) == 1
    assert lib.nm_acceleration_ex(None, None, None, 1, 32, None) == 1
    assert lib.nm_destroy(None) == 1
    assert lib.nm_batch_potential(-1, None, None, None, None) == 1
    o = __import__("paper_2301_06763_gb300.nm", fromlist=["Options"]).Options()
    lib.nm_default_options(3, 16, 0.5, ctypes.byref(o))
    assert (o.levels, o.N, o.dx0, o.G, o.precision, o.method) == (3, 16, 0.5, 1.0, 0, 0)
    o.precision = 7
    h = ctypes.c_void_p()
    assert lib.nm_plan_ex(ctypes.byref(o), ctypes.byref(h)) == 1


def test_bad_interp_rejected_before_the_device(lib):
    from paper_2301_06763_gb300 import nm
    o = nm.make_options(2, 8, 0.1, interp="diagonal")
    o.interp = 9
    assert lib.nm_potential_noalloc(ctypes.byref(o), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 1
    h = ctypes.c_void_p()
    assert lib.nm_plan_ex(ctypes.byref(o), ctypes.byref(h)) == 1
