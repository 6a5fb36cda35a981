"""The C-ABI library builds, loads and exports every symbol include/cbcttf.h declares;
argument validation that happens before any device work is checked without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cbcttf.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1008_2042_gb300 import build
    import paper_1008_2042_gb300 as cb
    build.build()
    return cb.load_library()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cbct_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cbct_geometry_create", "cbct_geometry_destroy", "cbct_project",
                     "cbct_backproject", "cbct_tf_analyze", "cbct_tf_synthesize_shrink",
                     "cbct_reconstruct", "cbct_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_launch_counter(lib):
    import paper_1008_2042_gb300 as cb
    assert "sm_103a" in cb.version()
    assert cb.launch_count() >= 0


def _desc(**kw):
    import paper_1008_2042_gb300 as cb
    base = dict(nx=8, ny=8, nz=4, dx=1.0, dy=1.0, dz=1.0, nu=16, nv=8, du=1.0, dv=1.0,
                u_off=0.0, v_off=0.0, sad=1000.0, sdd=1500.0, n_views=4, angles=None)
    base.update(kw)
    return cb.GeometryDesc(**base)


@pytest.mark.parametrize("bad", [dict(nx=0), dict(dz=-1.0), dict(sdd=900.0), dict(n_views=0),
                                 dict(nv=9000), dict(nx=4000, dx=1.0), dict(nx=4000, ny=4500, dx=0.01, dy=0.01), dict(du=float("nan"))])
def test_invalid_geometry_is_rejected_before_device_work(lib, bad):
    d = _desc(**bad)
    h = ctypes.c_void_p()
    st = lib.cbct_geometry_create(ctypes.byref(d), ctypes.byref(h))
    assert st == 1  # CBCT_ERR_INVALID_ARG
    assert not h.value
    assert lib.cbct_last_error()


@pytest.mark.parametrize("nx,ny,nz,ok", [(512, 512, 1024, True), (64, 3742, 1024, True), (64, 3743, 1024, False),
                                         (64, 4032, 990, True), (64, 4032, 991, False)])
def test_grids_beyond_the_projectors_shared_memory_are_unsupported(lib, nx, ny, nz, ok):
    """Largest grids: accepted up to the projector's shared-memory limit, UNSUPPORTED past
    it, before any device work (ok=True cases stop at the device allocation here)."""
    d = _desc(nx=nx, ny=ny, nz=nz, dx=0.2, dy=0.2, dz=0.1)
    h = ctypes.c_void_p()
    st = lib.cbct_geometry_create(ctypes.byref(d), ctypes.byref(h))
    if ok:
        assert st != 5, lib.cbct_last_error()
        if st == 0:
            lib.cbct_geometry_destroy(h)
    else:
        assert st == 5
        assert b"shared memory" in lib.cbct_last_error()


def test_null_arguments_are_rejected(lib):
    assert lib.cbct_geometry_create(None, None) == 1
    assert lib.cbct_project(None, None, None, None) == 1
    assert lib.cbct_backproject(None, None, None, None) == 1
    assert lib.cbct_tf_analyze(4, 4, 4, None, None, None) == 1
    assert lib.cbct_tf_analyze(0, 4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 1
    assert lib.cbct_tf_synthesize_shrink(4, 4, 4, ctypes.c_void_p(16), -1.0, 1, ctypes.c_void_p(16), None) == 1
    it = (ctypes.c_int * 1)(1)
    assert lib.cbct_reconstruct(None, None, 1e-3, 0.0, 1, it, None, None) == 1
    assert lib.cbct_geometry_destroy(None) == 0


def test_typed_entry_points_reject_bad_arguments_before_device_work(lib):
    p = ctypes.c_void_p(16)
    assert lib.cbct_tf_analyze_ex(4, 4, 4, p, p, 3, None) == 1            # unknown storage type
    assert lib.cbct_tf_analyze_ex(4, 4, 4, None, p, 1, None) == 1         # null input
    assert lib.cbct_tf_synthesize_shrink_ex(4, 4, 4, p, -1, 1e-3, 1, p, None) == 1
    assert lib.cbct_tf_synthesize_shrink_ex(4, 4, 4, p, 2, float("nan"), 1, p, None) == 1
    assert lib.cbct_project_ex(None, p, p, 1, None) == 1
    assert lib.cbct_backproject_ex(None, p, 2, p, None) == 1
