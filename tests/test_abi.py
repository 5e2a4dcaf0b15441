"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/polylla.h declares.  Host-only calls only (no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import paper_2204_05438_gb300 as pg
from paper_2204_05438_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polylla.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(polylla_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return ctypes.CDLL(pbuild.LIB)


def test_header_declares_the_pipeline():
    names = declared_functions()
    for required in ("polylla_mesh_create", "polylla_label", "polylla_seeds", "polylla_traverse",
                     "polylla_repair", "polylla_get_polygons", "polylla_mesh_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_entry_point():
    for n in declared_functions():
        assert hasattr(pg, n[len("polylla_"):]), f"no Python binding for {n}"


def test_status_strings():
    lib = pg.load_library()
    for code, name in pg.STATUS.items():
        assert lib.polylla_status_str(code).decode() == name


def test_argument_errors_need_no_device():
    lib = pg.load_library()
    h = ctypes.c_void_p(123)
    # null output pointer / null inputs / bad sizes are rejected before any CUDA call
    assert lib.polylla_mesh_create(None, 10, None, 10, None, 0, None, None) == 1
    assert lib.polylla_mesh_create(None, 10, None, 10, None, 0, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.polylla_mesh_create(16, 2, 16, 10, 16, 0, None, ctypes.byref(h)) == 1
    assert lib.polylla_mesh_create(16, 10, 16, 10, 16, 8, None, ctypes.byref(h)) == 1
    assert lib.polylla_mesh_create(20, 10, 16, 10, 16, 0, None, ctypes.byref(h)) == 1  # misaligned
    assert lib.polylla_label(None, None) == 1
    # the Neighbor-array entry point: null pointers, an unknown convention, misalignment
    create_nb = lib.polylla_mesh_create_neighbors
    create_nb.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                          ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p,
                          ctypes.c_void_p]
    assert create_nb(None, 10, None, 10, None, 0, 0, None, ctypes.byref(h)) == 1
    assert create_nb(16, 10, 16, 10, 16, 2, 0, None, ctypes.byref(h)) == 1
    assert create_nb(16, 10, 16, 10, 18, 0, 0, None, ctypes.byref(h)) == 1
    assert lib.polylla_get_twin(None, None) == 1
    assert lib.polylla_trivertex(None, None) == 1
    assert lib.polylla_mesh_destroy(None) == 1
    assert lib.polylla_launch_count(None) == -1


def test_size_limits_need_no_device():
    # 3 <= n < 2^30 vertices and 1 <= m < 2^29 triangles: an empty mesh and one past
    # either limit are argument errors before any CUDA call (16 stands in for an
    # aligned device pointer; it is never dereferenced)
    lib = pg.load_library()
    h = ctypes.c_void_p(123)
    for n, m in [(3, 0), (3, -1), (2, 1), ((1 << 30), 1), (3, (1 << 29))]:
        assert lib.polylla_mesh_create(16, n, 16, m, 16, 0, None, ctypes.byref(h)) == 1, (n, m)
        assert h.value is None
        assert lib.polylla_mesh_create_host(n, m, ctypes.byref(h)) == 1, (n, m)
    assert lib.polylla_mesh_footprint((1 << 30) - 1, (1 << 29) - 1, 1) > 0


def test_compiled_for_sm103a_only():
    flags = pbuild.compile_flags()
    assert "arch=compute_103a,code=sm_103a" in flags
    assert sum("arch=" in f for f in flags) == 1


def test_batch_argument_errors_need_no_device():
    lib = pg.load_library()
    b = ctypes.c_void_p(123)
    assert lib.polylla_batch_create(None, None, None, None, None, 1, 0, None, None) == 1
    assert lib.polylla_batch_create(None, None, None, None, None, 1, 0, None, ctypes.byref(b)) == 1
    assert b.value is None
    assert lib.polylla_batch_create(16, 16, 16, 16, 16, 0, 0, None, ctypes.byref(b)) == 1
    assert lib.polylla_batch_create(16, 16, 16, 16, 16, 2, 8, None, ctypes.byref(b)) == 1
    assert lib.polylla_batch_create(20, 16, 16, 16, 16, 2, 0, None, ctypes.byref(b)) == 1
    assert lib.polylla_batch_run(None, 0, None) == 1
    assert lib.polylla_batch_tune(None, 1, None, None, None) == 1
    assert lib.polylla_batch_destroy(None) == 1
    k = lib.polylla_batch_schedules()
    assert k >= 2
    cap, thr, ovl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    for s in range(k):
        assert lib.polylla_batch_schedule_info(s, ctypes.byref(cap), ctypes.byref(thr),
                                               ctypes.byref(ovl)) == 0
        assert cap.value in (16, 32, 48, 64) and thr.value in (0, 1, 2) and ovl.value in (0, 1)
    assert lib.polylla_batch_schedule_info(k, ctypes.byref(cap), ctypes.byref(thr), None) == 1
    assert lib.polylla_batch_schedule_info(-1, None, None, None) == 1


def test_server_argument_errors_need_no_device():
    lib = pg.load_library()
    assert lib.polylla_server_cancel(None, 1) == 1
    assert pg.status_str(8) == "POLYLLA_ERR_CANCELLED"
    pg.debug_fail_alloc(0)  # off: no effect
    s = ctypes.c_void_p(123)
    assert lib.polylla_server_create(1 << 30, 4, None) == 1
    assert lib.polylla_server_create(10, 4, ctypes.byref(s)) == 1
    assert s.value is None
    assert lib.polylla_server_create(1 << 30, 0, ctypes.byref(s)) == 1
    rid = ctypes.c_int64()
    assert lib.polylla_server_submit(None, None, 3, None, None, 1, None, None, ctypes.byref(rid)) == 1
    assert lib.polylla_server_poll(None, None, 1, 0) == -1
    assert lib.polylla_server_info(None, None) == 1
    assert lib.polylla_server_destroy(None) == 1
    assert lib.polylla_mesh_footprint(2, 1, 0) == -1
    a = lib.polylla_mesh_footprint(1000, 2000, 0)
    b = lib.polylla_mesh_footprint(1000, 2000, 1)
    # owned inputs: xy, tri, twin and the twin construction's scratch
    assert 0 < a < b and b - a == 16 * 1000 + 24 * 2000 + 8 * 1000 + 4 + 24 * 2000
