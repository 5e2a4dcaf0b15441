"""CPU oracle of the terminal-edge-region polygonal mesher -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.

A thin ctypes wrapper around ``polylla_oracle.c`` (plain sequential C), which
restates the paper's phases: Algorithm 2 (LabelMax, LabelSeed, LabelFrontier),
Algorithm 3 (TraversalTriangulation), Algorithm 4 (PolyConstruction) and
Algorithm 5 (PolygonReparation) driven by Algorithm 1.

Parity status: every routine here is pinned by the CPU tests (hand-built meshes
with exact expected outputs, the k x k grid closed form, brute force on tiny
Delaunay meshes, and invariants).  The choice of tip and of the middle internal
edge in reparation is a reading of the paper (it gives no rule for either) and is
pinned by hand-built tip fans only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polylla_oracle.c")
_HDR = os.path.join(_HERE, "polylla_oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    pass


def build_cmd(out: str = _LIB_PATH, src: str = _SRC) -> list[str]:
    return ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-I", _HERE, "-o", out, src]


def load_variant(src: str, out: str):
    """Compile another copy of the oracle source (e.g. one with a planted mistake,
    for the tests that show the pins catch it) and bind it."""
    subprocess.run(build_cmd(out, src), check=True)
    return _bind(out)


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(build_cmd(tmp), check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    lib = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.oracle_label_max.argtypes = [vp, vp, vp, i64, vp]
    lib.oracle_label_max.restype = ctypes.c_int
    lib.oracle_label_seed.argtypes = [vp, i64, vp, vp, vp]
    lib.oracle_label_seed.restype = ctypes.c_int
    lib.oracle_label_frontier.argtypes = [vp, i64, vp, vp]
    lib.oracle_label_frontier.restype = ctypes.c_int
    lib.oracle_seed_list.argtypes = [vp, i64, vp]
    lib.oracle_seed_list.restype = i64
    lib.oracle_traverse.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp, i64]
    lib.oracle_traverse.restype = i64
    lib.oracle_repair.argtypes = [i64, vp, vp, i64, vp, vp, vp, i64, vp, vp, i64, i64, vp, vp]
    lib.oracle_repair.restype = i64
    lib.oracle_run.argtypes = [vp, i64, vp, vp, i64, vp, vp, vp, vp, vp, vp]
    lib.oracle_run.restype = i64
    lib.oracle_lepp.argtypes = [vp, i64, vp, vp, vp]
    lib.oracle_lepp.restype = i64
    lib.oracle_trivertex.argtypes = [vp, i64, i64, vp]
    lib.oracle_trivertex.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB_PATH)
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _mesh_arrays(mesh):
    xy = np.ascontiguousarray(mesh["xy"], dtype=np.int64)
    tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32).reshape(-1, 3)
    twin = np.ascontiguousarray(mesh["twin"], dtype=np.int32).reshape(-1)
    return xy, tri, twin


def _check(rc):
    if rc < 0:
        raise OracleError(f"oracle error {rc}")
    return rc


def label(mesh, lib=None) -> dict:
    """Algorithm 2: max_edge[m], seed[m], terminal[3m], frontier[3m] (uint8)."""
    lib = lib or _load()
    xy, tri, twin = _mesh_arrays(mesh)
    m = tri.shape[0]
    max_edge = np.zeros(m, np.uint8)
    seed = np.zeros(m, np.uint8)
    terminal = np.zeros(3 * m, np.uint8)
    frontier = np.zeros(3 * m, np.uint8)
    _check(lib.oracle_label_max(_p(xy), _p(tri), _p(twin), m, _p(max_edge)))
    _check(lib.oracle_label_seed(_p(twin), m, _p(max_edge), _p(seed), _p(terminal)))
    _check(lib.oracle_label_frontier(_p(twin), m, _p(max_edge), _p(frontier)))
    return {"max_edge": max_edge, "seed": seed, "terminal": terminal, "frontier": frontier}


def seeds(lab: dict, lib=None) -> np.ndarray:
    lib = lib or _load()
    seed = np.ascontiguousarray(lab["seed"], dtype=np.uint8)
    out = np.zeros(max(seed.shape[0], 1), np.int32)
    ns = lib.oracle_seed_list(_p(seed), seed.shape[0], _p(out))
    return out[:ns].copy()


def lepp(mesh, max_edge: np.ndarray, lib=None):
    """Per triangle the seed of the terminal edge its longest-edge propagation path
    reaches, and the path's length (links).  Returns (region int32[m], depth int32[m])."""
    lib = lib or _load()
    _, tri, twin = _mesh_arrays(mesh)
    m = tri.shape[0]
    max_edge = np.ascontiguousarray(max_edge, dtype=np.uint8)
    region = np.zeros(m, np.int32)
    depth = np.zeros(m, np.int32)
    _check(lib.oracle_lepp(_p(twin), m, _p(max_edge), _p(region), _p(depth)))
    return region, depth


def trivertex(mesh, lib=None) -> np.ndarray:
    """The Trivertex array (Section 2): per vertex the smallest half-edge leaving
    it, or -1 (int64[n])."""
    lib = lib or _load()
    xy, tri, _ = _mesh_arrays(mesh)
    n, m = xy.shape[0], tri.shape[0]
    tv = np.zeros(max(n, 1), np.int64)
    _check(lib.oracle_trivertex(_p(tri), m, n, _p(tv)))
    return tv[:n].copy()


def traverse(mesh, frontier: np.ndarray, seed_list: np.ndarray, lib=None):
    """Algorithm 3: pre-reparation polygons as CSR (off int64[ns+1], vtx int32)."""
    lib = lib or _load()
    _, tri, twin = _mesh_arrays(mesh)
    m = tri.shape[0]
    frontier = np.ascontiguousarray(frontier, dtype=np.uint8)
    seed_list = np.ascontiguousarray(seed_list, dtype=np.int32)
    ns = seed_list.shape[0]
    off = np.zeros(ns + 1, np.int64)
    vtx = np.zeros(max(3 * m, 1), np.int32)
    nv = _check(lib.oracle_traverse(_p(tri), _p(twin), m, _p(frontier), _p(seed_list), ns,
                                    _p(off), _p(vtx), vtx.shape[0]))
    return off, vtx[:nv].copy()


def repair(mesh, frontier: np.ndarray, off: np.ndarray, vtx: np.ndarray, lib=None):
    """Algorithm 5 rounds.  Returns (off, vtx, frontier_after, stats)."""
    lib = lib or _load()
    xy, tri, twin = _mesh_arrays(mesh)
    n, m = xy.shape[0], tri.shape[0]
    fr = np.ascontiguousarray(frontier, dtype=np.uint8).copy()
    off = np.ascontiguousarray(off, dtype=np.int64)
    vtx = np.ascontiguousarray(vtx, dtype=np.int32)
    if vtx.size == 0:
        vtx = np.zeros(1, np.int32)
    np_in = off.shape[0] - 1
    cap_poly = max(m, 1)
    cap_vtx = max(3 * m, 1)
    off_out = np.zeros(cap_poly + 1, np.int64)
    vtx_out = np.zeros(cap_vtx, np.int32)
    np_out = np.zeros(1, np.int64)
    stats = np.zeros(2, np.int64)
    nv = _check(lib.oracle_repair(n, _p(tri), _p(twin), m, _p(fr), _p(off), _p(vtx), np_in,
                                  _p(off_out), _p(vtx_out), cap_poly, cap_vtx, _p(np_out),
                                  _p(stats)))
    k = int(np_out[0])
    return off_out[:k + 1].copy(), vtx_out[:nv].copy(), fr, {"rounds": int(stats[0]),
                                                            "splits": int(stats[1])}


def run(mesh, lib=None) -> dict:
    """Algorithm 1 end to end (all phases in one native call)."""
    lib = lib or _load()
    xy, tri, twin = _mesh_arrays(mesh)
    n, m = xy.shape[0], tri.shape[0]
    max_edge = np.zeros(max(m, 1), np.uint8)
    frontier = np.zeros(max(3 * m, 1), np.uint8)
    off = np.zeros(m + 1, np.int64)
    vtx = np.zeros(max(3 * m, 1), np.int32)
    np_out = np.zeros(1, np.int64)
    stats = np.zeros(2, np.int64)
    nv = _check(lib.oracle_run(_p(xy), n, _p(tri), _p(twin), m, _p(max_edge), _p(frontier),
                               _p(off), _p(vtx), _p(np_out), _p(stats)))
    k = int(np_out[0])
    return {"off": off[:k + 1].copy(), "vtx": vtx[:nv].copy(), "max_edge": max_edge[:m],
            "frontier": frontier[:3 * m], "rounds": int(stats[0]), "splits": int(stats[1])}


def full(mesh, lib=None) -> dict:
    """Every intermediate of Algorithm 1, phase by phase (for parity tests)."""
    lab = label(mesh, lib)
    sl = seeds(lab, lib)
    off0, vtx0 = traverse(mesh, lab["frontier"], sl, lib)
    off1, vtx1, fr1, st = repair(mesh, lab["frontier"], off0, vtx0, lib)
    return {"label": lab, "seeds": sl, "trav_off": off0, "trav_vtx": vtx0,
            "off": off1, "vtx": vtx1, "frontier_final": fr1, **st}
