"""Seeded synthetic inputs: lattice point sets and their exact Delaunay triangulation.

This module produces inputs only and holds none of the mesher's arithmetic.  It is
shared by the CUDA path (library, bench) and by the CPU oracle (tests).

The workloads stand in for the paper's inputs (Section 4: random points in a
square, triangulated by an external Delaunay program).  Each configuration draws
its points with SplitMix64 from a fixed seed, snaps them to an integer lattice,
deduplicates them and triangulates them exactly (see ``meshgen.cpp``):

* ``uniform-1k``  : 1,000 points uniform on [0, 2^20)^2, seed 0
* ``uniform-1m``  : 1,000,000 points uniform on [0, 2^24)^2, seed 1
* ``gmm16-10m``   : 10,000,000 points from a 16-component equal-weight Gaussian
  mixture (sigma uniform in [0.5%, 5%] of the side, means uniform) snapped to
  [0, 2^26)^2, seed 2; draws outside the square are rejected.

A mesh is a dict of numpy arrays: ``xy`` int64[n, 2], ``tri`` int32[m, 3] (ccw),
``twin`` int32[3m] (opposite half-edge of half-edge 3t+k, or -1 on the hull).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "meshgen.cpp")
_LIB_PATH = os.path.join(_HERE, "libmeshgen.so")
_CACHE = os.path.join(os.path.dirname(_HERE), "_cache", "meshes")
_lock = threading.Lock()
_lib = None

CONFIGS = {
    "uniform-1k": dict(kind="uniform", n=1_000, side=1 << 20, seed=0),
    "uniform-1m": dict(kind="uniform", n=1_000_000, side=1 << 24, seed=1),
    "gmm16-10m": dict(kind="gmm", n=10_000_000, side=1 << 26, seed=2),
    # half-size case of the same distribution, for profiler captures
    "gmm16-5m": dict(kind="gmm", n=5_000_000, side=1 << 26, seed=2),
}


def build_cmd(out: str = _LIB_PATH) -> list[str]:
    return ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
            "-o", out, _SRC]


def build(force: bool = False) -> str:
    """Compile the generator (host C++, no architecture-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(build_cmd(tmp), check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, u64, i32, dbl, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.mg_points_uniform.argtypes = [u64, i64, i64, vp]
            lib.mg_points_uniform.restype = i64
            lib.mg_points_gmm.argtypes = [u64, i64, i32, i64, dbl, dbl, vp]
            lib.mg_points_gmm.restype = i64
            lib.mg_delaunay.argtypes = [vp, i64, vp, vp, i64]
            lib.mg_delaunay.restype = i64
            lib.mg_batch.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32]
            lib.mg_batch.restype = i64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def points_uniform(n: int, side: int, seed: int) -> np.ndarray:
    lib = _load()
    xy = np.empty((n, 2), dtype=np.int64)
    got = lib.mg_points_uniform(seed, n, side, _ptr(xy))
    if got != n:
        raise RuntimeError(f"mg_points_uniform failed ({got})")
    return xy


def points_gmm(n: int, side: int, seed: int, ncomp: int = 16, smin: float = 0.005,
               smax: float = 0.05) -> np.ndarray:
    lib = _load()
    xy = np.empty((n, 2), dtype=np.int64)
    got = lib.mg_points_gmm(seed, n, ncomp, side, smin, smax, _ptr(xy))
    if got != n:
        raise RuntimeError(f"mg_points_gmm failed ({got})")
    return xy


def delaunay(xy: np.ndarray) -> dict:
    """Exact Delaunay triangulation of distinct lattice points (coords < 2^28)."""
    lib = _load()
    xy = np.ascontiguousarray(xy, dtype=np.int64)
    n = xy.shape[0]
    cap = max(2 * n, 4)
    tri = np.empty((cap, 3), dtype=np.int32)
    twin = np.empty(3 * cap, dtype=np.int32)
    m = lib.mg_delaunay(_ptr(xy), n, _ptr(tri), _ptr(twin), cap)
    if m < 0:
        raise RuntimeError(f"mg_delaunay failed ({m})")
    return {"xy": xy, "tri": np.ascontiguousarray(tri[:m]), "twin": np.ascontiguousarray(twin[:3 * m])}


def generate(kind: str, n: int, side: int, seed: int) -> dict:
    if kind == "uniform":
        xy = points_uniform(n, side, seed)
    elif kind == "gmm":
        xy = points_gmm(n, side, seed)
    else:
        raise ValueError(kind)
    return delaunay(xy)


def mesh_digest(mesh: dict) -> str:
    h = hashlib.sha256()
    for k in ("xy", "tri", "twin"):
        h.update(np.ascontiguousarray(mesh[k]).tobytes())
    return h.hexdigest()


def load(name: str, cache: bool = True) -> dict:
    """Generate (or read from the on-disk cache) one named configuration."""
    cfg = CONFIGS[name]
    path = os.path.join(_CACHE, f"{name}.npz")
    if cache and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        with np.load(path) as z:
            return {k: z[k] for k in ("xy", "tri", "twin")}
    mesh = generate(cfg["kind"], cfg["n"], cfg["side"], cfg["seed"])
    if cache:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, **mesh)
        os.replace(tmp, path)
    return mesh


def shuffled(mesh: dict, seed: int) -> dict:
    """Same triangulation with triangles in random order (a locality stress case)."""
    rng = np.random.default_rng(seed)
    m = mesh["tri"].shape[0]
    perm = rng.permutation(m)             # new id j holds old triangle perm[j]
    inv = np.empty(m, dtype=np.int64)
    inv[perm] = np.arange(m)
    tri = mesh["tri"][perm]
    tw_old = mesh["twin"].reshape(m, 3)[perm].reshape(-1).astype(np.int64)
    tw = np.where(tw_old >= 0, 3 * inv[np.maximum(tw_old, 0) // 3] + np.maximum(tw_old, 0) % 3, -1)
    return {"xy": mesh["xy"], "tri": np.ascontiguousarray(tri),
            "twin": np.ascontiguousarray(tw.astype(np.int32))}


def batch(ns, seeds, kinds, sides, threads: int | None = None) -> list[dict]:
    """Generate many meshes in parallel on the host cores."""
    lib = _load()
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    count = ns.shape[0]
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    kinds = np.ascontiguousarray(kinds, dtype=np.int32)
    sides = np.ascontiguousarray(sides, dtype=np.int64)
    vtx_off = np.zeros(count + 1, dtype=np.int64)
    vtx_off[1:] = np.cumsum(ns)
    xy = np.empty((int(vtx_off[-1]), 2), dtype=np.int64)
    cap = 2 * int(vtx_off[-1])
    tri = np.empty((cap, 3), dtype=np.int32)
    twin = np.empty(3 * cap, dtype=np.int32)
    tcount = np.zeros(count, dtype=np.int64)
    threads = threads or max(1, os.cpu_count() or 1)
    tot = lib.mg_batch(count, _ptr(ns), _ptr(seeds), _ptr(kinds), _ptr(sides), _ptr(vtx_off),
                       _ptr(xy), _ptr(tri), _ptr(twin), _ptr(tcount), threads)
    if tot < 0:
        raise RuntimeError(f"mg_batch failed ({tot})")
    out = []
    cap_off = 2 * vtx_off
    for i in range(count):
        m = int(tcount[i])
        c0 = int(cap_off[i])
        out.append({"xy": xy[vtx_off[i]:vtx_off[i + 1]],
                    "tri": tri[c0:c0 + m],
                    "twin": twin[3 * c0:3 * c0 + 3 * m]})
    return out


def batch_plan(count: int, seed: int, nmin: int = 200, nmax: int = 200_000,
               side: int = 1 << 22) -> dict:
    """Sizes, seeds and kinds of a batch of meshes: point counts log-uniform in
    [nmin, nmax], uniform or 16-component Gaussian mixture per mesh, all drawn from
    one seeded generator (numpy's PCG64 -- a driver of the workload, not of the
    method)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(nmin), np.log(nmax), count)).astype(np.int64)
    ns = np.maximum(ns, 3)
    return {"ns": ns, "seeds": rng.integers(1, 2**63 - 1, count, dtype=np.int64).astype(np.uint64),
            "kinds": rng.integers(0, 2, count).astype(np.int32),
            "sides": np.full(count, side, dtype=np.int64)}


def concat(meshes: list) -> dict:
    """Concatenate meshes for a batch: xy / tri / twin stacked with ids kept local to
    each mesh, and the vertex and triangle offsets (int64, n + 1 entries)."""
    nv = np.array([m["xy"].shape[0] for m in meshes], dtype=np.int64)
    nt = np.array([m["tri"].shape[0] for m in meshes], dtype=np.int64)
    vtx_off = np.zeros(len(meshes) + 1, dtype=np.int64)
    tri_off = np.zeros(len(meshes) + 1, dtype=np.int64)
    vtx_off[1:] = np.cumsum(nv)
    tri_off[1:] = np.cumsum(nt)
    return {"xy": np.ascontiguousarray(np.concatenate([m["xy"] for m in meshes])),
            "tri": np.ascontiguousarray(np.concatenate([m["tri"] for m in meshes])),
            "twin": np.ascontiguousarray(np.concatenate([m["twin"] for m in meshes])),
            "vtx_off": vtx_off, "tri_off": tri_off}


def twin_fast(tri) -> np.ndarray:
    """twin_from_tri by sorting (for large meshes); raises on a directed edge used twice."""
    tri = np.asarray(tri, dtype=np.int64).reshape(-1, 3)
    org = tri.reshape(-1)
    dst = tri[:, [1, 2, 0]].reshape(-1)
    n = int(tri.max()) + 1 if tri.size else 1
    key = org * n + dst
    order = np.argsort(key, kind="stable")
    sk = key[order]
    if sk.size > 1 and np.any(sk[1:] == sk[:-1]):
        raise ValueError("a directed edge is used twice")
    rev = dst * n + org
    pos = np.searchsorted(sk, rev)
    pos = np.minimum(pos, sk.size - 1)
    hit = sk[pos] == rev
    twin = np.full(org.size, -1, dtype=np.int32)
    twin[hit] = order[pos[hit]].astype(np.int32)
    return twin


def carve(mesh: dict, keep) -> dict:
    """The sub-mesh of the triangles whose centroid satisfies keep(cx, cy) (arrays),
    made a manifold domain -- triangles around a vertex where boundaries pinch are
    dropped until none is left -- with unused vertices removed (ids renumbered in
    order) and twins rebuilt.  For non-convex domains and domains with holes."""
    xy = np.asarray(mesh["xy"], dtype=np.int64).reshape(-1, 2)
    tri = np.asarray(mesh["tri"], dtype=np.int64).reshape(-1, 3)
    c = xy[tri].sum(axis=1) / 3.0
    tri = tri[keep(c[:, 0], c[:, 1])]
    for _ in range(64):
        if tri.shape[0] == 0:
            break
        twin = twin_fast(tri)
        org = tri.reshape(-1)
        bnd = org[twin < 0]
        cnt = np.bincount(bnd, minlength=xy.shape[0])
        bad = cnt > 1  # two boundary edges leave the vertex: boundaries pinch there
        if not bad.any():
            break
        tri = tri[~bad[tri].any(axis=1)]
    used = np.zeros(xy.shape[0], dtype=bool)
    used[tri.reshape(-1)] = True
    remap = np.cumsum(used) - 1
    tri2 = remap[tri].astype(np.int32)
    return {"xy": np.ascontiguousarray(xy[used]), "tri": np.ascontiguousarray(tri2),
            "twin": twin_fast(tri2)}


def domain_with_holes(kind: str, n: int, side: int, seed: int, holes: int = 6) -> dict:
    """A non-convex domain with holes: the Delaunay mesh of n seeded points, minus
    an L-shaped notch (the corner x > 0.6 side, y > 0.55 side) and `holes` disks at
    seeded centres (radius 4-9 % of the side)."""
    mesh = generate(kind, n, side, seed)
    rng = np.random.default_rng(seed + 1)
    cx = rng.uniform(0.1, 0.9, holes) * side
    cy = rng.uniform(0.1, 0.9, holes) * side
    r = rng.uniform(0.04, 0.09, holes) * side

    def keep(x, y):
        k = ~((x > 0.6 * side) & (y > 0.55 * side))
        for i in range(holes):
            k &= (x - cx[i]) ** 2 + (y - cy[i]) ** 2 > r[i] ** 2
        return k

    return carve(mesh, keep)


def twin_from_tri(tri) -> np.ndarray:
    """Half-edge twin array of a triangle list (for hand-built meshes).

    Half-edge 3t+k runs from tri[t][k] to tri[t][(k+1)%3]; its twin is the
    half-edge running the other way, or -1 if there is none.  Raises if an edge
    is shared by more than two triangles or used twice in the same direction."""
    tri = np.asarray(tri, dtype=np.int64).reshape(-1, 3)
    m = tri.shape[0]
    org = tri.reshape(-1)
    dst = tri[:, [1, 2, 0]].reshape(-1)
    where = {}
    for h in range(3 * m):
        key = (int(org[h]), int(dst[h]))
        if key in where:
            raise ValueError(f"directed edge {key} used twice")
        where[key] = h
    twin = np.full(3 * m, -1, dtype=np.int32)
    for h in range(3 * m):
        g = where.get((int(dst[h]), int(org[h])))
        if g is not None:
            twin[h] = g
    return twin
