"""The seeded input generator: valid, exact, deterministic Delaunay meshes.  No GPU."""
from __future__ import annotations

import numpy as np
import pytest

import meshgen


def check_triangulation(mesh, delaunay_brute=False):
    xy = mesh["xy"]
    tri = mesh["tri"].astype(np.int64)
    tw = mesh["twin"].astype(np.int64)
    m, n = tri.shape[0], xy.shape[0]
    p = xy[tri]
    orient = ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
              - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    assert (orient > 0).all(), "triangle not ccw"
    h = np.arange(3 * m)
    org = tri.reshape(-1)
    dst = tri[:, [1, 2, 0]].reshape(-1)
    inner = tw >= 0
    assert (tw[tw[inner]] == h[inner]).all(), "twin not an involution"
    assert (org[tw[inner]] == dst[inner]).all() and (dst[tw[inner]] == org[inner]).all()
    nb = int((~inner).sum())
    edges = (3 * m + nb) // 2
    assert n - edges + m == 1, "Euler characteristic of a disk"
    assert np.unique(tri).size == n, "unused vertex"
    # triangles are ordered by smallest vertex, which comes first
    assert (tri[:, 0] == tri.min(axis=1)).all()
    assert (np.diff(tri[:, 0]) >= 0).all()
    if delaunay_brute:
        pts = [tuple(map(int, q)) for q in xy]
        for t in tri:
            a, b, c = (pts[v] for v in t)
            for d in pts:
                adx, ady = a[0] - d[0], a[1] - d[1]
                bdx, bdy = b[0] - d[0], b[1] - d[1]
                cdx, cdy = c[0] - d[0], c[1] - d[1]
                det = ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy)
                       + (bdx * bdx + bdy * bdy) * (cdx * ady - adx * cdy)
                       + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))
                assert det <= 0, "empty-circle property violated"


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("kind,side", [("uniform", 1 << 20), ("uniform", 24), ("gmm", 1 << 16)])
def test_small_meshes_are_delaunay(kind, side, seed):
    mesh = meshgen.generate(kind, 50, side, seed)
    check_triangulation(mesh, delaunay_brute=True)


def test_degenerate_lattice_grid():
    xy = np.array([(i, j) for j in range(9) for i in range(9)], np.int64)
    mesh = meshgen.delaunay(xy)
    check_triangulation(mesh, delaunay_brute=True)
    assert mesh["tri"].shape[0] == 2 * 8 * 8


def test_collinear_start_and_hull():
    xy = np.array([(0, 0), (1, 1), (2, 2), (3, 3), (5, 1), (1, 5), (4, 4), (6, 6), (7, 7)], np.int64)
    check_triangulation(meshgen.delaunay(xy), delaunay_brute=True)


def test_all_collinear_is_rejected():
    xy = np.array([(i, 2 * i) for i in range(10)], np.int64)
    with pytest.raises(RuntimeError):
        meshgen.delaunay(xy)


def test_points_unique_sorted_and_deterministic():
    a = meshgen.points_gmm(20_000, 1 << 12, 9)  # dense: duplicates are drawn and removed
    b = meshgen.points_gmm(20_000, 1 << 12, 9)
    assert np.array_equal(a, b)
    assert np.unique(a, axis=0).shape[0] == a.shape[0] == 20_000
    assert a.min() >= 0 and a.max() < (1 << 12)
    c = meshgen.points_gmm(20_000, 1 << 12, 10)
    assert not np.array_equal(a, c)


def test_uniform_1k_config():
    mesh = meshgen.load("uniform-1k")
    check_triangulation(mesh, delaunay_brute=False)
    assert mesh["xy"].shape == (1000, 2)
    assert mesh["xy"].max() < (1 << 20)
    assert meshgen.mesh_digest(mesh) == meshgen.mesh_digest(meshgen.load("uniform-1k", cache=False))


def test_shuffled_is_same_triangulation():
    mesh = meshgen.load("uniform-1k")
    sh = meshgen.shuffled(mesh, 3)
    tw = sh["twin"].astype(np.int64)
    tri = sh["tri"]
    inner = tw >= 0
    assert (tw[tw[inner]] == np.arange(tw.size)[inner]).all()
    key = lambda t: tuple(np.roll(t, -int(np.argmin(t))))  # noqa: E731
    assert sorted(map(key, mesh["tri"])) == sorted(map(key, tri))


def test_batch_matches_single():
    ns, seeds, kinds, sides = [300, 1200, 50], [4, 5, 6], [0, 1, 0], [1 << 20, 1 << 22, 1 << 16]
    out = meshgen.batch(ns, seeds, kinds, sides, threads=3)
    for i in range(3):
        single = meshgen.generate("uniform" if kinds[i] == 0 else "gmm", ns[i], sides[i], seeds[i])
        for k in ("xy", "tri", "twin"):
            assert np.array_equal(out[i][k], single[k])
