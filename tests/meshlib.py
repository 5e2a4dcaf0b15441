"""Test-side helpers: hand-built meshes, golden fixtures, brute-force definitions
and invariant checks.  Independent of both the oracle and the CUDA library.

The brute force here restates the paper's definitions in the most direct form
(Section 3.2.1, Algorithm 2; terminal-edge regions as connected components), with
Python integers and union-find, so that the oracle's walk-based code is checked
against something other than itself.
"""
from __future__ import annotations

import glob
import json
import os

import numpy as np

import meshgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_cases():
    out = []
    for path in sorted(glob.glob(os.path.join(GOLDEN, "*.json"))):
        with open(path) as f:
            case = json.load(f)
        case["name"] = os.path.splitext(os.path.basename(path))[0]
        tri = np.asarray(case["tri"], dtype=np.int32)
        case["mesh"] = {"xy": np.asarray(case["xy"], dtype=np.int64), "tri": tri,
                        "twin": meshgen.twin_from_tri(tri)}
        out.append(case)
    return out


def grid_mesh(k: int, seed: int = 0, step: int = 1):
    """k x k unit cells, one diagonal per cell in a random direction.

    Closed form (each cell's diagonal is the longest edge of both of its
    triangles, every side is the longest edge of neither): k^2 square polygons,
    cell c's seed is its first triangle 2c, the polygon is the cell's four corners
    ccw from the smallest vertex id, and nothing is repaired."""
    rng = np.random.default_rng(seed)
    vid = lambda i, j: j * (k + 1) + i  # noqa: E731
    xy = np.array([(i * step, j * step) for j in range(k + 1) for i in range(k + 1)], np.int64)
    tri, polys = [], []
    for j in range(k):
        for i in range(k):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if rng.integers(2):
                tri += [(a, b, c), (a, c, d)]
            else:
                tri += [(a, b, d), (b, c, d)]
            polys.append([a, b, c, d])  # ccw, a is the smallest id
    tri = np.asarray(tri, np.int32)
    return {"xy": xy, "tri": tri, "twin": meshgen.twin_from_tri(tri)}, polys


def csr_to_lists(off, vtx):
    off = np.asarray(off)
    vtx = np.asarray(vtx)
    return [vtx[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]


# ------------------------------------------------------------------ brute force
def brute_labels(mesh):
    """Longest edge, terminal, frontier and seed flags straight from the definitions."""
    xy = [tuple(map(int, p)) for p in mesh["xy"]]
    tri = [tuple(map(int, t)) for t in mesh["tri"]]
    twin = [int(g) for g in mesh["twin"]]
    m = len(tri)

    def ends(h):
        t, k = divmod(h, 3)
        return tri[t][k], tri[t][(k + 1) % 3]

    def key(h):  # larger key = longer edge
        a, b = ends(h)
        d2 = (xy[a][0] - xy[b][0]) ** 2 + (xy[a][1] - xy[b][1]) ** 2
        eid = h if twin[h] < 0 else min(h, twin[h])
        return (d2, -eid)

    max_edge = [max(range(3), key=lambda k, t=t: key(3 * t + k)) for t in range(m)]
    is_max = [max_edge[h // 3] == h % 3 for h in range(3 * m)]
    terminal = [0] * (3 * m)
    frontier = [0] * (3 * m)
    seed = [0] * m
    for h in range(3 * m):
        g = twin[h]
        if g < 0:
            frontier[h] = 1
            if is_max[h]:
                terminal[h] = 1
                seed[h // 3] = 1
        else:
            if is_max[h] and is_max[g]:
                terminal[h] = 1
                seed[min(h // 3, g // 3)] = 1
            if not is_max[h] and not is_max[g]:
                frontier[h] = 1
    return {"max_edge": max_edge, "terminal": terminal, "frontier": frontier, "seed": seed}


def brute_regions(mesh, frontier):
    """Union-find components of triangles joined across non-frontier edges, and for
    each component the multiset of its frontier half-edges as (origin, dest)."""
    tri = [tuple(map(int, t)) for t in mesh["tri"]]
    twin = [int(g) for g in mesh["twin"]]
    m = len(tri)
    parent = list(range(m))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for h in range(3 * m):
        g = twin[h]
        if g >= 0 and not frontier[h]:
            ra, rb = find(h // 3), find(g // 3)
            if ra != rb:
                parent[ra] = rb
    comp = [find(t) for t in range(m)]
    bnd = {}
    for h in range(3 * m):
        if frontier[h]:
            t, k = divmod(h, 3)
            bnd.setdefault(comp[t], []).append((tri[t][k], tri[t][(k + 1) % 3]))
    return comp, {c: sorted(v) for c, v in bnd.items()}


def lepp_end(mesh, max_edge):
    """Follow each triangle's longest-edge link until a terminal edge: returns the
    terminal edge (as a sorted vertex pair) reached from every triangle."""
    tri = [tuple(map(int, t)) for t in mesh["tri"]]
    twin = [int(g) for g in mesh["twin"]]
    m = len(tri)
    out = []
    for t in range(m):
        cur, steps = t, 0
        while True:
            h = 3 * cur + max_edge[cur]
            g = twin[h]
            if g < 0 or max_edge[g // 3] == g % 3:
                k = max_edge[cur]
                out.append(tuple(sorted((tri[cur][k], tri[cur][(k + 1) % 3]))))
                break
            cur = g // 3
            steps += 1
            assert steps <= m, "longest-edge links form a cycle"
    return out


# ------------------------------------------------------------------ invariants
def twice_area(poly, xy):
    s = 0
    n = len(poly)
    for i in range(n):
        a, b = xy[poly[i]], xy[poly[(i + 1) % n]]
        s += int(a[0]) * int(b[1]) - int(b[0]) * int(a[1])
    return s


def hull_twice_area(xy):
    pts = sorted(set((int(p[0]), int(p[1])) for p in xy))

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in pts:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(pts):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    hull = lower[:-1] + upper[:-1]
    s = 0
    for i in range(len(hull)):
        a, b = hull[i], hull[(i + 1) % len(hull)]
        s += a[0] * b[1] - b[0] * a[1]
    return s


def tips(poly):
    n = len(poly)
    return [poly[(i + 1) % n] for i in range(n) if poly[i] == poly[(i + 2) % n]]


def check_final_mesh(mesh, polys, frontier_final, convex=True, pinch=False):
    """Invariants of the final polygonal mesh (Section 3.2.3's output): every
    polygon simple (with pinch=True: free of barrier-edge tips, since a region that
    touches itself at a vertex keeps that vertex twice), ccw, with positive area; areas add up to the domain's area (the
    triangles' total, which is the hull's for a convex domain); the polygons' edges
    are exactly the frontier edges (each frontier half-edge in exactly one
    polygon); every vertex is used; the Euler characteristic V - E + F is the
    triangulation's (1 for a disk, 1 - h with h holes)."""
    xy = mesh["xy"]
    tri = mesh["tri"]
    n = xy.shape[0]
    tot = 0
    used = set()
    directed = []
    for p in polys:
        assert len(p) >= 3
        if pinch:
            assert all(p[i - 1] != p[(i + 1) % len(p)] for i in range(len(p))), f"tip left: {p}"
        else:
            assert len(set(p)) == len(p), f"polygon not simple: {p}"
        a = twice_area(p, xy)
        assert a > 0, f"polygon not ccw / zero area: {p}"
        tot += a
        used.update(p)
        directed += [(p[i], p[(i + 1) % len(p)]) for i in range(len(p))]
    tri_area = sum(twice_area(list(map(int, t)), xy) for t in tri)
    assert tot == tri_area, "areas do not sum to the domain area"
    if convex:
        assert tot == hull_twice_area(xy), "areas do not sum to the hull area"
    assert used == set(range(n)), "vertex set changed"
    assert len(directed) == len(set(directed)), "a half-edge is in two polygons"
    org = tri.reshape(-1)
    dst = tri[:, [1, 2, 0]].reshape(-1)
    fr = np.asarray(frontier_final).astype(bool)
    expect = sorted(zip(org[fr].tolist(), dst[fr].tolist()))
    assert sorted(directed) == expect, "polygon edges differ from the frontier half-edges"
    undirected = {tuple(sorted(e)) for e in directed}
    tri_edges = {tuple(sorted((int(a), int(b)))) for a, b in zip(org.tolist(), dst.tolist())}
    chi = n - len(tri_edges) + tri.shape[0]
    assert n - len(undirected) + len(polys) == chi, "Euler characteristic"


# ------------------------------------------------------------------ brute-force repair
def brute_final_polygons(mesh):
    """The final polygonal mesh from the definitions, by recursion on triangle sets
    (Section 3.2.3 with readings #9 and #11): a polygon is the boundary of a set of
    triangles joined across non-frontier edges; while a polygon has a barrier-edge
    tip, take the tip with the smallest vertex id, mark the middle internal edge at
    it (the ceil(k/2)-th of the k internal edges met ccw after the barrier edge)
    frontier, split the triangle set into its connected components, and repair the
    component on the tip->x side first, then the other.  Polygons in ascending seed
    order, each from its smallest (origin, half-edge).  Written for tiny meshes: it
    recomputes components after every split instead of tracking rounds."""
    b = brute_labels(mesh)
    fr = list(b["frontier"])
    tri = [tuple(map(int, t)) for t in mesh["tri"]]
    twin = [int(g) for g in mesh["twin"]]
    m = len(tri)

    def nxt(h):
        return 3 * (h // 3) + (h % 3 + 1) % 3

    def prv(h):
        return 3 * (h // 3) + (h % 3 + 2) % 3

    def org(h):
        return tri[h // 3][h % 3]

    def components(tris):
        parent = {t: t for t in tris}

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        for t in tris:
            for k in range(3):
                h = 3 * t + k
                g = twin[h]
                if g >= 0 and not fr[h] and (g // 3) in parent:
                    ra, rb = find(t), find(g // 3)
                    if ra != rb:
                        parent[ra] = rb
        out = {}
        for t in tris:
            out.setdefault(find(t), set()).add(t)
        return list(out.values())

    def boundary_cycle(tris):
        hs = [3 * t + k for t in tris for k in range(3) if fr[3 * t + k]]
        h0 = min(hs, key=lambda h: (org(h), h))
        cyc, h = [], h0
        while True:
            cyc.append(h)
            g = nxt(h)
            while not fr[g]:
                g = nxt(twin[g])
            h = g
            if h == h0:
                break
            assert len(cyc) <= 3 * m
        assert sorted(cyc) == sorted(hs), "a region boundary is not one cycle"
        return cyc

    def repair(tris):
        cyc = boundary_cycle(tris)
        n = len(cyc)
        verts = [org(h) for h in cyc]
        cand = [(verts[i], cyc[(i - 1) % n]) for i in range(n)
                if n > 2 and verts[(i - 1) % n] == verts[(i + 1) % n]]
        if not cand:
            return [verts]
        b_tip, p = min(cand)           # smallest tip vertex; p = a->b
        o0 = twin[p]                   # b->a, the barrier half-edge leaving the tip
        internal, o = [], twin[prv(o0)]
        while o != o0:
            assert not fr[o], "a tip with a second frontier edge"
            internal.append(o)
            o = twin[prv(o)]
        k = len(internal)
        assert k >= 2
        oj = internal[(k + 1) // 2 - 1]  # e_ceil(k/2), 1-based
        fr[oj] = fr[twin[oj]] = 1
        parts = components(tris)
        assert len(parts) == 2
        first = next(p for p in parts if oj // 3 in p)
        second = next(p for p in parts if p is not first)
        return repair(first) + repair(second)

    regions = components(set(range(m)))
    by_tri = {}
    for r in regions:
        for t in r:
            by_tri[t] = r
    polys = []
    for t in range(m):
        if b["seed"][t]:
            polys += repair(by_tri[t])
    return polys, fr


def tip_order_meshes():
    """Meshes on which the order of the tips matters: the polygons differ when the
    largest tip is split first instead of the smallest (found by search over seeded
    generator meshes; the smallest has 25 triangles)."""
    return [meshgen.generate("gmm", 16, 1 << 10, 18 * 7919 + 16),
            meshgen.generate("gmm", 60, 1 << 10, 32 * 7919 + 60),
            meshgen.generate("uniform", 60, 1 << 10, 52 * 7919 + 60)]


# ------------------------------------------------------------------ hand-built regions
def _mesh_from(xy, tri):
    xy = np.asarray(xy, np.int64)
    tri = np.asarray(tri, np.int32)
    return {"xy": xy, "tri": tri, "twin": meshgen.twin_from_tri(tri)}


def spiral_wheel(k: int, radius: int = 1 << 22, step: int = 64, center=(1 << 24, 1 << 24)):
    """A fan of k triangles around one centre vertex (id 0) whose spokes grow
    strictly with the angle (a spiral, rim vertex i at radius radius + i * step).
    The rim is short next to the spokes, so each triangle's longest edge is its
    later spoke: the longest-edge links run around the fan to the last spoke, which
    is the longest of both its triangles (terminal), and the whole fan is one
    terminal-edge region.  The first spoke is the longest of neither of its
    triangles (frontier) with the region on both sides: a barrier edge whose tip is
    the centre (Section 3.2.3).  Traversal gives one polygon of k + 2 vertices with
    one tip; reparation splits it once."""
    ang = 2 * np.pi * np.arange(k) / k
    r = radius + step * np.arange(k)
    rim = np.stack([np.rint(center[0] + r * np.cos(ang)), np.rint(center[1] + r * np.sin(ang))], 1)
    xy = np.concatenate([np.array([center], np.float64), rim]).astype(np.int64)
    i = np.arange(k)
    tri = np.stack([np.zeros(k, np.int64), 1 + i, 1 + (i + 1) % k], 1)
    return _mesh_from(xy, tri)


def tip_hub(n_wheels: int = 9, hub_radius: int = 1 << 22, center=(1 << 24, 1 << 24)):
    """One terminal-edge region with n_wheels + 1 barrier-edge tips and a short
    boundary (6 n_wheels + 2 vertices): a spiral hub of n_wheels triangles around
    vertex 0 (spokes growing by 2 % per step, so the hub's first spoke is a barrier
    edge at the hub centre, as in spiral_wheel) and, glued outside each hub rim
    edge, a small wheel of 5 triangles around its own centre.  A small wheel's
    spokes grow ccw from one end of the hub edge to the other over four 50-degree
    triangles; its fifth triangle is the flat one (about 160 degrees at the centre)
    on the hub edge, whose longest edge is that hub edge.  The hub edge is not the
    longest edge of the hub triangle, so it is internal, the small wheel's links
    run into the hub, and its first spoke is a barrier edge whose tip is the wheel
    centre."""
    c = np.array(center, np.float64)
    ang = 2 * np.pi * np.arange(n_wheels) / n_wheels
    S = hub_radius * (1.0 + 0.02 * np.arange(n_wheels))
    q = c + np.stack([S * np.cos(ang), S * np.sin(ang)], 1)
    q = np.rint(q)
    pts = [c] + list(q)  # 0: hub centre, 1..n: hub rim q_j
    tri = [[0, 1 + j, 1 + (j + 1) % n_wheels] for j in range(n_wheels)]
    for j in range(n_wheels):
        a, b = q[j], q[(j + 1) % n_wheels]  # hub half-edge a -> b, hub on its left
        d = b - a
        e = np.hypot(*d)
        u = d / e
        out = np.array([u[1], -u[0]])  # right of a -> b: outside the hub
        # the centre sees the hub edge under about 160 degrees, a little nearer a
        cw = a + d * 0.47 + out * (0.5 * e / np.tan(np.radians(80.0)))
        r0, r4 = np.hypot(*(a - cw)), np.hypot(*(b - cw))
        a0 = np.arctan2(*(a - cw)[::-1])
        a4 = np.arctan2(*(b - cw)[::-1])
        span = (a4 - a0) % (2 * np.pi)  # ccw from a around the outside to b
        ci = len(pts)
        pts.append(np.rint(cw))
        ids = [1 + j]
        for i in (1, 2, 3):
            th = a0 + span * i / 4
            ri = r0 + (r4 - r0) * i / 4
            ids.append(len(pts))
            pts.append(np.rint(cw + ri * np.array([np.cos(th), np.sin(th)])))
        ids.append(1 + (j + 1) % n_wheels)
        for i in range(4):
            tri.append([ci, ids[i], ids[i + 1]])
        tri.append([ci, ids[4], ids[0]])
    return _mesh_from(np.array(pts), tri)


def disjoint_union(meshes, shift=(1 << 25, 0)):
    """Several meshes side by side in one triangulation (vertex and half-edge ids
    offset, coordinates shifted so the pieces do not overlap)."""
    xy, tri, twin = [], [], []
    nv = nh = 0
    for j, mesh in enumerate(meshes):
        xy.append(mesh["xy"] + np.array([shift[0] * j, shift[1] * j], np.int64))
        tri.append(mesh["tri"] + nv)
        tw = mesh["twin"].copy()
        tw[tw >= 0] += nh
        twin.append(tw)
        nv += mesh["xy"].shape[0]
        nh += 3 * mesh["tri"].shape[0]
    return {"xy": np.concatenate(xy), "tri": np.concatenate(tri).astype(np.int32),
            "twin": np.concatenate(twin).astype(np.int32)}


def neighbors_from_twin(mesh, convention: int = 0) -> np.ndarray:
    """The triangulator's Neighbor array (Section 2) of a mesh, from its twin
    array: entry [t, j] is the triangle across edge j of t, or -1.  Convention 0:
    edge j is opposite vertex j (Triangle's .neigh files), i.e. half-edge
    3t + (j + 1) % 3; convention 1: edge j is half-edge 3t + j."""
    twin = np.asarray(mesh["twin"], np.int64).reshape(-1, 3)
    cross = np.where(twin >= 0, twin // 3, -1)
    if convention == 0:
        cross = cross[:, [1, 2, 0]]
    return np.ascontiguousarray(cross.astype(np.int32))


def repeated_vertex_split():
    """tests/golden/meshes/repeated_vertex_split.json: 43 triangles cut out of a
    Gaussian-mixture lattice mesh (its generator sits beside it), with a one-tip
    polygon whose split edge ends at a vertex the polygon's boundary visits twice."""
    with open(os.path.join(GOLDEN, "meshes", "repeated_vertex_split.json")) as f:
        case = json.load(f)
    tri = np.asarray(case["tri"], dtype=np.int32)
    return _mesh_from(np.asarray(case["xy"], dtype=np.int64), tri)
