"""Writes repeated_vertex_split.json: a small mesh with a one-tip polygon whose split
edge b -> x ends at a vertex x that the polygon's boundary visits twice (Section
3.2.3: the split edge is the middle internal edge at the tip b; here x is a pinch
vertex of the region).  Such polygons are rare (3 of about 78,000 one-tip polygons
on the 5M-point Gaussian-mixture lattice mesh), so the fixture is cut out of that
mesh: the first such region, its triangles and the ring of triangles around it,
vertices and triangles renumbered in their original order.  Every edge of the region
keeps both of its triangles, so its labels, its polygon and its split are those of
the full mesh.

Inputs: meshgen only; the case is found with the oracle's traversal and reparation.
Run from the repository root:  python tests/golden/meshes/make_repeated_vertex_split.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
sys.path.insert(0, ROOT)
import meshgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "repeated_vertex_split.json")
SOURCE = dict(kind="gmm", n=5_000_000, side=1 << 26, seed=2)


def repeated_end_splits(full) -> list[int]:
    """Traversal polygons with one tip whose split edge's far end x occurs more than
    once in the polygon (x: the vertex after the tip b in the first piece)."""
    to, tv, fo, fv = full["trav_off"], full["trav_vtx"], full["off"], full["vtx"]
    out, j = [], 0
    for k in range(len(to) - 1):
        v = tv[to[k]:to[k + 1]]
        L = len(v)
        tips = [i for i in range(L) if v[i] == v[(i + 2) % L]]
        acc, p = 0, 0
        while True:  # the pieces of polygon k: lengths sum to L + 2 (pieces - 1)
            acc += int(fo[j + p + 1] - fo[j + p])
            p += 1
            if acc == L + 2 * (p - 1):
                break
        if len(tips) == 1 and p == 2:
            b = v[(tips[0] + 1) % L]
            P1, P2 = fv[fo[j]:fo[j + 1]], fv[fo[j + 1]:fo[j + 2]]
            ib = [i for i in range(len(P1)) if P1[i] == b and P1[(i + 1) % len(P1)] in P2]
            x = P1[(ib[0] + 1) % len(P1)]
            if int((v == x).sum()) > 1:
                out.append(k)
        j += p
    return out


def cut(mesh, full, k):
    tri, twin = mesh["tri"], mesh["twin"]
    fr = full["label"]["frontier"]
    t0 = int(full["seeds"][k])
    region, stack = {t0}, [t0]
    while stack:  # triangles of the region: across non-frontier edges
        t = stack.pop()
        for h in range(3 * t, 3 * t + 3):
            if not fr[h] and twin[h] >= 0 and twin[h] // 3 not in region:
                region.add(int(twin[h] // 3))
                stack.append(int(twin[h] // 3))
    ring = {int(twin[h] // 3) for t in region for h in range(3 * t, 3 * t + 3) if twin[h] >= 0}
    keep = np.array(sorted(region | ring), np.int64)
    verts, inv = np.unique(tri[keep].ravel(), return_inverse=True)
    return {"xy": mesh["xy"][verts], "tri": inv.reshape(-1, 3).astype(np.int32)}


def main():
    mesh = meshgen.generate(SOURCE["kind"], SOURCE["n"], SOURCE["side"], SOURCE["seed"])
    full = oracle.full(mesh)
    ks = repeated_end_splits(full)
    sub = cut(mesh, full, ks[0])
    sub["twin"] = meshgen.twin_from_tri(sub["tri"])
    assert repeated_end_splits(oracle.full(sub)), "the cut lost the case"
    with open(OUT, "w") as f:
        json.dump({"cite": "Section 3.2.3 (split at the middle internal edge of a tip); the "
                           "split edge's far end is visited twice by the polygon",
                   "source": dict(SOURCE, polygon=int(ks[0]), cases=len(ks)),
                   "xy": sub["xy"].tolist(), "tri": sub["tri"].tolist()}, f)
    print(f"{OUT}: {len(sub['tri'])} triangles, polygon {ks[0]} of {len(ks)} cases")


if __name__ == "__main__":
    main()
