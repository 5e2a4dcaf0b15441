"""Reading #11's order of splits, two ways (CPU only).

The oracle repairs a polygon as Section 3.2.3 states it, per polygon: the first
piece that has a barrier-edge tip is split at its smallest tip along the middle
internal edge of the tip's fan, and replaced by the piece through the new half-edge
tip->x followed by the other one, until no piece has a tip.  The one-block path of
the GPU library reaches the same polygons another way: it splits all of a polygon's
tips in increasing vertex order, skipping a tip that a smaller tip's split edge ended
on (which removes it), and orders the pieces afterwards as the tree of splits the rule
builds (the smallest tip's split at the root, the piece through tip->x on the left),
by joining the two sides of each split in decreasing tip order.  That rests on two
facts about the rule: a split changes only its own tip's fan and, when x is a tip of
the same piece, removes x; and tips of different pieces never meet.

Here that second form is written out plainly over the oracle's labels and seeds, and
its polygons must equal the oracle's, bit for bit, on a few hundred random meshes and
on the hand-built ones whose tip order matters.  This checks the reading the kernel
uses, independently of any GPU.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import meshgen
import oracle
from meshlib import repeated_vertex_split, spiral_wheel, tip_hub, tip_order_meshes


def nxt(h: int) -> int:
    return h - 2 if h % 3 == 2 else h + 1


def prv(h: int) -> int:
    return h + 2 if h % 3 == 0 else h - 1


def split_by_tip_order(mesh) -> tuple[np.ndarray, np.ndarray]:
    """The final polygons as CSR, from the labels, with the tips of each polygon split
    in increasing vertex order and the pieces ordered by the split tree."""
    tri = np.asarray(mesh["tri"], np.int64).reshape(-1)
    twin = np.asarray(mesh["twin"], np.int64)
    lab = oracle.label(mesh)
    seeds = oracle.seeds(lab)
    front = lab["frontier"].astype(bool).copy()
    H = tri.shape[0]

    def turn(h):  # the next frontier half-edge of the boundary after h
        g = nxt(h)
        for _ in range(H + 1):
            if front[g]:
                return g
            g = nxt(int(twin[g]))
        raise AssertionError("turn did not end")

    def turn_back(q):  # the frontier half-edge whose turn is q
        g = prv(q)
        for _ in range(H + 1):
            if front[g]:
                return g
            g = prv(int(twin[g]))
        raise AssertionError("turn did not end")

    succ = {h: turn(h) for h in range(H) if front[h]}

    def is_tip(h):  # h = a->b ends at a tip b: the boundary comes straight back
        return twin[h] >= 0 and succ[h] == twin[h]

    def cycle(h0):
        out, h = [h0], succ[h0]
        while h != h0:
            out.append(h)
            h = succ[h]
            assert len(out) <= H
        return out

    def canonical(hs):  # from the half-edge with the smallest (origin, id)
        k = min(range(len(hs)), key=lambda i: (tri[hs[i]], hs[i]))
        return [int(tri[h]) for h in hs[k:] + hs[:k]]

    def middle_of_fan(p):  # p = a->b, b a tip: the middle internal edge leaving b
        o0 = int(twin[p])
        fan, o = [], int(twin[prv(o0)])
        while o != o0:
            fan.append(o)
            o = int(twin[prv(o)])
            assert len(fan) <= H
        assert len(fan) >= 2
        return fan[math.ceil(len(fan) / 2) - 1]

    polys = []
    for t in seeds:
        t = int(t)
        entry = next((3 * t + k for k in range(3) if front[3 * t + k]), None)
        if entry is None:
            entry = turn(prv(3 * t))  # the frontier half-edge leaving tri[3t] first met
        hs = cycle(entry)
        tips = sorted((h for h in hs if is_tip(h)), key=lambda h: tri[nxt(h)])
        if not tips:
            polys.append(canonical(hs))
            continue
        chords = []  # (oj, tw) of each split made, in increasing tip order
        for p in tips:
            if not is_tip(p):
                continue  # a smaller tip's split edge ended here
            oj = middle_of_fan(p)
            tw = int(twin[oj])
            q = turn(oj)
            pq = turn_back(q)  # before oj is frontier
            front[oj] = front[tw] = True
            pn = succ[p]
            succ[p], succ[oj], succ[pq], succ[tw] = oj, q, tw, pn
            chords.append((oj, tw))
        # the pieces: cycles through the split edges, named by their smallest one
        chord_set = {h for c in chords for h in c}
        piece_of, pieces = {}, []
        for h0 in sorted(chord_set):
            if h0 in piece_of:
                continue
            hs_p = cycle(h0)
            for h in hs_p:
                if h in chord_set:
                    piece_of[h] = len(pieces)
            pieces.append(canonical(hs_p))
        assert len(pieces) == len(chords) + 1
        # the split tree: the two sides of each split joined, largest tip first
        group = {i: [i] for i in range(len(pieces))}
        root = list(range(len(pieces)))

        def find(i):
            while root[i] != i:
                i = root[i]
            return i
        for oj, tw in reversed(chords):
            a, b = find(piece_of[oj]), find(piece_of[tw])
            assert a != b
            group[a] = group[a] + group.pop(b)
            root[b] = a
        (order,) = group.values()
        polys.extend(pieces[i] for i in order)
    off = np.zeros(len(polys) + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in polys])
    vtx = np.array([v for p in polys for v in p], np.int32)
    return off, vtx


def assert_same(mesh):
    ref = oracle.run(mesh)
    off, vtx = split_by_tip_order(mesh)
    np.testing.assert_array_equal(off, ref["off"])
    np.testing.assert_array_equal(vtx, ref["vtx"])
    return ref


@pytest.mark.parametrize("seed", range(300))
def test_random_meshes(seed):
    rng = np.random.default_rng(500 + seed)
    kind = "gmm" if seed % 2 else "uniform"
    n = int(rng.integers(10, 400))
    side = 1 << int(rng.integers(6, 21))  # small lattices: many equal lengths
    assert_same(meshgen.generate(kind, n, side, 70_000 + seed))


def test_hand_built_meshes():
    splits = 0
    for mesh in tip_order_meshes() + [repeated_vertex_split(), tip_hub(), spiral_wheel(300)]:
        splits += assert_same(mesh)["splits"]
    assert splits >= 12


def test_uniform_1k():
    assert assert_same(meshgen.load("uniform-1k"))["splits"] > 0
