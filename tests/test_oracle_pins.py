"""Pins for the CPU oracle: hand-built cases with expected values written by hand
from the paper's definitions (tests/golden), the k x k grid closed form, brute
force on tiny Delaunay meshes, invariants on larger ones, and planted mistakes
that the pins must catch.  No GPU."""
from __future__ import annotations

import os
import shutil

import numpy as np
import pytest

import meshgen
import oracle
from meshlib import (brute_final_polygons, brute_labels, brute_regions, check_final_mesh,
                     repeated_vertex_split,
                     csr_to_lists, golden_cases, grid_mesh, lepp_end, spiral_wheel, tip_hub,
                     tip_order_meshes, tips)

GOLDEN = golden_cases()


def _halfedges(flags):
    return np.nonzero(np.asarray(flags))[0].tolist()


# --------------------------------------------------------------------- pin suite
def pin_repair_bruteforce(mesh, lib=None):
    """The oracle's final polygons and final frontier against the recursive
    brute-force repair (smallest tip first, middle internal edge, connected
    components after every split)."""
    r = oracle.run(mesh, lib)
    polys, fr = brute_final_polygons(mesh)
    assert csr_to_lists(r["off"], r["vtx"]) == polys
    assert r["frontier"].tolist() == fr


TIP_ORDER = tip_order_meshes()
def pin_golden(case, lib=None):
    e = case["expect"]
    r = oracle.full(case["mesh"], lib)
    lab = r["label"]
    assert lab["max_edge"].tolist() == e["max_edge"]
    assert _halfedges(lab["terminal"]) == e["terminal_halfedges"]
    assert _halfedges(lab["frontier"]) == e["frontier_halfedges"]
    assert r["seeds"].tolist() == e["seeds"]
    assert csr_to_lists(r["trav_off"], r["trav_vtx"]) == e["traverse"]
    assert csr_to_lists(r["off"], r["vtx"]) == e["final"]
    assert r["splits"] == e["splits"]
    added = sorted(set(_halfedges(r["frontier_final"])) - set(e["frontier_halfedges"]))
    assert added == e.get("final_new_frontier_halfedges", [])


def pin_grid(k, seed, lib=None):
    mesh, polys = grid_mesh(k, seed)
    r = oracle.full(mesh, lib)
    m = 2 * k * k
    assert r["seeds"].tolist() == list(range(0, m, 2))
    assert csr_to_lists(r["trav_off"], r["trav_vtx"]) == polys
    assert csr_to_lists(r["off"], r["vtx"]) == polys
    assert r["splits"] == 0
    # the diagonal (local edge 2 of the first and 0 / 1 of the second triangle) is
    # the only non-frontier edge of every cell
    fr = r["label"]["frontier"].reshape(m, 3)
    assert int(fr.sum()) == 3 * m - 2 * k * k


def pin_bruteforce(mesh, lib=None, convex=True, pinch=False):
    r = oracle.full(mesh, lib)
    b = brute_labels(mesh)
    lab = r["label"]
    assert lab["max_edge"].tolist() == b["max_edge"]
    assert lab["terminal"].tolist() == b["terminal"]
    assert lab["frontier"].tolist() == b["frontier"]
    assert lab["seed"].tolist() == b["seed"]
    comp, bnd = brute_regions(mesh, b["frontier"])
    seeds = r["seeds"].tolist()
    # one seed per region, and every region has one
    assert sorted(comp[s] for s in seeds) == sorted(set(comp))
    # each region's longest-edge paths all end at the same terminal edge
    ends = lepp_end(mesh, b["max_edge"])
    for c in set(comp):
        assert len({ends[t] for t in range(len(comp)) if comp[t] == c}) == 1
    polys = csr_to_lists(r["trav_off"], r["trav_vtx"])
    assert len(polys) == len(seeds)
    for s, p in zip(seeds, polys):
        edges = sorted((p[i], p[(i + 1) % len(p)]) for i in range(len(p)))
        assert edges == bnd[comp[s]], "polygon is not the region boundary"
        assert p[0] == min(p), "polygon does not start at its smallest vertex"
    final = csr_to_lists(r["off"], r["vtx"])
    check_final_mesh(mesh, final, r["frontier_final"], convex=convex, pinch=pinch)
    assert len(final) == len(polys) + r["splits"]
    assert len(r["vtx"]) == len(r["trav_vtx"]) + 2 * r["splits"]
    return r


def tiny_meshes(count=60):
    out = []
    for s in range(count):
        n = 4 + s % 9
        side = 16 if s % 3 == 0 else (1 << 12)
        kind = "uniform" if s % 2 == 0 else "gmm"
        if kind == "gmm" and side == 16:
            kind = "uniform"
        out.append(meshgen.generate(kind, n, side, 1000 + s))
    return out


TINY = tiny_meshes()


# --------------------------------------------------------------------- tests
@pytest.mark.parametrize("case", GOLDEN, ids=[c["name"] for c in GOLDEN])
def test_golden(case):
    pin_golden(case)


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (5, 2), (16, 3)])
def test_grid_closed_form(k, seed):
    pin_grid(k, seed)


@pytest.mark.parametrize("idx", range(len(TINY)))
def test_bruteforce_tiny(idx):
    pin_bruteforce(TINY[idx])


@pytest.mark.parametrize("idx", range(len(TIP_ORDER)))
def test_repair_bruteforce_tip_order(idx):
    """Meshes on which splitting the largest tip first gives other polygons: the
    oracle's rounds must give exactly the recursive brute force's polygons."""
    pin_repair_bruteforce(TIP_ORDER[idx])


def test_repair_bruteforce_small():
    for s in range(12):
        pin_repair_bruteforce(meshgen.generate("gmm", 120, 1 << 12, 500 + s))


def test_bruteforce_small_with_tips():
    """Small Delaunay meshes that do have barrier-edge tips: brute-force labels and
    regions, then every final-mesh invariant after reparation."""
    seen = 0
    for s in range(40):
        mesh = meshgen.generate("uniform", 300, 1 << 16, 77 + s)
        r = pin_bruteforce(mesh)
        seen += r["splits"]
    assert seen > 0


@pytest.mark.parametrize("k", [7, 40, 5000])
def test_spiral_wheel_is_one_region_with_one_tip(k):
    """The hand-built fan of spiral_wheel (one region of k triangles, the centre a
    barrier-edge tip): labels, regions and the final polygons from brute force,
    and the traversal polygon of k + 2 vertices with its one tip, split once.  The
    GPU tests rely on these properties to reach the one-thread walk of regions too
    large for a thread block."""
    mesh = spiral_wheel(k)
    if k <= 40:
        pin_bruteforce(mesh, convex=False)
    r = oracle.full(mesh)
    trav = csr_to_lists(r["trav_off"], r["trav_vtx"])
    assert len(trav) == 1 and len(trav[0]) == k + 2
    assert tips(trav[0]) == [0]
    assert r["seeds"].tolist() == [k - 2]  # the lower triangle of the last spoke
    polys, fr = brute_final_polygons(mesh)
    assert csr_to_lists(r["off"], r["vtx"]) == polys
    assert r["frontier_final"].tolist() == fr
    assert r["splits"] == 1 and len(polys) == 2
    check_final_mesh(mesh, polys, fr, convex=False)


def test_tip_hub_has_ten_tips_on_a_short_boundary():
    """tip_hub: one region whose boundary has 56 vertices and 10 tips (more than the
    GPU's shared-memory node list holds, fewer vertices than its thread walk's
    cap), pinned by brute force, with 10 splits."""
    mesh = tip_hub()
    pin_bruteforce(mesh, convex=False)
    pin_repair_bruteforce(mesh)
    r = oracle.full(mesh)
    trav = csr_to_lists(r["trav_off"], r["trav_vtx"])
    assert [len(p) for p in trav] == [56]
    assert len(tips(trav[0])) == 10
    assert r["splits"] == 10
    polys, fr = brute_final_polygons(mesh)
    check_final_mesh(mesh, polys, fr, convex=False)


def test_split_edge_ending_at_a_repeated_vertex():
    """A one-tip polygon whose split edge b -> x ends at a vertex its boundary visits
    twice (a pinch of the region): labels, regions and the final polygons pinned by
    brute force; x is the vertex after b in the first piece and occurs twice in the
    traversal polygon."""
    mesh = repeated_vertex_split()
    pin_bruteforce(mesh, convex=False, pinch=True)
    pin_repair_bruteforce(mesh)
    r = oracle.full(mesh)
    trav = csr_to_lists(r["trav_off"], r["trav_vtx"])
    final = csr_to_lists(r["off"], r["vtx"])
    found = False
    j = 0
    for v in trav:
        t = tips(v)
        n_pieces = 1 + (len(t) > 0)
        if len(t) == 1:
            b = t[0]  # the tip vertex
            p1, p2 = final[j], final[j + 1]
            assert len(p1) + len(p2) == len(v) + 2
            i = next(i for i in range(len(p1)) if p1[i] == b and p1[(i + 1) % len(p1)] in p2)
            x = p1[(i + 1) % len(p1)]
            found |= v.count(x) == 2
        elif len(t) > 1:
            break  # piece counts of several-tip polygons are not needed here
        j += n_pieces
    assert found


def test_trivertex_bruteforce():
    """The oracle's Trivertex array (Section 2): for every vertex the smallest
    half-edge leaving it, -1 for an unused vertex, against a direct search."""
    meshes = list(TINY[:20]) + [c["mesh"] for c in GOLDEN]
    base = TINY[3]
    extra = np.array([[(1 << 20) + 5, 9], [(1 << 20) + 7, 3]], np.int64)
    meshes.append({"xy": np.concatenate([base["xy"], extra]), "tri": base["tri"],
                   "twin": base["twin"]})  # two vertices no triangle uses
    for mesh in meshes:
        tv = oracle.trivertex(mesh)
        tri = np.asarray(mesh["tri"]).reshape(-1).tolist()
        for v in range(mesh["xy"].shape[0]):
            hs = [h for h, w in enumerate(tri) if w == v]
            assert tv[v] == (min(hs) if hs else -1), v


def test_invariants_uniform_1k():
    mesh = meshgen.load("uniform-1k")
    r = oracle.full(mesh)
    polys = csr_to_lists(r["trav_off"], r["trav_vtx"])
    # before reparation: one polygon per seed, sum of lengths = frontier half-edges
    assert len(polys) == len(r["seeds"])
    assert len(r["trav_vtx"]) == int(r["label"]["frontier"].sum())
    assert any(tips(p) for p in polys)
    final = csr_to_lists(r["off"], r["vtx"])
    check_final_mesh(mesh, final, r["frontier_final"])
    assert not any(tips(p) for p in final)
    # Section 3.2.3: each split adds one polygon and two vertex slots
    assert len(final) == len(polys) + r["splits"]
    assert len(r["vtx"]) == len(r["trav_vtx"]) + 2 * r["splits"]


def test_invariants_gmm_20k():
    mesh = meshgen.generate("gmm", 20_000, 1 << 26, 5)
    r = oracle.full(mesh)
    final = csr_to_lists(r["off"], r["vtx"])
    check_final_mesh(mesh, final, r["frontier_final"])
    assert len(final) == len(r["seeds"]) + r["splits"]


@pytest.mark.parametrize("seed", range(8))
def test_domain_with_holes_bruteforce(seed):
    """Non-convex domains with holes (border edges inside the hull): brute-force
    labels, regions and repair, and every final-mesh invariant with the domain's
    area and Euler characteristic."""
    mesh = meshgen.domain_with_holes("gmm" if seed % 2 else "uniform", 300, 1 << 16, 40 + seed)
    pin_bruteforce(mesh, convex=False)
    pin_repair_bruteforce(mesh)


def test_domain_with_holes_invariants_20k():
    mesh = meshgen.domain_with_holes("gmm", 20_000, 1 << 20, 9)
    r = oracle.full(mesh)
    final = csr_to_lists(r["off"], r["vtx"])
    check_final_mesh(mesh, final, r["frontier_final"], convex=False)
    assert len(final) == len(r["seeds"]) + r["splits"]


def test_run_matches_phases():
    mesh = meshgen.load("uniform-1k")
    a = oracle.full(mesh)
    b = oracle.run(mesh)
    assert np.array_equal(a["off"], b["off"]) and np.array_equal(a["vtx"], b["vtx"])
    assert np.array_equal(a["frontier_final"], b["frontier"])
    assert np.array_equal(a["label"]["max_edge"], b["max_edge"])


# --------------------------------------------------------------------- planted mistakes
MUTATIONS = {
    "tie_direction": ("return edge_id(twin, h) < edge_id(twin, g);",
                      "return edge_id(twin, h) > edge_id(twin, g);"),
    "tie_ignores_twin": ("return (g >= 0 && g < h) ? g : h;", "return h;"),
    "frontier_or": ("} else if (!is_longest(max_edge, h) && !is_longest(max_edge, g)) {",
                    "} else if (!is_longest(max_edge, h) || !is_longest(max_edge, g)) {"),
    "seed_upper_triangle": ("seed[ta < tb ? ta : tb] = 1;", "seed[ta < tb ? tb : ta] = 1;"),
    "border_seed_dropped": ("        seed[h / 3] = 1;\n", "        (void)0;\n"),
    "start_largest_origin": ("if (tri[h] < tri[start] || (tri[h] == tri[start] && h < start)) start = h;",
                             "if (tri[h] > tri[start] || (tri[h] == tri[start] && h < start)) start = h;"),
    "middle_floor_plus_one": ("const int64_t j = (k + 1) / 2;", "const int64_t j = k / 2 + 1;"),
    "middle_cw": ("static int64_t rot_ccw(const int32_t* twin, int64_t o) { return twin[he_prev(o)]; }",
                  "static int64_t rot_ccw(const int32_t* twin, int64_t o) { return he_next(twin[o]); }"),
    "halves_swapped": ("int64_t la = region_polygon(c, oj / 3, buf, NULL);",
                       "int64_t la = region_polygon(c, twin[oj] / 3, buf, NULL);"),
    "longest_is_shortest": ("if (edge_longer(xy, tri, twin, 3 * t + k, 3 * t + best)) best = k;",
                            "if (edge_longer(xy, tri, twin, 3 * t + best, 3 * t + k)) best = k;"),
    "length_dx_only": ("return dx * dx + dy * dy;", "return dx * dx + dy;"),
    "tip_largest_first": ("if (va == vc && (tip < 0 || vb < tip)) {",
                          "if (va == vc && (tip < 0 || vb > tip)) {"),
    "lepp_upper_seed": ("region[t] = (int32_t)(u < g / 3 ? u : g / 3);",
                        "region[t] = (int32_t)(u < g / 3 ? g / 3 : u);"),
    "lepp_depth_from_one": ("int64_t u = t, d = 0;", "int64_t u = t, d = 1;"),
}


def _run_pins(lib):
    """Run the pin suite on a given oracle build; returns the names of failed pins."""
    failed = []
    for case in GOLDEN:
        try:
            pin_golden(case, lib)
        except Exception:
            failed.append(case["name"])
    for k, seed in [(2, 1), (5, 2)]:
        try:
            pin_grid(k, seed, lib)
        except Exception:
            failed.append(f"grid{k}")
    for i, mesh in enumerate(TINY[:30]):
        try:
            pin_bruteforce(mesh, lib)
        except Exception:
            failed.append(f"tiny{i}")
    for i, mesh in enumerate(TIP_ORDER):
        try:
            pin_repair_bruteforce(mesh, lib)
        except Exception:
            failed.append(f"tiporder{i}")
    for i, mesh in enumerate(TINY[:10]):
        try:
            pin_lepp(mesh, lib)
        except Exception:
            failed.append(f"lepp{i}")
    return failed


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(oracle._SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor not found: {name}"
    mutated = tmp_path / "polylla_oracle.c"
    mutated.write_text(src.replace(old, new))
    shutil.copy(oracle._HDR, tmp_path / "polylla_oracle.h")
    lib = oracle.load_variant(str(mutated), str(tmp_path / f"lib_{name}.so"))
    failed = _run_pins(lib)
    assert failed, f"planted mistake '{name}' passed every pin"


def test_unmutated_oracle_passes_pin_suite():
    assert _run_pins(None) == []


# --------------------------------------------------------------------- LEPP
def pin_lepp(mesh, lib=None):
    """Longest-edge propagation paths: each triangle's path ends at the terminal
    edge the brute force reaches; the region it names is the triangle's connected
    component across non-frontier edges (and that component's seed); depth is 0
    exactly on the terminal edges' triangles and one more than the next triangle's
    elsewhere."""
    b = brute_labels(mesh)
    region, depth = oracle.lepp(mesh, np.asarray(b["max_edge"], np.uint8), lib)
    comp, _ = brute_regions(mesh, b["frontier"])
    ends = lepp_end(mesh, b["max_edge"])
    twin = mesh["twin"]
    seed_of = {}
    for t in range(len(comp)):
        if b["seed"][t]:
            seed_of[comp[t]] = t
    for t in range(len(comp)):
        assert region[t] == seed_of[comp[t]]
        assert ends[t] == ends[region[t]]
        h = 3 * t + b["max_edge"][t]
        g = int(twin[h])
        on_terminal = g < 0 or b["max_edge"][g // 3] == g % 3
        if on_terminal:
            assert depth[t] == 0
        else:
            assert depth[t] == depth[g // 3] + 1


@pytest.mark.parametrize("idx", range(0, 60, 6))
def test_lepp_tiny(idx):
    pin_lepp(TINY[idx])


def test_lepp_small_and_holes():
    for s in range(4):
        pin_lepp(meshgen.generate("gmm", 400, 1 << 16, 900 + s))
        pin_lepp(meshgen.domain_with_holes("uniform", 400, 1 << 16, 950 + s))
