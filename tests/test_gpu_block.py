"""The one-block path of polylla_run against the oracle and the multi-kernel path.

A mesh of at most polylla_one_block_limit() triangles is meshed by one thread
block (labels, seeds, walks, splits and CSR in one launch).  Its final CSR, seed
list and labels after reparation must equal the oracle's bit for bit, and the
multi-kernel path's on the same handle, with polygons of several tips split in
increasing tip order (the default) and piece by piece (a test switch); the
statistic n_one_block shows which path ran.  The cases reach every branch of the
kernel: no tips, one tip, many tips on one polygon, a tip order that changes the
result, a single region of thousands of triangles, border-only and disconnected
meshes, non-convex domains with holes, the largest size the block takes and the
first it does not."""
from __future__ import annotations

import numpy as np
import pytest

import meshgen
import oracle
from meshlib import (disjoint_union, golden_cases, grid_mesh, repeated_vertex_split, spiral_wheel,
                     tip_hub, tip_order_meshes)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2204_05438_gb300 as pg  # noqa: E402


def run_path(M, one_block: int):
    M.set_one_block(one_block)
    M.run()
    off, vtx = (t.cpu().numpy().copy() for t in M.polygons())
    seeds = M.seed_list().cpu().numpy().copy()
    lab = M.labels().cpu().numpy().copy()
    return off, vtx, seeds, lab, M.stats()


def check_block(mesh, runs: int = 2):
    ref = oracle.full(mesh)
    m = mesh["tri"].shape[0]
    assert m <= pg.one_block_limit()
    M = pg.from_numpy(mesh)
    multi = run_path(M, 0)
    # polygons with several tips: split in increasing tip order (the default) and,
    # on the second run, piece by piece; the same handle again each time
    for r in range(runs):
        pg.debug_split_by_pieces(M.handle, r % 2 == 1)
        off, vtx, seeds, lab, st = run_path(M, pg.one_block_limit())
        np.testing.assert_array_equal(off, ref["off"])
        np.testing.assert_array_equal(vtx, ref["vtx"])
        np.testing.assert_array_equal(seeds, ref["seeds"])
        np.testing.assert_array_equal(off, multi[0])
        np.testing.assert_array_equal(vtx, multi[1])
        np.testing.assert_array_equal(seeds, multi[2])
        np.testing.assert_array_equal(lab, multi[3])  # labels after reparation
        fr = np.stack([(lab.astype(np.int64) >> (2 + k)) & 1 for k in range(3)], 1).reshape(-1)
        np.testing.assert_array_equal(fr.astype(np.uint8), ref["frontier_final"])
        assert st["n_one_block"] == len(ref["seeds"]) == st["n_seeds"]
        assert st["n_splits"] == ref["splits"]
        assert st["n_poly"] == len(ref["off"]) - 1 and st["n_vtx"] == len(ref["vtx"])
        assert st["n_poly_trav"] == multi[4]["n_poly_trav"]
        assert st["n_vtx_trav"] == multi[4]["n_vtx_trav"]
        assert st["n_tips"] == multi[4]["n_tips"]
        assert st["n_tip_polygons"] == multi[4]["n_tip_polygons"]
        assert st["n_long"] == st["n_one_tip"] == st["n_multi_tip"] == 0
    assert multi[4]["n_one_block"] == 0
    M.close()
    return ref


GOLDEN = golden_cases()


@pytest.mark.parametrize("case", GOLDEN, ids=[c["name"] for c in GOLDEN])
def test_golden(case):
    check_block(case["mesh"])


@pytest.mark.parametrize("k", [1, 3, 45])
def test_grid(k):
    ref = check_block(grid_mesh(k, seed=k)[0])
    assert len(ref["off"]) - 1 == k * k


@pytest.mark.parametrize("seed", range(12))
def test_tiny(seed):
    n = 4 + seed % 9
    check_block(meshgen.generate("uniform", n, 16 if seed % 3 == 0 else 1 << 12, 3000 + seed))


@pytest.mark.parametrize("n,kind,seed", [(300, "uniform", 5), (800, "gmm", 6), (1500, "gmm", 7),
                                         (2000, "gmm", 9), (2000, "uniform", 8)])
def test_random(n, kind, seed):
    check_block(meshgen.generate(kind, n, 1 << 20, seed))


@pytest.mark.parametrize("seed", range(40))
def test_random_sweep(seed):
    """Random small meshes of both kinds, 50 to 2,000 points, on lattices from 2^8
    (many equal lengths, so the tie rule decides) to 2^22, in both split orders."""
    rng = np.random.default_rng(7000 + seed)
    kind = "gmm" if seed % 2 else "uniform"
    n = int(rng.integers(50, 2001))
    side = 1 << int(rng.integers(8, 23))
    mesh = meshgen.generate(kind, n, side, 9000 + seed)
    if mesh["tri"].shape[0] > pg.one_block_limit():
        pytest.skip("larger than the one-block limit")
    check_block(mesh)


def test_uniform_1k():
    ref = check_block(meshgen.load("uniform-1k"))
    assert ref["splits"] > 0


def test_many_tips_on_one_polygon():
    """tip_hub: one region whose polygon has ten tips, split by the thread that
    walked it; three of them side by side."""
    ref = check_block(disjoint_union([tip_hub(), tip_hub(), tip_hub()]))
    assert ref["splits"] >= 30


def hub_grid(count: int, cols: int = 9):
    """`count` tip hubs side by side on a grid (coordinates stay below 2^30)."""
    meshes = [tip_hub() for _ in range(count)]
    xy, tri, twin, nv, nh = [], [], [], 0, 0
    for j, mesh in enumerate(meshes):
        xy.append(mesh["xy"] + np.array([(j % cols) << 25, (j // cols) << 25], np.int64))
        tri.append(mesh["tri"] + nv)
        tw = mesh["twin"].copy()
        tw[tw >= 0] += nh
        twin.append(tw)
        nv += mesh["xy"].shape[0]
        nh += 3 * mesh["tri"].shape[0]
    return {"xy": np.concatenate(xy), "tri": np.concatenate(tri).astype(np.int32),
            "twin": np.concatenate(twin).astype(np.int32)}


def test_split_scratch_overflow_falls_back_to_pieces():
    """75 tip hubs (4,050 triangles, 750 tips): their tip lists and piece trees
    need more than the block's split scratch, so the polygons that come late split
    piece by piece while the others split in tip order; all match the oracle."""
    mesh = hub_grid(75)
    assert mesh["tri"].shape[0] <= pg.one_block_limit() and mesh["xy"].max() < (1 << 30)
    ref = check_block(mesh, runs=1)
    assert ref["splits"] == 750


def test_tip_order_and_repeated_vertex():
    for mesh in tip_order_meshes() + [repeated_vertex_split()]:
        check_block(mesh)


def test_one_region_of_thousands_of_triangles():
    """spiral_wheel(4000): one region, one polygon of 4002 vertices with one tip."""
    ref = check_block(spiral_wheel(4000), runs=1)
    assert ref["splits"] == 1


@pytest.mark.parametrize("seed", [3, 4])
def test_domain_with_holes(seed):
    mesh = meshgen.domain_with_holes("gmm", 2000, 1 << 20, seed)
    check_block(mesh)


def test_disconnected_and_border_only():
    single = {"xy": np.array([[0, 0], [8, 0], [3, 5]], np.int64),
              "tri": np.array([[0, 1, 2]], np.int32), "twin": np.array([-1, -1, -1], np.int32)}
    check_block(disjoint_union([single, single, single]))


def test_size_limit_switches_paths():
    """The largest mesh the block takes (the limit set to m) and the first it
    leaves to the multi-kernel path (the limit set to m - 1): same polygons."""
    mesh = None
    for n in range(2000, 2100):  # a uniform mesh just below the block's limit
        cand = meshgen.generate("uniform", n, 1 << 20, 11)
        if cand["tri"].shape[0] <= pg.one_block_limit():
            mesh = cand
    assert mesh is not None and mesh["tri"].shape[0] > pg.one_block_limit() - 64
    m = mesh["tri"].shape[0]
    ref = oracle.run(mesh)
    M = pg.from_numpy(mesh)
    a = run_path(M, m)
    b = run_path(M, m - 1)
    M.close()
    assert a[4]["n_one_block"] > 0 and b[4]["n_one_block"] == 0
    for x in (a, b):
        np.testing.assert_array_equal(x[0], ref["off"])
        np.testing.assert_array_equal(x[1], ref["vtx"])
    np.testing.assert_array_equal(a[3], b[3])


def test_larger_mesh_takes_the_multi_kernel_path():
    mesh = meshgen.generate("uniform", 5000, 1 << 20, 12)
    assert mesh["tri"].shape[0] > pg.one_block_limit()
    M = pg.from_numpy(mesh)
    M.run()
    st = M.stats()
    M.close()
    assert st["n_one_block"] == 0 and st["n_poly"] > 0


def test_setting_is_checked():
    M = pg.from_numpy(GOLDEN[0]["mesh"])
    for bad in (-1, pg.one_block_limit() + 1):
        with pytest.raises(pg.PolyllaError) as e:
            M.set_one_block(bad)
        assert e.value.code == 1  # POLYLLA_ERR_INVALID_ARG
    M.close()


def test_one_launch():
    mesh = meshgen.load("uniform-1k")
    M = pg.from_numpy(mesh)
    M.run()
    M.polygons()
    before = pg.launch_count(M.handle)
    M.run()
    M.polygons()
    assert pg.launch_count(M.handle) - before == 1
    M.close()
