"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle on
the same seeded inputs.  Integer work, so every comparison is bit-exact: label
bytes (unpacked into the oracle's Max / terminal / frontier / Seed arrays), the
seed list, the traversal CSR, the final CSR and the labels after reparation."""
from __future__ import annotations

import numpy as np
import pytest

import meshgen
import oracle
from meshlib import golden_cases, grid_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2204_05438_gb300 as pg  # noqa: E402


def unpack_labels(lab: np.ndarray):
    lab = lab.astype(np.int64)
    m = lab.shape[0]
    max_edge = (lab & 3).astype(np.uint8)
    frontier = np.stack([(lab >> (2 + k)) & 1 for k in range(3)], axis=1).reshape(-1)
    seed = ((lab >> 5) & 1).astype(np.uint8)
    terminal = np.zeros(3 * m, np.uint8)
    tbit = ((lab >> 6) & 1).astype(bool)
    terminal[(3 * np.arange(m) + max_edge)[tbit]] = 1
    return {"max_edge": max_edge, "frontier": frontier.astype(np.uint8), "seed": seed,
            "terminal": terminal}


def gpu_phases(mesh, stream=None):
    M = pg.from_numpy(mesh)
    M.label(stream)
    lab0 = M.labels().cpu().numpy().copy()
    M.seeds(stream)
    seeds = M.seed_list().cpu().numpy().copy()
    M.traverse(stream)
    off0, vtx0 = (t.cpu().numpy().copy() for t in M.polygons())
    M.repair(stream)
    off1, vtx1 = (t.cpu().numpy().copy() for t in M.polygons())
    lab1 = M.labels().cpu().numpy().copy()
    stats = M.stats()
    M.close()
    return dict(lab0=lab0, seeds=seeds, off0=off0, vtx0=vtx0, off1=off1, vtx1=vtx1, lab1=lab1,
                stats=stats)


def gpu_run(mesh, repeats=1):
    M = pg.from_numpy(mesh)
    outs = []
    for _ in range(repeats):
        M.run()
        off, vtx = (t.cpu().numpy().copy() for t in M.polygons())
        outs.append((off, vtx, M.labels().cpu().numpy().copy(), M.stats()))
    M.close()
    return outs


def assert_parity(mesh, ref=None):
    ref = ref or oracle.full(mesh)
    g = gpu_phases(mesh)
    lab = unpack_labels(g["lab0"])
    for k in ("max_edge", "frontier", "seed", "terminal"):
        assert np.array_equal(lab[k], ref["label"][k]), f"label array {k} differs"
    assert np.array_equal(g["seeds"], ref["seeds"]), "seed list differs"
    assert np.array_equal(g["off0"], ref["trav_off"]), "traversal offsets differ"
    assert np.array_equal(g["vtx0"], ref["trav_vtx"]), "traversal polygons differ"
    assert np.array_equal(g["off1"], ref["off"]), "final offsets differ"
    assert np.array_equal(g["vtx1"], ref["vtx"]), "final polygons differ"
    fin = unpack_labels(g["lab1"])
    assert np.array_equal(fin["frontier"], ref["frontier_final"]), "labels after repair differ"
    st = g["stats"]
    assert st["n_seeds"] == len(ref["seeds"])
    assert st["n_splits"] == ref["splits"]
    assert st["n_poly"] == len(ref["off"]) - 1
    assert st["n_vtx"] == len(ref["vtx"])
    (off, vtx, lab_run, st_run), = gpu_run(mesh)
    assert np.array_equal(off, ref["off"]) and np.array_equal(vtx, ref["vtx"]), "run() differs"
    assert np.array_equal(lab_run, g["lab1"]), "run() labels differ"
    return g


GOLDEN = golden_cases()


@pytest.mark.parametrize("case", GOLDEN, ids=[c["name"] for c in GOLDEN])
def test_golden(case):
    g = assert_parity(case["mesh"])
    off, vtx = g["off1"], g["vtx1"]
    assert [vtx[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)] == case["expect"]["final"]


@pytest.mark.parametrize("k", [1, 2, 5, 33])
def test_grid(k):
    mesh, polys = grid_mesh(k, seed=k)
    g = assert_parity(mesh)
    assert g["stats"]["n_splits"] == 0 and g["stats"]["n_poly"] == k * k


@pytest.mark.parametrize("seed", range(24))
def test_tiny(seed):
    n = 4 + seed % 9
    mesh = meshgen.generate("uniform", n, 16 if seed % 3 == 0 else 1 << 12, 1000 + seed)
    assert_parity(mesh)


@pytest.mark.parametrize("n,kind,seed", [(300, "uniform", 77), (5_000, "gmm", 3),
                                         (20_000, "gmm", 5), (123_457, "uniform", 9)])
def test_random(n, kind, seed):
    mesh = meshgen.generate(kind, n, 1 << 22, seed)
    assert_parity(mesh)


def test_uniform_1k():
    g = assert_parity(meshgen.load("uniform-1k"))
    assert g["stats"]["n_splits"] > 0  # the configuration exercises reparation


def test_shuffled_triangles():
    mesh = meshgen.shuffled(meshgen.generate("gmm", 30_000, 1 << 24, 8), seed=1)
    assert_parity(mesh)


def test_disconnected_triangles():
    # two triangles sharing no edge: every edge is a border edge
    xy = np.array([[0, 0], [4, 0], [0, 3], [10, 10], [13, 10], [10, 14]], np.int64)
    tri = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    assert_parity({"xy": xy, "tri": tri, "twin": meshgen.twin_from_tri(tri)})


def test_vertex_where_two_fans_touch():
    # vertex 0 lies in two triangles that share no edge (a bow tie): the
    # per-vertex successor pass covers one fan, the per-triangle pass the rest
    xy = np.array([[0, 0], [4, 1], [1, 4], [-4, -1], [-1, -4]], np.int64) + 8
    tri = np.array([[0, 1, 2], [0, 3, 4]], np.int32)
    assert_parity({"xy": xy, "tri": tri, "twin": meshgen.twin_from_tri(tri)})
    # the same inside a larger mesh: carve the triangles around a vertex except two
    # opposite ones
    mesh = meshgen.generate("uniform", 2_000, 1 << 20, 31)
    tri = mesh["tri"]
    v = int(tri[len(tri) // 2, 0])
    around = np.nonzero((tri == v).any(axis=1))[0]
    assert len(around) >= 4
    keep = np.ones(len(tri), bool)
    keep[around] = False
    keep[around[0]] = keep[around[len(around) // 2]] = True
    tri = np.ascontiguousarray(tri[keep])
    assert_parity({"xy": mesh["xy"], "tri": tri, "twin": meshgen.twin_fast(tri)})


def test_unused_vertices():
    # vertices no triangle uses: more of them than half-edges, and a few
    xy = np.concatenate([np.array([[0, 0], [4, 0], [0, 3]], np.int64),
                         np.arange(20, dtype=np.int64).reshape(10, 2) + 100])
    tri = np.array([[0, 1, 2]], np.int32)
    assert_parity({"xy": xy, "tri": tri, "twin": meshgen.twin_from_tri(tri)})
    mesh = meshgen.generate("gmm", 3_000, 1 << 22, 12)
    extra = np.array([[(1 << 22) + 5, 7], [(1 << 22) + 9, 11]], np.int64)
    assert_parity({"xy": np.concatenate([mesh["xy"], extra]), "tri": mesh["tri"],
                   "twin": mesh["twin"]})


def test_uniform_1m_full():
    assert_parity(meshgen.load("uniform-1m"))


def test_gmm16_10m_full():
    """The benchmarked workload at full size, in the fused launch the bench times."""
    mesh = meshgen.load("gmm16-10m")
    ref = oracle.run(mesh)
    (off, vtx, lab, st), = gpu_run(mesh)
    assert np.array_equal(off, ref["off"]) and np.array_equal(vtx, ref["vtx"])
    fin = unpack_labels(lab)
    assert np.array_equal(fin["max_edge"], ref["max_edge"])
    assert np.array_equal(fin["frontier"], ref["frontier"])
    assert st["n_splits"] == ref["splits"]


def test_repeat_is_deterministic():
    mesh = meshgen.generate("gmm", 50_000, 1 << 24, 11)
    outs = gpu_run(mesh, repeats=3)
    for off, vtx, lab, _ in outs[1:]:
        assert np.array_equal(off, outs[0][0]) and np.array_equal(vtx, outs[0][1])
        assert np.array_equal(lab, outs[0][2])


def test_side_stream():
    mesh = meshgen.generate("uniform", 40_000, 1 << 22, 12)
    ref = oracle.full(mesh)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = gpu_phases(mesh, stream=s)
    assert np.array_equal(g["off1"], ref["off"]) and np.array_equal(g["vtx1"], ref["vtx"])


def test_run_host_matches_device():
    mesh = meshgen.generate("gmm", 60_000, 1 << 24, 13)
    ref = oracle.run(mesh)
    n, m = mesh["xy"].shape[0], mesh["tri"].shape[0]
    h = pg.mesh_create_host(n, m)
    xy = torch.from_numpy(mesh["xy"]).pin_memory()
    tri = torch.from_numpy(mesh["tri"]).pin_memory()
    twin = torch.from_numpy(mesh["twin"]).pin_memory()
    off = torch.empty(m + 1, dtype=torch.int64).pin_memory()
    vtx = torch.empty(3 * m, dtype=torch.int32).pin_memory()
    for _ in range(2):
        npoly, nv = pg.run_host(h, xy, tri, twin, off, vtx)
        assert np.array_equal(off[:npoly + 1].numpy(), ref["off"])
        assert np.array_equal(vtx[:nv].numpy(), ref["vtx"])
    pg.mesh_destroy(h)


# ------------------------------------------------------------------ error paths
def _expect(code, fn):
    codes = code if isinstance(code, tuple) else (code,)
    with pytest.raises(pg.PolyllaError) as e:
        fn()
    assert e.value.code in codes


def test_validate_rejects_bad_meshes():
    base = meshgen.load("uniform-1k")
    bad_twin = {k: v.copy() for k, v in base.items()}
    i = int(np.nonzero(bad_twin["twin"] >= 0)[0][0])
    bad_twin["twin"][i] = (bad_twin["twin"][i] + 1) % (3 * base["tri"].shape[0])
    _expect(3, lambda: pg.from_numpy(bad_twin))
    cw = {k: v.copy() for k, v in base.items()}
    cw["tri"][0] = cw["tri"][0][::-1].copy()  # clockwise (twins no longer match either)
    _expect(3, lambda: pg.from_numpy(cw))
    far = {k: v.copy() for k, v in base.items()}
    far["xy"][5, 0] = 1 << 30
    _expect(2, lambda: pg.from_numpy(far))
    bad_id = {k: v.copy() for k, v in base.items()}
    bad_id["tri"][3, 1] = base["xy"].shape[0]
    _expect((2, 3), lambda: pg.from_numpy(bad_id))  # out of range, and its twins mismatch
    bad_range = {k: v.copy() for k, v in base.items()}
    bad_range["twin"][7] = 3 * base["tri"].shape[0] + 5
    _expect((2, 3), lambda: pg.from_numpy(bad_range))


def test_phase_order_is_enforced():
    M = pg.from_numpy(meshgen.load("uniform-1k"))
    _expect(7, lambda: M.seeds())
    _expect(7, lambda: M.polygons())
    M.label()
    _expect(7, lambda: M.traverse())
    M.seeds()
    _expect(7, lambda: M.repair())
    M.traverse()
    M.repair()
    _expect(7, lambda: M.repair())
    M.label()  # restarts
    M.close()


def test_launch_count_and_timing():
    M = pg.from_numpy(meshgen.load("uniform-1k"))
    pg.set_timing(M.handle, True)
    for one_block, launches in ((0, 6), (pg.one_block_limit(), 1)):
        M.set_one_block(one_block)
        before = pg.launch_count(M.handle)
        M.run()
        times = pg.kernel_times(M.handle, reset=True)
        assert pg.launch_count(M.handle) - before == len(times) >= launches
        assert all(ms >= 0 for _, ms in times)
    assert [k for k, _ in times] == ["mesh_block"]
    M.close()


def test_tip_order_meshes():
    """Meshes on which the order of the tips changes the polygons."""
    from meshlib import tip_order_meshes
    for mesh in tip_order_meshes():
        ref = oracle.run(mesh)
        off, vtx, lab, _ = gpu_run(mesh)[0]
        np.testing.assert_array_equal(off, ref["off"])
        np.testing.assert_array_equal(vtx, ref["vtx"])


@pytest.mark.parametrize("n,kind,seed", [(300, "uniform", 1), (3000, "gmm", 2), (200_000, "gmm", 3)])
def test_domain_with_holes(n, kind, seed):
    """Non-convex domains with holes: border edges inside the hull."""
    mesh = meshgen.domain_with_holes(kind, n, 1 << 20, seed)
    assert_parity(mesh)


@pytest.mark.parametrize("name", ["uniform-1k", "uniform-1m", "holes-20k", "tiny"])
def test_lepp(name):
    """Longest-edge paths: region seed and path length per triangle, bit-exact."""
    if name == "holes-20k":
        meshes = [meshgen.domain_with_holes("gmm", 20_000, 1 << 20, 7)]
    elif name == "tiny":
        meshes = [c["mesh"] for c in golden_cases()] + [grid_mesh(6, 2)[0]]
    else:
        meshes = [meshgen.load(name)]
    for mesh in meshes:
        lab = oracle.label(mesh)
        ref_r, ref_d = oracle.lepp(mesh, lab["max_edge"])
        M = pg.from_numpy(mesh)
        M.label()
        with pytest.raises(pg.PolyllaError):
            pg.get_lepp(M.handle, M.m)  # before polylla_lepp
        r, d = (t.cpu().numpy() for t in M.lepp())
        M.seeds()  # the paths survive the later phases (they keep the Max array)
        M.traverse()
        M.repair()
        r2, _ = (t.cpu().numpy() for t in pg.get_lepp(M.handle, M.m))
        M.run()  # a new label phase: the paths must be asked for again
        with pytest.raises(pg.PolyllaError):
            pg.get_lepp(M.handle, M.m)
        M.close()
        np.testing.assert_array_equal(r, ref_r)
        np.testing.assert_array_equal(d, ref_d)
        np.testing.assert_array_equal(r2, ref_r)


@pytest.mark.parametrize("name", ["golden", "uniform-1k", "uniform-1m", "holes"])
def test_twin_built_on_device(name):
    """mesh_create without twin: the twin array built from tri equals the
    generator's, and the run gives the same polygons."""
    if name == "golden":
        meshes = [c["mesh"] for c in golden_cases()] + [grid_mesh(5, 1)[0]]
    elif name == "holes":
        meshes = [meshgen.domain_with_holes("gmm", 30_000, 1 << 20, 4)]
    else:
        meshes = [meshgen.load(name)]
    for mesh in meshes:
        xy = torch.as_tensor(mesh["xy"]).cuda().contiguous()
        tri = torch.as_tensor(np.ascontiguousarray(mesh["tri"])).cuda().contiguous()
        h = pg.mesh_create(xy, tri, None, pg.VALIDATE)
        pg.run(h)
        off, vtx = (t.cpu().numpy().copy() for t in pg.get_polygons(h))
        pg.mesh_destroy(h)
        ref = oracle.run(mesh)
        np.testing.assert_array_equal(off, ref["off"])
        np.testing.assert_array_equal(vtx, ref["vtx"])


def test_twin_built_on_device_twin_values_and_host_path():
    mesh = meshgen.load("uniform-1m")
    n, m = mesh["xy"].shape[0], mesh["tri"].shape[0]
    hm = pg.mesh_create_host(n, m)
    xy = torch.from_numpy(mesh["xy"]).reshape(-1).pin_memory()
    tri = torch.from_numpy(np.ascontiguousarray(mesh["tri"])).reshape(-1).pin_memory()
    off = torch.empty(m + 1, dtype=torch.int64).pin_memory()
    vtx = torch.empty(3 * m, dtype=torch.int32).pin_memory()
    np_, nv = pg.run_host(hm, xy, tri, None, off, vtx)
    _, _, tw = pg.mesh_inputs(hm, n, m)
    np.testing.assert_array_equal(tw.cpu().numpy(), mesh["twin"])
    pg.mesh_destroy(hm)
    ref = oracle.run(mesh)
    np.testing.assert_array_equal(off[:np_ + 1].numpy(), ref["off"])
    np.testing.assert_array_equal(vtx[:nv].numpy(), ref["vtx"])


def test_twin_built_on_device_rejects_non_manifold():
    base = [c["mesh"] for c in golden_cases()][1]
    tri = np.ascontiguousarray(base["tri"])
    bad = np.concatenate([tri, tri[:1]])  # a triangle twice: its directed edges twice
    xy = torch.as_tensor(base["xy"]).cuda().contiguous()
    t = torch.as_tensor(bad).cuda().contiguous()
    with pytest.raises(pg.PolyllaError) as e:
        pg.mesh_create(xy, t, None, 0)
    assert e.value.code == 3  # POLYLLA_ERR_TOPOLOGY
    # an edge of three triangles (0->1 twice, with a 1->0), and a directed edge twice
    # with no reverse (0->1 in two triangles on the same side)
    pts = torch.tensor([[0, 0], [10, 0], [5, 5], [5, -5], [4, 8]], dtype=torch.int64).cuda()
    for tris in ([[0, 1, 2], [1, 0, 3], [0, 1, 4]], [[0, 1, 2], [0, 1, 4]]):
        t = torch.tensor(tris, dtype=torch.int32).cuda().contiguous()
        with pytest.raises(pg.PolyllaError) as e:
            pg.mesh_create(pts, t, None, 0)
        assert e.value.code == 3, tris
