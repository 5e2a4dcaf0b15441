"""Every device path against the oracle, with evidence that it ran.

Most polygons are walked by one thread and split by the one-tip or the several-tip
kernel; a few take rarer paths, which give the same polygons by other means:
regions too large for any thread block's shared memory are walked and split by one
thread (n_long_seq), polygons with more tips than the several-tip kernel's node
list holds are split by re-walking (n_multi_seq), and in the batch schedules that
try small blocks first, regions a small block cannot hold are handed to the large
blocks (n_long_handoff).  Hand-built meshes (tests/meshlib.py: spiral_wheel,
tip_hub) drive each counter above zero, and the output must still equal the
oracle's bit for bit.  The last test makes a turn exceed its step bound on a
corrupt (not validated) mesh and expects POLYLLA_ERR_LIMIT, not a hang."""
from __future__ import annotations

import numpy as np
import pytest

import meshgen
import oracle
from meshlib import disjoint_union, repeated_vertex_split, spiral_wheel, tip_hub

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2204_05438_gb300 as pg  # noqa: E402
from test_gpu_parity import assert_parity  # noqa: E402


def test_region_too_large_for_a_block_is_walked_by_one_thread():
    """A 5000-triangle region (5002 boundary vertices, one tip) exceeds the large
    block's 4096 members: the one-thread walk and re-walking split take it."""
    mesh = disjoint_union([spiral_wheel(5000), meshgen.generate("gmm", 3000, 1 << 22, 31)])
    g = assert_parity(mesh)
    st = g["stats"]
    assert st["n_long"] >= 1
    assert st["n_long_seq"] == 1
    assert st["n_splits"] >= 1


def test_polygon_with_more_tips_than_the_node_list_is_split_by_rewalking():
    """Three 56-vertex polygons with 10 tips each (the node list holds 8 splits), in a
    mesh of more than 2^16 triangles (smaller meshes give such polygons to the
    block kernel)."""
    mesh = disjoint_union([tip_hub(), tip_hub(), meshgen.generate("uniform", 40_000, 1 << 22, 32),
                           tip_hub()])
    g = assert_parity(mesh)
    st = g["stats"]
    assert st["n_multi_seq"] == 3
    assert st["n_multi_tip"] >= 3
    assert st["n_splits"] >= 30


def test_one_tip_split_ending_at_a_repeated_vertex_chases_the_arcs():
    """The one-tip kernel cuts its two pieces out of the traversal's vertex
    sequence; when the split edge ends at a vertex the polygon visits twice, the
    sequence does not say where the second piece starts, and the kernel chases the
    successors instead (n_one_chase).  Alone and next to an ordinary mesh."""
    for mesh in (repeated_vertex_split(),
                 disjoint_union([meshgen.generate("gmm", 3000, 1 << 22, 36), repeated_vertex_split()])):
        g = assert_parity(mesh)
        st = g["stats"]
        assert st["n_one_chase"] == 1
        assert st["n_one_tip"] > st["n_one_chase"] or st["n_one_tip"] == 1


@pytest.mark.parametrize("which", ["gmm-3k", "uniform-40k", "repeated-vertex", "hub+uniform"])
def test_rare_split_paths_give_the_same_polygons(which):
    """With the test switch on, every one-tip polygon is split by chasing the
    successors, every several-tip piece is ordered by (origin, half-edge) keys with
    its half-edges found by turning, and every split finds its far node through
    turn(oj): the paths kept for repeated vertices, run on whole meshes against the
    oracle (below 2^16 triangles the several-tip kernel sees two-tip polygons only,
    above it up to eight)."""
    mesh = {"gmm-3k": lambda: meshgen.generate("gmm", 3000, 1 << 22, 37),
            "uniform-40k": lambda: meshgen.generate("uniform", 40_000, 1 << 22, 38),
            "repeated-vertex": repeated_vertex_split,
            "hub+uniform": lambda: disjoint_union([tip_hub(), meshgen.generate("uniform", 40_000, 1 << 22, 39)]),
            }[which]()
    ref = oracle.run(mesh)
    M = pg.from_numpy(mesh)
    pg.debug_rare_paths(M.handle, True)
    for _ in range(2):
        M.run()
        off, vtx = (t.cpu().numpy() for t in M.polygons())
        np.testing.assert_array_equal(off, ref["off"])
        np.testing.assert_array_equal(vtx, ref["vtx"])
    st = M.stats()
    assert st["n_one_chase"] == st["n_one_tip"]
    if st["n_multi_tip"] > st["n_multi_seq"]:
        assert st["n_multi_turn"] >= 2 * (st["n_multi_tip"] - st["n_multi_seq"])
    pg.debug_rare_paths(M.handle, False)
    M.run()
    off, vtx = (t.cpu().numpy() for t in M.polygons())
    np.testing.assert_array_equal(vtx, ref["vtx"])
    M.close()


def test_small_mesh_gives_several_tip_polygons_to_the_block_kernel():
    """Below 2^16 triangles, polygons with three or more tips are split by one thread
    block each (the tips in parallel) instead of one thread; the result is the same."""
    mesh = disjoint_union([tip_hub(), meshgen.generate("gmm", 3000, 1 << 22, 34), tip_hub()])
    g = assert_parity(mesh)
    st = g["stats"]
    assert st["n_multi_seq"] == 0
    assert st["n_long"] >= 2
    assert st["n_splits"] >= 20


def test_batch_schedules_hand_long_regions_to_large_blocks():
    """Wheels of 100, 200, 1000 and 5000 triangles and a ten-tip hub in one batch:
    under the schedules that try one-warp (128 members) or small (512) blocks first,
    the larger regions are handed to the large blocks, and the 5000-triangle one on
    to the one-thread walk; every schedule gives every mesh the oracle's polygons."""
    meshes = [spiral_wheel(100), spiral_wheel(200), meshgen.generate("gmm", 1500, 1 << 22, 33),
              spiral_wheel(1000), tip_hub(), spiral_wheel(5000),
              meshgen.generate("uniform", 40_000, 1 << 22, 35)]  # > 2^16 triangles in all
    refs = [oracle.run(m) for m in meshes]
    cat = meshgen.concat(meshes)
    B = pg.batch_from_numpy(cat)
    for k in range(pg.batch_schedules()):
        info = pg.batch_schedule_info(k)
        for _ in range(3):  # eager, capture, replay
            B.run(k)
        off, vtx, first = (t.cpu().numpy().copy() for t in B.all_polygons())
        for j, ref in enumerate(refs):
            p0, p1 = int(first[j]), int(first[j + 1])
            o = off[p0:p1 + 1]
            np.testing.assert_array_equal(o - o[0], ref["off"], err_msg=f"schedule {k} mesh {j}")
            np.testing.assert_array_equal(vtx[o[0]:o[-1]] - cat["vtx_off"][j], ref["vtx"],
                                          err_msg=f"schedule {k} mesh {j}")
        st = B.stats()
        assert st["n_long_seq"] == 1, f"schedule {k}"
        if info["long_mode"] == 1:  # 512-member blocks: the 1000 and 5000 wheels move on
            assert st["n_long_handoff"] == 2, f"schedule {k}"
        elif info["long_mode"] == 2:  # 128-member warps: also the 200 wheel
            assert st["n_long_handoff"] >= 3, f"schedule {k}"
        else:
            assert st["n_long_handoff"] == 0, f"schedule {k}"
        if info["walk_cap"] >= 56:  # the hub's polygon is walked by a thread
            assert st["n_multi_seq"] == 1, f"schedule {k}"
    B.close()


def test_turn_bound_ends_with_limit_error():
    """A corrupt mesh, not validated: one triangle whose first half-edge names its
    third as twin (every id in range, but not an involution between reversed
    edges).  The first half-edge is the longest edge, so it is not frontier, and the
    turn around vertex 0 from the third half-edge re-enters the first forever; the
    bounded turn gives up after 3m steps and the run reports POLYLLA_ERR_LIMIT.  The
    context stays usable: a valid mesh runs afterwards."""
    mesh = {"xy": np.array([[0, 0], [10, 0], [5, 1]], np.int64),
            "tri": np.array([[0, 1, 2]], np.int32),
            "twin": np.array([2, -1, -1], np.int32)}
    M = pg.from_numpy(mesh, validate=False)
    M.run()
    with pytest.raises(pg.PolyllaError) as e:
        M.polygons()
    assert e.value.code == 6  # POLYLLA_ERR_LIMIT
    M.close()
    good = meshgen.load("uniform-1k")
    ref = oracle.run(good)
    M = pg.from_numpy(good)
    M.run()
    off, vtx = (t.cpu().numpy() for t in M.polygons())
    M.close()
    np.testing.assert_array_equal(off, ref["off"])
    np.testing.assert_array_equal(vtx, ref["vtx"])
