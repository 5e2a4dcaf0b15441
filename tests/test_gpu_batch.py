"""Batched form: many meshes in one run (polylla_batch_*), through the C ABI.

Each mesh's polygons from the batch must equal, bit for bit, both the oracle's
polygons for that mesh alone and the plain single-mesh path's -- for every
schedule, for the tuned one, and on graph replays.  Vertex ids in the batch
index the concatenated coordinates, so mesh j's ids are shifted by vtx_off[j]."""
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


def small_batch(count=40, seed=11, nmin=40, nmax=6000):
    plan = meshgen.batch_plan(count, seed, nmin, nmax, side=1 << 20)
    meshes = meshgen.batch(plan["ns"], plan["seeds"], plan["kinds"], plan["sides"])
    return meshes


def batch_outputs(B, n):
    off, vtx, first = B.all_polygons()
    off, vtx, first = (t.cpu().numpy().copy() for t in (off, vtx, first))
    out = []
    for j in range(n):
        p0, p1 = int(first[j]), int(first[j + 1])
        o = off[p0:p1 + 1]
        out.append((o - o[0], vtx[o[0]:o[-1]].copy()))
    return out


def check_against_oracle(meshes, outs, cat):
    for j, mesh in enumerate(meshes):
        ref = oracle.run(mesh)
        off, vtx = outs[j]
        np.testing.assert_array_equal(off, ref["off"], err_msg=f"mesh {j} offsets")
        np.testing.assert_array_equal(vtx - cat["vtx_off"][j], ref["vtx"],
                                      err_msg=f"mesh {j} vertices")


def test_batch_every_schedule_matches_oracle():
    meshes = small_batch()
    cat = meshgen.concat(meshes)
    B = pg.batch_from_numpy(cat)
    for k in range(pg.batch_schedules()):
        for _ in range(3):  # eager, capture, replay
            B.run(k)
        check_against_oracle(meshes, batch_outputs(B, len(meshes)), cat)
    B.close()


def test_batch_tuned_and_replays_are_stable():
    meshes = small_batch(count=24, seed=12)
    cat = meshgen.concat(meshes)
    B = pg.batch_from_numpy(cat)
    best, ms = B.tune(reps=2)
    assert 0 <= best < pg.batch_schedules()
    assert len(ms) == pg.batch_schedules() and all(t > 0 for t in ms)
    B.run()
    first = batch_outputs(B, len(meshes))
    for _ in range(3):
        B.run()
    again = batch_outputs(B, len(meshes))
    for (a0, a1), (b0, b1) in zip(first, again):
        np.testing.assert_array_equal(a0, b0)
        np.testing.assert_array_equal(a1, b1)
    check_against_oracle(meshes, again, cat)
    B.close()


def test_batch_equals_plain_path_mesh_by_mesh():
    """A mesh's result is the same alone and in the mix."""
    meshes = small_batch(count=16, seed=13)
    meshes.append(grid_mesh(9, seed=3)[0])
    meshes += [c["mesh"] for c in golden_cases()]
    cat = meshgen.concat(meshes)
    B = pg.batch_from_numpy(cat)
    B.run(0)
    outs = batch_outputs(B, len(meshes))
    stats = B.stats()
    B.close()
    tot_poly = 0
    for j, mesh in enumerate(meshes):
        M = pg.from_numpy(mesh)
        M.run()
        off, vtx = (t.cpu().numpy().copy() for t in M.polygons())
        tot_poly += M.stats()["n_poly"]
        M.close()
        np.testing.assert_array_equal(outs[j][0], off)
        np.testing.assert_array_equal(outs[j][1] - cat["vtx_off"][j], vtx)
    assert stats["n_poly"] == tot_poly


def test_batch_single_mesh_get():
    meshes = small_batch(count=5, seed=14)
    cat = meshgen.concat(meshes)
    B = pg.batch_from_numpy(cat)
    B.run(1)
    for j, mesh in enumerate(meshes):
        off, vtx = B.polygons(j)
        off = off.cpu().numpy()
        vtx = vtx.cpu().numpy()
        ref = oracle.run(mesh)
        np.testing.assert_array_equal(off - off[0], ref["off"])
        np.testing.assert_array_equal(vtx[off[0]:off[-1]] - cat["vtx_off"][j], ref["vtx"])
    B.close()


def test_batch_rejects_bad_local_ids():
    meshes = small_batch(count=3, seed=15)
    cat = meshgen.concat(meshes)
    bad = dict(cat)
    bad["tri"] = cat["tri"].copy()
    t0 = int(cat["tri_off"][1])
    bad["tri"][t0, 0] = int(cat["vtx_off"][2] - cat["vtx_off"][1])  # one past mesh 1's vertices
    with pytest.raises(pg.PolyllaError) as e:
        pg.batch_from_numpy(bad)
    assert e.value.code == 2  # POLYLLA_ERR_RANGE
    bad = dict(cat)
    bad["twin"] = cat["twin"].copy()
    bad["twin"][3 * t0] = 3 * int(cat["tri_off"][2] - cat["tri_off"][1])
    with pytest.raises(pg.PolyllaError) as e:
        pg.batch_from_numpy(bad)
    assert e.value.code == 2
