"""The triangulator's own formats, through the C ABI (Section 2's data structure):
the Neighbor array (N[3t + j], the triangle across edge j of t) converted to the
twin array on the device, in Triangle's opposite-vertex layout and in the
edge-from-vertex-j layout, and the Trivertex array (one half-edge leaving each
vertex) computed on the device.  Integer work: the twin array must equal the
generator's, the polygons and labels the oracle's, and the Trivertex array the
oracle's, element by element."""
from __future__ import annotations

import numpy as np
import pytest

import meshgen
import oracle
from meshlib import golden_cases, grid_mesh, neighbors_from_twin, spiral_wheel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2204_05438_gb300 as pg  # noqa: E402


def _meshes(name):
    if name == "golden":
        return [c["mesh"] for c in golden_cases()] + [grid_mesh(5, 1)[0], spiral_wheel(40)]
    if name == "holes":
        return [meshgen.domain_with_holes("gmm", 30_000, 1 << 20, 4)]
    return [meshgen.load(name)]


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt).contiguous()


@pytest.mark.parametrize("convention", [pg.NEIGHBOR_OPPOSITE, pg.NEIGHBOR_EDGE],
                         ids=["opposite-vertex", "edge-from-vertex"])
@pytest.mark.parametrize("name", ["golden", "uniform-1k", "holes", "uniform-1m"])
def test_neighbor_array_gives_the_twin_and_the_oracle_polygons(name, convention):
    for mesh in _meshes(name):
        m = mesh["tri"].shape[0]
        nb = neighbors_from_twin(mesh, convention)
        xy, tri = _dev(mesh["xy"], torch.int64), _dev(mesh["tri"], torch.int32)
        h = pg.mesh_create_neighbors(xy, tri, _dev(nb, torch.int32), convention, pg.VALIDATE)
        np.testing.assert_array_equal(pg.get_twin(h, m).cpu().numpy(), mesh["twin"])
        pg.run(h)
        off, vtx = (t.cpu().numpy().copy() for t in pg.get_polygons(h))
        lab = pg.get_labels(h, m).cpu().numpy().copy()
        pg.mesh_destroy(h)
        ref = oracle.run(mesh)
        np.testing.assert_array_equal(off, ref["off"])
        np.testing.assert_array_equal(vtx, ref["vtx"])
        np.testing.assert_array_equal((lab & 3).astype(np.uint8), ref["max_edge"])


def test_neighbor_array_rejects_inconsistent_entries():
    mesh = meshgen.load("uniform-1k")
    xy, tri = _dev(mesh["xy"], torch.int64), _dev(mesh["tri"], torch.int32)
    nb = neighbors_from_twin(mesh, 0)
    t = int(np.nonzero((nb >= 0).all(axis=1))[0][0])  # an interior triangle
    bad = nb.copy()
    bad[t, 0] = (bad[t, 0] + 7) % mesh["tri"].shape[0]  # a triangle not across that edge
    with pytest.raises(pg.PolyllaError) as e:
        pg.mesh_create_neighbors(xy, tri, _dev(bad, torch.int32), 0, 0)
    assert e.value.code == 3  # POLYLLA_ERR_TOPOLOGY
    bad = nb.copy()
    bad[t, 1] = mesh["tri"].shape[0]  # one past the last triangle
    with pytest.raises(pg.PolyllaError) as e:
        pg.mesh_create_neighbors(xy, tri, _dev(bad, torch.int32), 0, 0)
    assert e.value.code == 2  # POLYLLA_ERR_RANGE


@pytest.mark.parametrize("name", ["golden", "uniform-1k", "holes", "gmm16-10m"])
def test_trivertex_matches_the_oracle(name):
    meshes = _meshes(name)
    if name == "golden":  # and two vertices no triangle uses
        base = meshes[-2]
        extra = np.array([[(1 << 22) + 5, 7], [(1 << 22) + 9, 11]], np.int64)
        meshes.append({"xy": np.concatenate([base["xy"], extra]), "tri": base["tri"],
                       "twin": base["twin"]})
    for mesh in meshes:
        n = mesh["xy"].shape[0]
        M = pg.from_numpy(mesh)
        with pytest.raises(pg.PolyllaError) as e:
            pg.get_trivertex(M.handle, n)
        assert e.value.code == 7  # POLYLLA_ERR_STATE before polylla_trivertex
        pg.trivertex(M.handle)
        tv = pg.get_trivertex(M.handle, n).cpu().numpy().astype(np.int64)
        M.close()
        np.testing.assert_array_equal(tv, oracle.trivertex(mesh))
