"""The paper's mixed variant (Sections 3.2 and 4): labels, seeds and traversal on
the GPU, the reparation phase by one host thread (polylla_repair_host), through
the C ABI.  Its final polygons and label bytes must equal the oracle's and the
all-GPU path's bit for bit (integer work), on the golden cases, the meshes where
the order of the tips matters, hand-built regions with one and ten tips, a domain
with holes and the 1k, 1M and 10M configurations."""
from __future__ import annotations

import numpy as np
import pytest

import meshgen
import oracle
from meshlib import disjoint_union, golden_cases, spiral_wheel, tip_hub, tip_order_meshes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2204_05438_gb300 as pg  # noqa: E402
from test_gpu_parity import unpack_labels  # noqa: E402


def _mixed(mesh):
    M = pg.from_numpy(mesh)
    M.label()
    M.seeds()
    M.traverse()
    M.repair_host()
    off, vtx = (t.cpu().numpy().copy() for t in M.polygons())
    lab = M.labels().cpu().numpy().copy()
    st = M.stats()
    M.close()
    return off, vtx, lab, st


CASES = {
    "golden": lambda: [c["mesh"] for c in golden_cases()],
    "tip-order": tip_order_meshes,
    "hand-built": lambda: [disjoint_union([tip_hub(), spiral_wheel(300), tip_hub()])],
    "holes": lambda: [meshgen.domain_with_holes("gmm", 20_000, 1 << 20, 5)],
    "uniform-1k": lambda: [meshgen.load("uniform-1k")],
    "uniform-1m": lambda: [meshgen.load("uniform-1m")],
    "gmm16-10m": lambda: [meshgen.load("gmm16-10m")],
}


@pytest.mark.parametrize("name", list(CASES))
def test_host_repair_matches_the_oracle_and_the_gpu_repair(name):
    for mesh in CASES[name]():
        ref = oracle.run(mesh)
        off, vtx, lab, st = _mixed(mesh)
        np.testing.assert_array_equal(off, ref["off"])
        np.testing.assert_array_equal(vtx, ref["vtx"])
        fin = unpack_labels(lab)
        np.testing.assert_array_equal(fin["frontier"], ref["frontier"])
        assert st["n_splits"] == ref["splits"]
        assert st["n_poly"] == len(ref["off"]) - 1 and st["n_vtx"] == len(ref["vtx"])
        M = pg.from_numpy(mesh)
        M.run()
        g_off, g_vtx = (t.cpu().numpy() for t in M.polygons())
        g_lab = M.labels().cpu().numpy()
        M.close()
        np.testing.assert_array_equal(off, g_off)
        np.testing.assert_array_equal(vtx, g_vtx)
        np.testing.assert_array_equal(lab, g_lab)


def test_host_repair_needs_a_traversal():
    M = pg.from_numpy(meshgen.load("uniform-1k"))
    M.label()
    M.seeds()
    with pytest.raises(pg.PolyllaError) as e:
        M.repair_host()
    assert e.value.code == 7  # POLYLLA_ERR_STATE
    M.traverse()
    M.repair_host()
    with pytest.raises(pg.PolyllaError) as e:  # the phase is done
        M.repair_host()
    assert e.value.code == 7
    M.close()
