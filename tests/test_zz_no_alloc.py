"""The allocation-free entry point (polylla_label_seeds_noalloc), for callers that
cannot allocate device memory: called through the C ABI twice in a row, its label
bytes, seed list and seed count must equal those of the handle-based entry points
(polylla_label + polylla_seeds) exactly -- the work is integer, so the tolerance
is zero.  This file is collected last on purpose."""
from __future__ import annotations

import numpy as np
import pytest

import meshgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2204_05438_gb300 as pg  # noqa: E402


def _reference(mesh):
    M = pg.from_numpy(mesh)
    M.label()
    M.seeds()
    lab = M.labels().cpu().numpy().copy()
    seeds = M.seed_list().cpu().numpy().copy()
    M.close()
    return lab, seeds


@pytest.mark.parametrize("mesh_fn", [
    lambda: meshgen.load("uniform-1k"),
    lambda: meshgen.generate("gmm", 200_003, 1 << 24, 21),
], ids=["uniform-1k", "gmm-200k"])
def test_noalloc_matches_handle_path(mesh_fn):
    mesh = mesh_fn()
    ref_lab, ref_seeds = _reference(mesh)
    m = mesh["tri"].shape[0]
    xy = torch.as_tensor(mesh["xy"]).cuda().contiguous()
    tri = torch.as_tensor(mesh["tri"]).cuda().contiguous()
    twin = torch.as_tensor(mesh["twin"]).cuda().contiguous()
    for call in range(2):  # two calls in a row share the one scratch array
        lab = torch.full((m,), 0xFF, dtype=torch.uint8, device="cuda")
        seeds = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        ns = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        pg.label_seeds_noalloc(xy, tri, twin, lab, seeds, ns)
        k = int(ns.item())
        assert k == len(ref_seeds), f"call {call}: seed count"
        assert np.array_equal(lab.cpu().numpy(), ref_lab), f"call {call}: label bytes"
        assert np.array_equal(seeds[:k].cpu().numpy(), ref_seeds), f"call {call}: seed list"


def test_noalloc_rejects_oversize():
    xy = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    tri = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    twin = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    lab = torch.zeros(1, dtype=torch.uint8, device="cuda")
    seeds = torch.zeros(1, dtype=torch.int32, device="cuda")
    ns = torch.zeros(1, dtype=torch.int64, device="cuda")
    lib = pg.load_library()
    code = lib.polylla_label_seeds_noalloc(xy.data_ptr(), 4, tri.data_ptr(), twin.data_ptr(),
                                           (1 << 26) + 1, lab.data_ptr(), seeds.data_ptr(),
                                           ns.data_ptr(), None)
    assert code == 1  # POLYLLA_ERR_INVALID_ARG, before any launch
