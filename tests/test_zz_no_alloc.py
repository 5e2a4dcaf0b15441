"""The allocation-free entry point (polylla_label_seeds_noalloc).

It serves callers that cannot call cudaMalloc: an application that carves all
device memory into its own arena at start-up, or code where an allocation's
implicit device synchronisation would stall other work.  Its scratch lives in a
fixed device array inside the library.  Called through the C ABI twice in a row,
its label bytes, seed list and seed count must equal those of the handle-based
entry points (polylla_label + polylla_seeds) and the CPU oracle's exactly -- the
work is integer, so the tolerance is zero -- also when the caller's label array
starts only 4 bytes into a larger buffer.  This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2204_05438_gb300 as pg  # noqa: E402


def _handle_path(mesh):
    M = pg.from_numpy(mesh)
    M.label()
    M.seeds()
    lab = M.labels().cpu().numpy().copy()
    seeds = M.seed_list().cpu().numpy().copy()
    M.close()
    return lab, seeds


def _oracle_label_bytes(mesh):
    """The label bytes as the library packs them, from the oracle's arrays."""
    r = oracle.full(mesh)
    lab = r["label"]
    m = mesh["tri"].shape[0]
    k = lab["max_edge"].astype(np.int64)
    fr = lab["frontier"].reshape(m, 3).astype(np.int64)
    term = lab["terminal"].reshape(m, 3)[np.arange(m), k].astype(np.int64)
    packed = k | (fr[:, 0] << 2) | (fr[:, 1] << 3) | (fr[:, 2] << 4) | \
        (lab["seed"].astype(np.int64) << 5) | (term << 6)
    return packed.astype(np.uint8), r["seeds"]


@pytest.mark.parametrize("mesh_fn", [
    lambda: meshgen.load("uniform-1k"),
    lambda: meshgen.generate("gmm", 200_003, 1 << 24, 21),
], ids=["uniform-1k", "gmm-200k"])
@pytest.mark.parametrize("lab_offset", [0, 4], ids=["aligned", "label-array-4-bytes-in"])
def test_noalloc_matches_handle_path_and_oracle(mesh_fn, lab_offset):
    mesh = mesh_fn()
    ref_lab, ref_seeds = _handle_path(mesh)
    ora_lab, ora_seeds = _oracle_label_bytes(mesh)
    assert np.array_equal(ref_lab, ora_lab) and np.array_equal(ref_seeds, ora_seeds)
    m = mesh["tri"].shape[0]
    xy = torch.as_tensor(mesh["xy"]).cuda().contiguous()
    tri = torch.as_tensor(mesh["tri"]).cuda().contiguous()
    twin = torch.as_tensor(mesh["twin"]).cuda().contiguous()
    for call in range(2):  # two calls in a row share the one scratch array
        big = torch.full((m + 16,), 0xFF, dtype=torch.uint8, device="cuda")
        lab = big[lab_offset:lab_offset + m]
        seeds = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        ns = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        pg.label_seeds_noalloc(xy, tri, twin, lab, seeds, ns)
        k = int(ns.item())
        got = lab.cpu().numpy()
        assert k == len(ref_seeds), f"call {call}: seed count"
        assert np.array_equal(got, ref_lab), f"call {call}: label bytes"
        assert np.array_equal(got, ora_lab), f"call {call}: label bytes against the oracle"
        assert np.array_equal(seeds[:k].cpu().numpy(), ora_seeds), f"call {call}: seed list"
        rest = big.cpu().numpy()
        assert (rest[:lab_offset] == 0xFF).all() and (rest[lab_offset + m:] == 0xFF).all(), \
            "bytes outside the label array were written"


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
