"""Served form: the native request loop (polylla_server_*) with continuous
batching.  Every result must equal, bit for bit, the plain single-mesh path's
result for the same mesh (and the oracle's) -- alone and in the mix, whatever
else the server had in flight -- and admission must respect the memory budget."""
from __future__ import annotations

import time

import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2204_05438_gb300 as pg  # noqa: E402


def pinned(mesh):
    return (torch.from_numpy(np.ascontiguousarray(mesh["xy"]).reshape(-1)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(mesh["tri"]).reshape(-1)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(mesh["twin"])).pin_memory())


def plain(mesh):
    M = pg.from_numpy(mesh)
    M.run()
    off, vtx = (t.cpu().numpy().copy() for t in M.polygons())
    M.close()
    return off, vtx


def drain(S, n, timeout_s=60.0):
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < n and time.time() < t_end:
        for r in S.poll(wait_us=20000):
            got[r["id"]] = r
    assert len(got) == n, f"{len(got)} of {n} requests completed"
    return got


def mixed_meshes(count, seed, nmin=200, nmax=60000):
    plan = meshgen.batch_plan(count, seed, nmin, nmax, side=1 << 20)
    return meshgen.batch(plan["ns"], plan["seeds"], plan["kinds"], plan["sides"])


def test_served_results_equal_alone_and_in_the_mix():
    meshes = mixed_meshes(24, 21)
    S = pg.Server(budget_bytes=8 << 30, max_slots=16)
    ids = [S.submit(*pinned(m)) for m in meshes]  # a burst: many in flight at once
    got = drain(S, len(ids))
    peak = S.info()["peak_running"]
    for rid, mesh in zip(ids, meshes):
        r = got[rid]
        assert r["status"] == 0
        off, vtx = plain(mesh)
        np.testing.assert_array_equal(r["off"].numpy(), off)
        np.testing.assert_array_equal(r["vtx"].numpy(), vtx)
        assert r["submit_s"] <= r["admit_s"] <= r["done_s"]
    # the first mesh again, alone
    rid = S.submit(*pinned(meshes[0]))
    r = drain(S, 1)[rid]
    ref = oracle.run(meshes[0])
    np.testing.assert_array_equal(r["off"].numpy(), ref["off"])
    np.testing.assert_array_equal(r["vtx"].numpy(), ref["vtx"])
    S.close()
    assert peak >= 2  # requests overlapped on the device


def test_served_admission_waits_for_memory():
    meshes = mixed_meshes(6, 22, 2000, 40000)
    big = max(meshes, key=lambda m: m["tri"].shape[0])
    c = 4096
    while c < max(big["tri"].shape[0], 2 * big["xy"].shape[0]):
        c <<= 1
    budget = int(pg.mesh_footprint(c // 2 + 2, c, True) * 1.3) + (1 << 20)
    S = pg.Server(budget_bytes=budget, max_slots=8)
    ids = [S.submit(*pinned(m)) for m in meshes]
    got = drain(S, len(ids))
    info = S.info()
    assert info["bytes_in_use"] <= budget
    for rid, mesh in zip(ids, meshes):
        off, vtx = plain(mesh)
        np.testing.assert_array_equal(got[rid]["off"].numpy(), off)
        np.testing.assert_array_equal(got[rid]["vtx"].numpy(), vtx)
    S.close()


def test_served_request_larger_than_budget_fails_cleanly():
    mesh = mixed_meshes(1, 23, 30000, 30001)[0]
    S = pg.Server(budget_bytes=2 << 20, max_slots=2)
    rid = S.submit(*pinned(mesh))
    r = drain(S, 1)[rid]
    assert r["status"] == 4  # POLYLLA_ERR_OOM
    small = mixed_meshes(1, 24, 10, 11)[0]
    rid = S.submit(*pinned(small))  # a request that fits still runs
    r = drain(S, 1)[rid]
    if pg.mesh_footprint(4096 // 2 + 2, 4096, True) + 4096 <= (2 << 20):
        assert r["status"] == 0
    S.close()


def test_served_without_twin():
    """Requests without a twin array: built on the device from tri."""
    meshes = mixed_meshes(6, 25, 500, 20000)
    S = pg.Server(budget_bytes=4 << 30, max_slots=4)
    ids = []
    for m in meshes:
        xy, tri, _ = pinned(m)
        ids.append(S.submit(xy, tri, None))
    got = drain(S, len(ids))
    for rid, mesh in zip(ids, meshes):
        assert got[rid]["status"] == 0
        off, vtx = plain(mesh)
        np.testing.assert_array_equal(got[rid]["off"].numpy(), off)
        np.testing.assert_array_equal(got[rid]["vtx"].numpy(), vtx)
    S.close()
