"""Failure handling driven from the host, with no GPU fault: device allocations
made to fail by the library's injection hook (every entry point must return
POLYLLA_ERR_OOM and free what it had taken), and served requests cancelled
while queued."""
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

OOM, STATE, CANCELLED = 4, 7, 8


def pinned(mesh):
    return (torch.from_numpy(np.ascontiguousarray(mesh["xy"]).reshape(-1)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(mesh["tri"]).reshape(-1)).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(mesh["twin"])).pin_memory())


def drain(S, n, timeout_s=60.0):
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < n and time.time() < t_end:
        for r in S.poll(wait_us=20000):
            got[r["id"]] = r
    assert len(got) == n, f"{len(got)} of {n} requests completed"
    return got


@pytest.mark.parametrize("twin", [True, False], ids=["twin", "twin-built"])
def test_mesh_create_fails_cleanly_at_every_allocation(twin):
    mesh = meshgen.generate("uniform", 100_000, 1 << 22, 21)
    xy = torch.as_tensor(mesh["xy"]).cuda().contiguous()
    tri = torch.as_tensor(mesh["tri"]).cuda().contiguous()
    tw = torch.as_tensor(mesh["twin"]).cuda().contiguous() if twin else None
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    k = 1
    try:
        while True:
            pg.debug_fail_alloc(k)
            try:
                h = pg.mesh_create(xy, tri, tw, 1)
            except pg.PolyllaError as e:
                assert e.code == OOM, (k, e)
                k += 1
                assert k < 200
                continue
            break  # fewer allocations than k: the injection never fired
    finally:
        pg.debug_fail_alloc(0)
    pg.run(h)
    off, vtx = pg.get_polygons(h)
    ref = oracle.run(mesh)
    assert np.array_equal(off.cpu().numpy(), ref["off"])
    assert np.array_equal(vtx.cpu().numpy(), ref["vtx"])
    pg.mesh_destroy(h)
    torch.cuda.synchronize()
    # every failed creation freed what it had allocated (k - 1 of them, a handle's
    # worth of buffers each: a leak would show as tens of MB)
    assert k > 10
    assert free0 - torch.cuda.mem_get_info()[0] < 8 << 20


def test_served_request_fails_on_allocation_and_the_server_recovers():
    mesh = meshgen.generate("gmm", 20_000, 1 << 20, 22)
    ref = oracle.run(mesh)
    S = pg.Server(budget_bytes=4 << 30, max_slots=4)
    try:
        pg.debug_fail_alloc(1)  # the new slot's first buffer
        rid = S.submit(*pinned(mesh))
        got = drain(S, 1)
        assert got[rid]["status"] == OOM
        pg.debug_fail_alloc(0)
        rid = S.submit(*pinned(mesh))
        got = drain(S, 1)
        assert got[rid]["status"] == 0
        assert np.array_equal(got[rid]["off"].numpy(), ref["off"])
        assert np.array_equal(got[rid]["vtx"].numpy(), ref["vtx"])
    finally:
        pg.debug_fail_alloc(0)
        S.close()


def test_served_cancel_removes_queued_requests_only():
    mesh = meshgen.generate("gmm", 150_000, 1 << 22, 23)
    ref = oracle.run(mesh)
    S = pg.Server(budget_bytes=8 << 30, max_slots=1)  # one slot: the rest queue
    try:
        # every pinned buffer first, so that the submissions and cancellations follow
        # each other within microseconds
        inp = pinned(mesh)
        m = mesh["tri"].shape[0]
        outs = [(torch.empty(m + 1, dtype=torch.int64).pin_memory(),
                 torch.empty(3 * m, dtype=torch.int32).pin_memory()) for _ in range(8)]
        ids = [S.submit(*inp, *o) for o in outs]
        cancelled = {rid for rid in ids[2:] if S.cancel(rid)}
        assert not S.cancel(10_000)  # unknown id
        got = drain(S, len(ids))
        for rid in ids:
            if rid in cancelled:
                assert got[rid]["status"] == CANCELLED
                assert not S.cancel(rid)  # already completed
            else:
                assert got[rid]["status"] == 0
                assert np.array_equal(got[rid]["off"].numpy(), ref["off"])
                assert np.array_equal(got[rid]["vtx"].numpy(), ref["vtx"])
        assert len(cancelled) >= 1  # at least the last one was still queued
        assert S.info()["pending"] == 0
    finally:
        S.close()
