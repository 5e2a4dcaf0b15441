"""The bench's multi-GPU bookkeeping on CPU ranks (gloo, world size 2): the
barrier, the maximum over ranks, the whole-job aggregate, and that the
reference arm runs on rank 0 alone.  The mesher itself does not shard -- each
rank runs a replica -- so there is no data-path collective to test."""
from __future__ import annotations

import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    try:
        out = {"world": d.world, "rank": d.rank}
        out["max"] = d.max(float(10 * (rank + 1)))
        d.barrier()
        # rank r took (r + 1) * 100 ms for 5 steps of 1000 units each
        out["agg"] = bench.aggregate(d, 1000, 5, 100.0 * (rank + 1))
        args = types.SimpleNamespace(workload="uniform-1k", steps=2, warmup=3, ref_seconds=1.0)
        ref = bench.run_reference(args, d)
        out["ref"] = None if ref is None else {k: ref[k] for k in ("impl", "n_gpus", "unit")}
        out["ref_value"] = None if ref is None else ref["value"]
        d.barrier()
    finally:
        d.close()
    q.put(out)


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    outs.sort(key=lambda o: o["rank"])
    assert [o["world"] for o in outs] == [2, 2]
    assert [o["max"] for o in outs] == [20.0, 20.0]
    for o in outs:
        ms, value = o["agg"]
        assert ms == pytest.approx(40.0)          # the slower rank: 200 ms / 5 steps
        assert value == pytest.approx(2 * 1000 * 5 / 0.2)
    assert outs[1]["ref"] is None                 # only rank 0 runs the reference arm
    assert outs[0]["ref"] == {"impl": "reference", "n_gpus": 2, "unit": "triangles/s"}
    assert outs[0]["ref_value"] > 0
