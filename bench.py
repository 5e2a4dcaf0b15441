#!/usr/bin/env python
"""Benchmark of the terminal-edge-region mesher on one GB300 (or N replicas).

One step = the whole mesher (Algorithm 1: label, seeds, traversal, reparation)
over one mesh of the workload, through the C ABI (polylla_run), inputs resident
in HBM.  Default workload: 10,000,000 lattice points from a 16-component Gaussian
mixture on a 2^26 grid, exact Delaunay (about 20M triangles).  Its inputs
(xy 160 MB, tri 240 MB, twin 240 MB) are larger than L2, so no flush is done
between steps.

Prints one JSON line: triangles/s (device-timed with CUDA events), per-kernel
times and the HBM roofline of the dominant kernel, the end-to-end figure through
the host-buffer entry point (copies included), the CPU oracle as a reported
baseline, clocks sampled during the timed region, and the kernel-launch count.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --impl reference the oracle (plain sequential C, the only reference there
is) is timed on the host cores on a bounded sample of the same workload.
Under torchrun (N > 1) each rank runs an independent replica on its own GPU
(the path does not shard); the timed region is bracketed by a barrier and the
max over ranks is taken.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "triangles/sec end-to-end (device-timed) at 10M pts"
UNIT = "triangles/s"
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# on the gmm16-10m workload, keyed by the hash of the files that define these kernels
# (source_hash(TRAFFIC_FILES)); reported as null once that code changes.
TRAFFIC_FILES = ("final.cu", "label.cu", "long.cu", "polylla_internal.cuh", "trav.cu", "walk.cuh")
NCU_TRAFFIC = {
    "sources": "fe8214375f1b7185",
    # one ncu --set full capture per kernel on gmm16-5m (9,999,947 triangles),
    # scaled x2.0000 by triangle count to a gmm16-10m launch
    "bytes": {"walk": int((311.370 + 70.850) * 1e6 * 19999948 / 9999947),
              "succ": int((232.247 + 105.619) * 1e6 * 19999948 / 9999947),
              "out_write": int((90.156 + 27.965) * 1e6 * 19999948 / 9999947),
              "label_class": int((130.077 + 80.119) * 1e6 * 19999948 / 9999947),
              "label_max": int((200.068 + 8.866) * 1e6 * 19999948 / 9999947),
              "seed_write": int((10.046 + 0.001) * 1e6 * 19999948 / 9999947),
              "repair_one": int((83.686 + 3.596) * 1e6 * 19999948 / 9999947),
              "repair_multi": int((15.205 + 0.003) * 1e6 * 19999948 / 9999947)},
}


# ------------------------------------------------------------------ helpers
def source_hash(files=None) -> str:
    """Hash of the CUDA sources that hold device code (files with __global__ or
    __device__ functions; only `files` when given): the kernels the ncu counters
    were taken on.  Host-only files (the C-ABI entry points, the server) do not
    change it, and neither do comments (// to the end of a line and /* ... */ are
    left out) or the layout of white space."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2204_05438_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if files is not None and f not in files:
            continue
        with open(os.path.join(csrc, f), "rb") as fh:
            data = fh.read()
        if b"__global__" not in data and b"__device__" not in data:
            continue
        code = re.sub(rb"/\*.*?\*/", b"", data, flags=re.S)
        code = re.sub(rb"//[^\n]*", b"", code)
        code = re.sub(rb"\s+", b" ", code)
        h.update(f.encode())
        h.update(code)
    return h.hexdigest()[:16]


L2_BYTES = 126 << 20  # the GB300's L2 as the CUDA runtime reports it (when no device says)


def l2_note(input_bytes: int, l2_bytes: int = L2_BYTES) -> str:
    """How the timed steps stand to the L2 cache (no flush between steps either way)."""
    mb = input_bytes / 1e6
    if input_bytes > l2_bytes:
        return f"inputs larger than L2 ({mb:.0f} MB vs {l2_bytes >> 20} MiB); no flush"
    return (f"inputs ({mb:.2f} MB) fit in L2 and stay resident between steps; no flush "
            "(a latency measurement of one small mesh)")


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes(name: str, s: dict) -> float:
    """Bytes a kernel must move if every element it needs is read or written once
    (n vertices, m triangles, ns seeds, nv0 / nv traversal / final polygon
    vertices, np final polygons, ntp polygons with tips).  The reparation kernels and the long-polygon
    kernel touch about 1% of the mesh along dependent-load chains: they are
    latency-bound and carry no byte count."""
    n, m, ns, nv0, nv, npoly = s["n"], s["m"], s["ns"], s["nv0"], s["nv"], s["np"]
    return {
        # tri (3 x int32) and each vertex's xy (2 x int64) in, one label byte out
        "label_max": 12 * m + 16 * n + m,
        # twin in, own and neighbour label bytes in, label byte and tf words out
        "label_class": 12 * m + 2 * m + 12 * m,
        # label byte in, seed list and each seed's entry half-edge out
        "seed_write": m + 8 * ns,
        # label bytes and every tf word once, the successor of every frontier
        # half-edge out
        "succ": m + 12 * m + 4 * nv0,
        # per polygon its entry half-edge in and its output record (count, length,
        # pos) out, per vertex succ + origin in and pool out, and start, length,
        # tips and tip for each polygon with tips
        "walk": 4 * ns + 12 * nv0 + 16 * ns + 16 * s.get("ntp", 0),
        # per polygon its piece count and length
        "out_tiles": 8 * ns,
        # per polygon record in, pool in, offsets and vertices out
        "out_write": 16 * ns + 8 * nv + 8 * (npoly + 1),
    }.get(name, 0.0)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


class Dist:
    """Replica bookkeeping under torchrun: barrier and max-over-ranks only (gloo)."""

    def __init__(self):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(dist: Dist, units: int, steps: int, local_ms: float):
    """Whole-job figure over replicas: the slowest rank's time, every rank's units.
    Returns (ms per step, units per second)."""
    total_ms = dist.max(local_ms)
    return total_ms / steps, dist.world * units * steps / (total_ms / 1e3)


# ------------------------------------------------------------------ our arm
def run_ours(args, dist: Dist) -> dict | None:
    import numpy as np
    import torch

    import meshgen
    import paper_2204_05438_gb300 as pg

    torch.cuda.set_device(dist.local_rank)
    dev = torch.device("cuda", dist.local_rank)
    mesh = meshgen.load(args.workload)
    if args.shuffle is not None:  # locality stress: the same mesh, triangles in random order
        mesh = meshgen.shuffled(mesh, args.shuffle)
    n, m = mesh["xy"].shape[0], mesh["tri"].shape[0]
    M = pg.from_numpy(mesh, device=str(dev), validate=True)
    stream = torch.cuda.current_stream(dev)

    # warm-up (also yields the output sizes used for the byte counts)
    for _ in range(args.warmup):
        M.run(stream)
    torch.cuda.synchronize(dev)
    st = M.stats()

    # timed region: K fused steps, CUDA events on the launching stream
    clocks = ClockSampler(dist.local_rank)
    clocks.start()
    time.sleep(0.3)
    launches0 = pg.launch_count(M.handle)
    dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        M.run(stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dist.barrier()
    local_ms = e0.elapsed_time(e1)
    launches = pg.launch_count(M.handle) - launches0
    clk = clocks.stop()
    ms_per_step, value = aggregate(dist, m, args.steps, local_ms)
    # a mesh small enough for the one-block path: the multi-kernel path beside it
    # (same steps, outside the timed region)
    paths = None
    if m <= pg.one_block_limit():
        M.set_one_block(0)
        for _ in range(args.warmup):
            M.run(stream)
        e0.record(stream)
        for _ in range(args.steps):
            M.run(stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        M.set_one_block(pg.one_block_limit())
        paths = {"one_block_ms_per_step": round(local_ms / args.steps, 5),
                 "multi_kernel_ms_per_step": round(e0.elapsed_time(e1) / args.steps, 5)}

    # per-kernel durations: the same steps with events around every launch
    if args.kernel_steps <= 0:
        M.close()
        return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic", "config": {"workload": args.workload},
                "roofline": None, "gpu_launches": launches, "clocks": clk}
    pg.set_timing(M.handle, True)
    for _ in range(args.kernel_steps):
        M.run(stream)
    recs = pg.kernel_times(M.handle, reset=True)
    # the twin array from tri on the device (not part of the step): a handle that
    # builds it, timed per launch
    tw_h = pg.mesh_create(M.xy, M.tri, None, 0)
    pg.set_timing(tw_h, True)
    tw_ms = []
    for _ in range(5):
        pg.mesh_build_twin(tw_h, stream)
        tw_ms += [t for k, t in pg.kernel_times(tw_h, reset=True) if k == "build_twin"]
    pg.mesh_destroy(tw_h)
    # the longest-edge paths (not part of the step): mean of a few launches
    lepp_ms = []
    for _ in range(5):
        pg.lepp(M.handle, stream)
        lepp_ms += [t for k, t in pg.kernel_times(M.handle, reset=True) if k == "lepp"]
    pg.set_timing(M.handle, False)
    # the paper's mixed variant: the reparation phase on one host thread
    # (polylla_repair_host, wall clock, its copies included) against the GPU
    # reparation pass (polylla_repair, device events), after the same traversal
    mixed = {"host_ms": [], "gpu_ms": []}
    for _ in range(3):
        M.label(stream)
        M.seeds(stream)
        M.traverse(stream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        M.repair_host(stream)
        mixed["host_ms"].append((time.perf_counter() - t0) * 1e3)
        M.label(stream)
        M.seeds(stream)
        M.traverse(stream)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        M.repair(stream)
        r1.record(stream)
        torch.cuda.synchronize(dev)
        mixed["gpu_ms"].append(r0.elapsed_time(r1))
    mixed = {"host_repair_ms": round(statistics.median(mixed["host_ms"]), 3),
             "gpu_repair_ms": round(statistics.median(mixed["gpu_ms"]), 4),
             "what": "polylla_repair_host (one host thread, copies included) vs polylla_repair "
                     "(device) after the same traversal; median of 3"}
    per = {}
    for name, ms in recs:
        per.setdefault(name, []).append(ms)
    sizes = {"n": n, "m": m, "ns": st["n_seeds"], "nv0": st["n_vtx_trav"], "nv": st["n_vtx"],
             "np": st["n_poly"], "ntp": st["n_tip_polygons"]}
    peak, peak_kind = hbm_peak()
    kernels = {}
    step_sum = sum(statistics.mean(v) for v in per.values())
    for name, v in per.items():
        avg = statistics.mean(v)
        b = algorithmic_bytes(name, sizes)
        gbs = b / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        kernels[name] = {"ms": round(avg, 5), "share": round(avg / step_sum, 4),
                         "alg_bytes": int(b), "gbs": round(gbs, 1),
                         "frac": round(gbs / peak, 4)}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    label_seed = [k for k in ("label_max", "label_class", "scan_seeds", "seed_write") if k in kernels]
    ls_ms = sum(kernels[k]["ms"] for k in label_seed)
    ls_bytes = sum(kernels[k]["alg_bytes"] for k in label_seed)
    ls_io = 24 * m + 16 * n + m + 4 * sizes["ns"]
    # traversal: the successor pass and the walk together, against their own
    # algorithmic bytes and against the survey's estimate of the traversal phase's
    # bytes (about 35 B per triangle: twin, label and origin reads over the visited
    # half-edges, the vertex and offset writes)
    trav = [k for k in ("succ", "walk") if k in kernels]
    tr_ms = sum(kernels[k]["ms"] for k in trav)
    tr_bytes = sum(kernels[k]["alg_bytes"] for k in trav)
    tr_survey = 35 * m
    traffic = None
    if NCU_TRAFFIC["sources"] == source_hash(TRAFFIC_FILES):
        traffic = NCU_TRAFFIC["bytes"].get(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["gbs"], "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": kernels[dom]["frac"],
                "traffic": traffic, "alg_bytes_per_launch": kernels[dom]["alg_bytes"]}
    step_bytes = sum(k["alg_bytes"] for k in kernels.values())
    step_gbs = step_bytes / (ms_per_step * 1e-3) / 1e9

    # end to end from pinned host memory, through the public API: (1) the native
    # server with resident slots, requests back to back (one request's copies
    # overlap another's compute); (2) the synchronous single-call entry point
    e2e = None
    if args.e2e_steps > 0:
        hxy = torch.from_numpy(mesh["xy"]).reshape(-1).pin_memory()
        htri = torch.from_numpy(np.ascontiguousarray(mesh["tri"])).reshape(-1).pin_memory()
        htwin = torch.from_numpy(mesh["twin"]).pin_memory()
        outs = [(torch.empty(m + 1, dtype=torch.int64).pin_memory(),
                 torch.empty(3 * m, dtype=torch.int32).pin_memory()) for _ in range(3)]
        cls = 4096
        while cls < max(m, 2 * n):
            cls <<= 1
        slot = pg.mesh_footprint(cls // 2 + 2, cls, True)
        S = pg.Server(budget_bytes=int(3.2 * slot), max_slots=3)
        for k in range(3):  # creates the slots
            S.submit(hxy, htri, htwin, *outs[k])
        got = 0
        while got < 3:
            got += len(S.poll(wait_us=100000))
        dist.barrier()
        t0 = time.perf_counter()
        free, live, done, res = list(range(3)), {}, 0, None
        for k in range(args.e2e_steps):
            while not free:
                for r in S.poll(wait_us=1000):
                    free.append(live.pop(r["id"]))
                    done += 1
                    res = r
            b = free.pop()
            live[S.submit(hxy, htri, htwin, *outs[b])] = b
        while live:
            for r in S.poll(wait_us=1000):
                free.append(live.pop(r["id"]))
                done += 1
                res = r
        t1 = time.perf_counter()
        dist.barrier()
        info = S.info()
        S.close()
        bad = res is None or res["status"] != 0
        npoly, nvtx = (res["n_poly"], res["n_vtx"]) if not bad else (0, 0)
        e2e_s = dist.max(t1 - t0)
        # the same, the twin array built on the device from tri (one copy less)
        S = pg.Server(budget_bytes=int(3.2 * slot), max_slots=3)
        for k in range(3):
            S.submit(hxy, htri, None, *outs[k])
        got = 0
        while got < 3:
            got += len(S.poll(wait_us=100000))
        tn0 = time.perf_counter()
        free, live = list(range(3)), {}
        for k in range(args.e2e_steps):
            while not free:
                for r in S.poll(wait_us=1000):
                    free.append(live.pop(r["id"]))
            b = free.pop()
            live[S.submit(hxy, htri, None, *outs[b])] = b
        while live:
            for r in S.poll(wait_us=1000):
                free.append(live.pop(r["id"]))
        tn1 = time.perf_counter()
        S.close()
        notwin_s = dist.max(tn1 - tn0)
        # the synchronous entry point, for comparison
        hm = pg.mesh_create_host(n, m)
        pg.run_host(hm, hxy, htri, htwin, outs[0][0], outs[0][1], stream)
        ts0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            pg.run_host(hm, hxy, htri, htwin, outs[0][0], outs[0][1], stream)
        ts1 = time.perf_counter()
        pg.mesh_destroy(hm)
        sync_s = dist.max(ts1 - ts0)
        e2e = {"value": dist.world * m * args.e2e_steps / e2e_s, "unit": UNIT,
               "ms_per_step": 1e3 * e2e_s / args.e2e_steps,
               "h2d_bytes_per_step": int(16 * n + 24 * m),
               "d2h_bytes_per_step": int(8 * (npoly + 1) + 4 * nvtx + 8 * 3),
               "api": "polylla_server_submit / polylla_server_poll (3 resident slots)",
               "peak_running": info["peak_running"], "failed": int(bad),
               "sync": {"value": dist.world * m * args.e2e_steps / sync_s,
                        "ms_per_step": 1e3 * sync_s / args.e2e_steps,
                        "api": "polylla_run_host"},
               "twin_built_on_device": {"value": dist.world * m * args.e2e_steps / notwin_s,
                                        "ms_per_step": 1e3 * notwin_s / args.e2e_steps,
                                        "h2d_bytes_per_step": int(16 * n + 12 * m)}}

    M.close()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": args.workload + ("" if args.shuffle is None else
                                                 f", triangles shuffled (seed {args.shuffle})"),
                   "points": n, "triangles": m,
                   "generator": "SplitMix64 16-component Gaussian mixture on a 2^26 lattice, "
                                "exact Delaunay (seed 2)",
                   "parallelism": f"replicas x{dist.world}" if dist.world > 1 else "single GPU",
                   "l2": l2_note(16 * n + 24 * m,
                                 getattr(torch.cuda.get_device_properties(dev), "L2_cache_size",
                                         L2_BYTES) or L2_BYTES),
                   "step": "polylla_run: label + seeds + traverse + repair, inputs resident"},
        "roofline": roofline,
        # alg_bytes: what the four kernels read and write, each array once (the
        # Max bytes handed from label_max to label_class and the tf words the
        # traversal consumes included); alg_bytes_io: the phases' own inputs and
        # outputs only (tri, xy, twin in; label byte and seed list out)
        "label_seed": {"ms": round(ls_ms, 5), "alg_bytes": int(ls_bytes),
                       "gbs": round(ls_bytes / (ls_ms * 1e-3) / 1e9, 1) if ls_ms else None,
                       "frac": round(ls_bytes / (ls_ms * 1e-3) / 1e9 / peak, 4) if ls_ms else None,
                       "alg_bytes_io": int(ls_io),
                       "frac_io": round(ls_io / (ls_ms * 1e-3) / 1e9 / peak, 4) if ls_ms else None},
        "traversal": {"kernels": trav, "ms": round(tr_ms, 5), "alg_bytes": int(tr_bytes),
                      "frac": round(tr_bytes / (tr_ms * 1e-3) / 1e9 / peak, 4) if tr_ms else None,
                      "alg_bytes_survey": int(tr_survey),
                      "frac_survey": round(tr_survey / (tr_ms * 1e-3) / 1e9 / peak, 4) if tr_ms else None},
        "twin_build": {"ms": round(statistics.mean(tw_ms), 5) if tw_ms else None,
                       "what": "polylla_mesh_build_twin: twin from tri on the device"},
        "lepp": {"ms": round(statistics.mean(lepp_ms), 5) if lepp_ms else None,
                 "value": m / (statistics.mean(lepp_ms) * 1e-3) if lepp_ms else None,
                 "unit": UNIT, "what": "polylla_lepp: region seed and path length per triangle"},
        "step_roofline": {"alg_bytes": int(step_bytes), "gbs": round(step_gbs, 1),
                          "frac": round(step_gbs / peak, 4)},
        "kernels": kernels,
        "mesh_stats": st,
        "mixed": mixed,
        "paths": paths,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "sources": source_hash(),
    }
    return out


def run_batched(args, dist: Dist) -> dict | None:
    """The batched form: 4,096 meshes (point counts log-uniform in [200, 200,000],
    uniform or Gaussian mixture per mesh) as one batch -- autotuned schedule, CUDA
    graph replays, inputs resident -- against the plain per-mesh path (one
    polylla_run per mesh on one stream) on every 8th mesh of the same batch."""
    import numpy as np
    import torch

    import meshgen
    import paper_2204_05438_gb300 as pg

    dev = torch.device("cuda", dist.local_rank)
    t0 = time.perf_counter()
    plan = meshgen.batch_plan(args.batch_meshes, 2024 + dist.rank)
    meshes = meshgen.batch(plan["ns"], plan["seeds"], plan["kinds"], plan["sides"])
    cat = meshgen.concat(meshes)
    gen_s = time.perf_counter() - t0
    m = int(cat["tri_off"][-1])
    stream = torch.cuda.current_stream(dev)
    B = pg.batch_from_numpy(cat, device=str(dev), validate=True)
    best, tune_ms = B.tune(reps=2)
    for _ in range(args.warmup):
        B.run()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    e0.record(stream)
    for _ in range(args.batch_steps):
        B.run()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dist.barrier()
    ms = dist.max(e0.elapsed_time(e1)) / args.batch_steps
    st = B.stats()
    # one run with per-kernel events (eager: timing bypasses the graphs)
    hm = pg.batch_mesh(B.handle)
    pg.set_timing(hm, True)
    B.run(best)
    recs = pg.kernel_times(hm, reset=True)
    pg.set_timing(hm, False)
    kern = {}
    for name, t in recs:
        kern[name] = round(kern.get(name, 0.0) + t, 4)
    B.close()

    # plain path, one mesh at a time, on a sample of the same meshes
    sample = list(range(0, len(meshes), 8))
    plain_ms, plain_tri = 0.0, 0
    for j in sample:
        M = pg.from_numpy(meshes[j], device=str(dev), validate=False)
        M.run(stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        M.run(stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms += a.elapsed_time(b)
        plain_tri += meshes[j]["tri"].shape[0]
        M.close()
    plain_tps = plain_tri / (plain_ms * 1e-3)
    value = dist.world * m / (ms * 1e-3)
    return {"meshes": len(meshes), "triangles": m, "points": int(cat["vtx_off"][-1]),
            "ms_per_run": ms, "value": value, "unit": UNIT,
            "schedule": best, "schedule_info": pg.batch_schedule_info(best),
            "tune_ms": [round(t, 4) for t in tune_ms],
            "plain": {"value": plain_tps, "unit": UNIT, "meshes": len(sample),
                      "triangles": plain_tri, "ms": round(plain_ms, 3),
                      "sample": "every 8th mesh of the batch, one polylla_run each"},
            "batched_over_plain": value / dist.world / plain_tps,
            "n_poly": st["n_poly"], "stats": st, "kernels_ms": kern,
            "generation_s": round(gen_s, 1),
            "graph": "CUDA graph per schedule, replayed"}


def run_served(args, dist: Dist) -> dict | None:
    """The served form: Poisson arrivals (mean 2,000 requests/s) of meshes with
    point counts log-uniform in [1,000, 1,000,000], replayed from a pre-generated
    pool, through the native request loop (memory-budgeted admission, resident
    slots, overlapping requests).  Latency = completion - submission per request."""
    import numpy as np
    import torch

    import meshgen
    import paper_2204_05438_gb300 as pg

    plan = meshgen.batch_plan(args.serve_pool, 4048 + dist.rank, 1000, 1_000_000)
    pool = meshgen.batch(plan["ns"], plan["seeds"], plan["kinds"], plan["sides"])
    host = [(torch.from_numpy(np.ascontiguousarray(m["xy"]).reshape(-1)).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(m["tri"]).reshape(-1)).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(m["twin"])).pin_memory()) for m in pool]
    free = {j: [] for j in range(len(pool))}

    def outbuf(j):
        if free[j]:
            return free[j].pop()
        mm = pool[j]["tri"].shape[0]
        return (torch.empty(mm + 1, dtype=torch.int64, pin_memory=True),
                torch.empty(3 * mm, dtype=torch.int32, pin_memory=True))

    S = pg.Server(budget_bytes=args.serve_budget_gb << 30, max_slots=args.serve_slots)
    # pinned output buffers for several requests of each mesh in flight, allocated
    # before the timed window (a pinned allocation during it stalls the device)
    for j in range(len(pool)):
        free[j] = [outbuf(j) for _ in range(4)]
    # warm the slots of every size class (allocation is not part of serving): each
    # mesh once, then every mesh twice at once, so that the bursts of the timed
    # streams find idle slots instead of creating them (a slot's allocations stall
    # the device while the worker holds the queue)
    for burst in (1, 2):
        warm = [outbuf(j) for j in range(len(pool)) for _ in range(burst)]
        for k, bufs in enumerate(warm):
            S.submit(*host[k // burst], *bufs)
        t_end = time.time() + 120
        done = 0
        while done < len(warm) and time.time() < t_end:
            done += len(S.poll(wait_us=20000))
        for k, bufs in enumerate(warm):
            free[k // burst].append(bufs)
    def poisson(n_req, seed):
        """Submit n_req requests at Poisson arrivals; returns (latencies, triangles
        done, failures, first submission, last completion) once all completed."""
        rng = np.random.default_rng(seed)
        gaps = rng.exponential(1.0 / args.serve_rate, n_req)
        pick = rng.integers(0, len(pool), n_req)
        owner, lat, tri_done, bad = {}, [], 0, 0

        def collect(wait_us):
            nonlocal tri_done, bad
            for r in S.poll(wait_us=wait_us):
                j, bufs = owner.pop(r["id"])
                free[j].append(bufs)
                bad += r["status"] != 0
                lat.append(r["done_s"] - r["submit_s"])
                tri_done += pool[j]["tri"].shape[0]

        t_next = time.perf_counter()
        for k in range(n_req):
            t_next += gaps[k]
            while time.perf_counter() < t_next:
                collect(0)
                if t_next - time.perf_counter() > 2e-4:
                    time.sleep(1e-4)
            j = int(pick[k])
            bufs = outbuf(j)
            owner[S.submit(*host[j], *bufs)] = (j, bufs)
        while owner:
            collect(20000)
        return lat, tri_done, bad

    # one untimed second of the same stream first: the slots its bursts need are
    # created before the timed window (a slot's allocation stalls the device)
    poisson(int(args.serve_rate), 1077 + dist.rank)
    slots_before = S.info()["slots"]
    n_req = int(args.serve_rate * args.serve_seconds)
    # the tail varies from stream to stream: several independent timed streams,
    # reported as the median with the spread
    trials = []
    for trial in range(max(1, args.serve_trials)):
        t0 = time.perf_counter()
        lat, tri_done, status_bad = poisson(n_req, 77 + 1000 * trial + dist.rank)
        wall = time.perf_counter() - t0
        lat = np.array(lat) * 1e3
        trials.append({"value": tri_done / wall, "p50_ms": float(np.percentile(lat, 50)),
                       "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                       "failed": status_bad})
    info = S.info()
    S.close()

    def med(k):
        return float(np.median([t[k] for t in trials]))

    return {"requests": n_req, "rate_per_s": args.serve_rate, "seconds": args.serve_seconds,
            "trials": len(trials),
            "pool_meshes": len(pool), "mean_points": float(np.mean(plan["ns"])),
            "offered_triangles_per_s": float(np.mean([p["tri"].shape[0] for p in pool])) * args.serve_rate,
            "value": med("value"), "unit": UNIT,
            "p50_ms": med("p50_ms"), "p99_ms": med("p99_ms"),
            "p99_ms_range": [min(t["p99_ms"] for t in trials), max(t["p99_ms"] for t in trials)],
            "max_ms": max(t["max_ms"] for t in trials),
            "failed": int(sum(t["failed"] for t in trials)),
            "per_trial": trials,
            "peak_running": info["peak_running"], "slots": info["slots"],
            "slots_created_in_timed_streams": info["slots"] - slots_before,
            "budget_gb": args.serve_budget_gb,
            "latency": "completion minus submission, seconds on the server's steady clock; "
                       "median over the trials"}


def cpu_baseline(mesh_name: str, budget_s: float) -> dict:
    """The oracle as it stands, one host thread, on the full workload mesh (or a
    smaller mesh of the same distribution if the full one would exceed the budget)."""
    import meshgen
    import oracle

    mesh = meshgen.load(mesh_name)
    m = mesh["tri"].shape[0]
    t0 = time.perf_counter()
    oracle.run(mesh)
    dt = time.perf_counter() - t0
    return {"value": m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one full run of {mesh_name} ({m} triangles) in {dt:.2f} s, "
                      "sequential C, 1 thread"}


# ------------------------------------------------------------------ reference arm
def run_reference(args, dist: Dist) -> dict | None:
    """The CPU oracle, timed on the host cores, each step one run over a bounded
    sample of the workload: a mesh of the same distribution (16-component Gaussian
    mixture on a 2^26 lattice) sized so that warm-up + steps take about two minutes."""
    import meshgen
    import oracle

    if dist.rank != 0:
        return None
    cfg = meshgen.CONFIGS[args.workload]
    per_step = max(0.01, args.ref_seconds / max(1, args.steps + args.warmup))
    sec_per_tri = 1.0 / 2.4e6  # oracle throughput measured on the full workload (one Arm core)
    tri_target = per_step / sec_per_tri
    n_sample = int(min(cfg["n"], max(500, tri_target / 2)))
    mesh = meshgen.generate(cfg["kind"], n_sample, cfg["side"], cfg["seed"])
    m = mesh["tri"].shape[0]
    for _ in range(args.warmup):
        oracle.run(mesh)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(mesh)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = m * args.steps / total
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": args.workload, "sample_points": n_sample, "sample_triangles": m,
                   "parallelism": "host CPU, 1 thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n_sample}-point mesh of the {args.workload} distribution "
                                   f"({m} triangles) per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="gmm16-10m")
    ap.add_argument("--shuffle", type=int, default=None,
                    help="put the workload's triangles in a seeded random order (locality stress)")
    ap.add_argument("--kernel-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="reference arm: host time of warm-up + steps, which sizes its sample")
    ap.add_argument("--batch-meshes", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-trials", type=int, default=3,
                    help="independent timed Poisson streams (median and spread reported)")
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-budget-gb", type=int, default=64)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    dist = Dist()
    try:
        if args.impl == "reference":
            out = run_reference(args, dist)
        else:
            out = run_ours(args, dist)
            # the served stream before the batch: measured after the 237M-triangle
            # batch in the same process, its latency tail is 2-4x longer (p99 1.4-2.4
            # ms instead of 0.6 ms), a state a server process does not meet
            if out is not None and not args.no_serve and args.kernel_steps > 0:
                out["served"] = run_served(args, dist)
            if out is not None and not args.no_batch and args.kernel_steps > 0:
                out["batched"] = run_batched(args, dist)
            if out is not None and dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
                out["cpu_baseline"] = cpu_baseline(args.workload, 30.0)
        if out is not None and dist.rank == 0:
            print(json.dumps(out), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
