"""GB300-native terminal-edge-region polygonal mesher (Python binding).

Argument marshalling only: every step of the mesher runs in the CUDA kernels of
``libpolylla.so`` (sources in ``csrc/``, C ABI in ``include/polylla.h``).  PyTorch
provides device memory and streams.  The functions mirror the C entry points:

    mesh_create, label, seeds, traverse, repair, run, get_labels, get_seeds,
    get_polygons, get_stats, mesh_destroy, status_str, mesh_create_host,
    run_host, set_timing, kernel_times, launch_count, label_seeds_noalloc,
    mesh_create_neighbors, get_twin, trivertex, get_trivertex, repair_host

There is no CPU fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB

VALIDATE = 1
LAB_MAX_MASK = 0x03
LAB_FRONTIER_SHIFT = 2
LAB_SEED = 0x20
LAB_TERMINAL = 0x40

STATUS = {0: "POLYLLA_OK", 1: "POLYLLA_ERR_INVALID_ARG", 2: "POLYLLA_ERR_RANGE",
          3: "POLYLLA_ERR_TOPOLOGY", 4: "POLYLLA_ERR_OOM", 5: "POLYLLA_ERR_CUDA",
          6: "POLYLLA_ERR_LIMIT", 7: "POLYLLA_ERR_STATE", 8: "POLYLLA_ERR_CANCELLED"}


class PolyllaError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_poly", ctypes.c_int64), ("n_vtx", ctypes.c_int64), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("slots", "bytes_in_use", "budget_bytes", "pending",
                                               "running", "peak_running", "completed")] + \
               [("now_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "n_seeds", "n_poly_trav", "n_vtx_trav", "n_tip_polygons", "n_tips", "n_splits",
        "n_poly", "n_vtx", "n_long", "n_long_handoff", "n_long_seq", "n_one_tip", "n_multi_tip",
        "n_multi_seq", "n_one_chase", "n_multi_turn", "n_one_block")]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load (building it first if needed) the CUDA library.  Raises on failure."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if path is None and not os.path.exists(p):
            _build.build()
        if not os.path.exists(p):
            raise ImportError(f"libpolylla not found at {p}; run __graft_entry__.build()")
        lib = ctypes.CDLL(p)
        vp, i64, u32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
        st = ctypes.c_int
        sig = {
            "polylla_mesh_create": ([vp, i64, vp, i64, vp, u32, vp, ctypes.POINTER(vp)], st),
            "polylla_label": ([vp, vp], st),
            "polylla_seeds": ([vp, vp], st),
            "polylla_traverse": ([vp, vp], st),
            "polylla_repair": ([vp, vp], st),
            "polylla_run": ([vp, vp], st),
            "polylla_get_labels": ([vp, ctypes.POINTER(vp)], st),
            "polylla_get_seeds": ([vp, ctypes.POINTER(vp), ctypes.POINTER(i64)], st),
            "polylla_get_polygons": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      ctypes.POINTER(i64), ctypes.POINTER(i64)], st),
            "polylla_get_stats": ([vp, ctypes.POINTER(Stats)], st),
            "polylla_mesh_destroy": ([vp], st),
            "polylla_status_str": ([st], ctypes.c_char_p),
            "polylla_mesh_create_host": ([i64, i64, ctypes.POINTER(vp)], st),
            "polylla_run_host": ([vp, vp, vp, vp, vp, vp, ctypes.POINTER(i64),
                                  ctypes.POINTER(i64), vp], st),
            "polylla_set_timing": ([vp, i32], st),
            "polylla_kernel_times": ([vp, ctypes.POINTER(ctypes.c_char_p),
                                      ctypes.POINTER(ctypes.c_float), i64, i32], i64),
            "polylla_launch_count": ([vp], i64),
            "polylla_label_seeds_noalloc": ([vp, i64, vp, vp, i64, vp, vp, vp, vp], st),
            "polylla_batch_create": ([vp, vp, vp, vp, vp, i64, u32, vp, ctypes.POINTER(vp)], st),
            "polylla_batch_schedules": ([], i32),
            "polylla_batch_schedule_info": ([i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                             ctypes.POINTER(i32)], st),
            "polylla_batch_tune": ([vp, i32, vp, ctypes.POINTER(i32),
                                    ctypes.POINTER(ctypes.c_float)], st),
            "polylla_batch_run": ([vp, i32, vp], st),
            "polylla_batch_get": ([vp, i64, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                   ctypes.POINTER(i64), ctypes.POINTER(i64)], st),
            "polylla_batch_get_all": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), ctypes.POINTER(i64),
                                       ctypes.POINTER(i64)], st),
            "polylla_batch_stats": ([vp, ctypes.POINTER(Stats)], st),
            "polylla_batch_mesh": ([vp], vp),
            "polylla_batch_destroy": ([vp], st),
            "polylla_mesh_footprint": ([i64, i64, i32], i64),
            "polylla_mesh_set_size": ([vp, i64, i64], st),
            "polylla_mesh_inputs": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(vp)], st),
            "polylla_get_polygons_async": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                            ctypes.POINTER(vp), ctypes.POINTER(vp)], st),
            "polylla_server_create": ([i64, i32, ctypes.POINTER(vp)], st),
            "polylla_server_submit": ([vp, vp, i64, vp, vp, i64, vp, vp, ctypes.POINTER(i64)], st),
            "polylla_server_poll": ([vp, ctypes.POINTER(Result), i64, i64], i64),
            "polylla_server_info": ([vp, ctypes.POINTER(ServerStats)], st),
            "polylla_server_cancel": ([vp, i64], st),
            "polylla_debug_fail_alloc": ([i64], None),
            "polylla_debug_rare_paths": ([vp, i32], st),
            "polylla_set_one_block": ([vp, i64], st),
            "polylla_debug_split_by_pieces": ([vp, i32], st),
            "polylla_one_block_limit": ([], i64),
            "polylla_server_destroy": ([vp], st),
            "polylla_lepp": ([vp, vp], st),
            "polylla_mesh_build_twin": ([vp, vp], st),
            "polylla_get_lepp": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp)], st),
            "polylla_mesh_create_neighbors": ([vp, i64, vp, i64, vp, i32, u32, vp,
                                               ctypes.POINTER(vp)], st),
            "polylla_get_twin": ([vp, ctypes.POINTER(vp)], st),
            "polylla_trivertex": ([vp, vp], st),
            "polylla_get_trivertex": ([vp, ctypes.POINTER(vp)], st),
            "polylla_repair_host": ([vp, vp], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        if path is None:
            _lib = lib
        return lib


def _check(code: int, where: str):
    if code != 0:
        raise PolyllaError(code, where)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dptr(t: torch.Tensor, dtype: torch.dtype, name: str) -> int:
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t.data_ptr()


class _DeviceArray:
    """A borrowed device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr) if n else 0, False), "version": 3,
                                         "strides": None}


def _view(ptr: int, n: int, typestr: str, dtype: torch.dtype) -> torch.Tensor:
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda")


# ------------------------------------------------------------------ C-ABI mirror
def mesh_create(xy: torch.Tensor, tri: torch.Tensor, twin: torch.Tensor | None,
                flags: int = VALIDATE, stream=None) -> int:
    """polylla_mesh_create: xy int64 [n,2], tri int32 [m,3], twin int32 [3m] on the GPU
    (twin None: built on the device from tri)."""
    lib = load_library()
    n = xy.numel() // 2
    m = tri.numel() // 3
    h = ctypes.c_void_p()
    tw = None if twin is None else _dptr(twin, torch.int32, "twin")
    _check(lib.polylla_mesh_create(_dptr(xy, torch.int64, "xy"), n, _dptr(tri, torch.int32, "tri"),
                                   m, tw, flags, _stream(stream), ctypes.byref(h)),
           "polylla_mesh_create")
    return h.value


NEIGHBOR_OPPOSITE = 0
NEIGHBOR_EDGE = 1


def mesh_create_neighbors(xy: torch.Tensor, tri: torch.Tensor, neighbor: torch.Tensor,
                          convention: int = NEIGHBOR_OPPOSITE, flags: int = VALIDATE,
                          stream=None) -> int:
    """polylla_mesh_create_neighbors: the twin array built on the device from the
    triangulator's Neighbor array (int32 [m,3]; convention NEIGHBOR_OPPOSITE: entry
    j across the edge opposite vertex j, as in Triangle's .neigh files)."""
    lib = load_library()
    n = xy.numel() // 2
    m = tri.numel() // 3
    h = ctypes.c_void_p()
    _check(lib.polylla_mesh_create_neighbors(
        _dptr(xy, torch.int64, "xy"), n, _dptr(tri, torch.int32, "tri"), m,
        _dptr(neighbor, torch.int32, "neighbor"), convention, flags, _stream(stream),
        ctypes.byref(h)), "polylla_mesh_create_neighbors")
    return h.value


def get_twin(mesh: int, m: int) -> torch.Tensor:
    p = ctypes.c_void_p()
    _check(load_library().polylla_get_twin(mesh, ctypes.byref(p)), "polylla_get_twin")
    return _view(p.value, 3 * m, "<i4", torch.int32)


def trivertex(mesh: int, stream=None):
    _check(load_library().polylla_trivertex(mesh, _stream(stream)), "polylla_trivertex")


def get_trivertex(mesh: int, n: int) -> torch.Tensor:
    p = ctypes.c_void_p()
    _check(load_library().polylla_get_trivertex(mesh, ctypes.byref(p)), "polylla_get_trivertex")
    return _view(p.value, n, "<i4", torch.int32)


def label(mesh: int, stream=None):
    _check(load_library().polylla_label(mesh, _stream(stream)), "polylla_label")


def seeds(mesh: int, stream=None):
    _check(load_library().polylla_seeds(mesh, _stream(stream)), "polylla_seeds")


def traverse(mesh: int, stream=None):
    _check(load_library().polylla_traverse(mesh, _stream(stream)), "polylla_traverse")


def repair(mesh: int, stream=None):
    _check(load_library().polylla_repair(mesh, _stream(stream)), "polylla_repair")


def repair_host(mesh: int, stream=None):
    """polylla_repair_host: the reparation phase on the host (the paper's mixed
    variant), after traverse; synchronises."""
    _check(load_library().polylla_repair_host(mesh, _stream(stream)), "polylla_repair_host")


def run(mesh: int, stream=None):
    _check(load_library().polylla_run(mesh, _stream(stream)), "polylla_run")


def get_labels(mesh: int, m: int) -> torch.Tensor:
    """View of the handle's label bytes (uint8 [m]); valid until the next phase call."""
    p = ctypes.c_void_p()
    _check(load_library().polylla_get_labels(mesh, ctypes.byref(p)), "polylla_get_labels")
    return _view(p.value, m, "|u1", torch.uint8)


def get_seeds(mesh: int) -> torch.Tensor:
    p, n = ctypes.c_void_p(), ctypes.c_int64()
    _check(load_library().polylla_get_seeds(mesh, ctypes.byref(p), ctypes.byref(n)),
           "polylla_get_seeds")
    return _view(p.value, n.value, "<i4", torch.int32)


def get_polygons(mesh: int):
    """Views (off int64 [np+1], vtx int32 [nv]) of the latest CSR polygons."""
    po, pv = ctypes.c_void_p(), ctypes.c_void_p()
    npoly, nv = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().polylla_get_polygons(mesh, ctypes.byref(po), ctypes.byref(pv),
                                               ctypes.byref(npoly), ctypes.byref(nv)),
           "polylla_get_polygons")
    off = torch.as_tensor(_DeviceArray(po.value, npoly.value + 1, "<i8"), device="cuda")
    return off, _view(pv.value, nv.value, "<i4", torch.int32)


def get_stats(mesh: int) -> dict:
    s = Stats()
    _check(load_library().polylla_get_stats(mesh, ctypes.byref(s)), "polylla_get_stats")
    return s.as_dict()


def mesh_destroy(mesh: int):
    _check(load_library().polylla_mesh_destroy(mesh), "polylla_mesh_destroy")


def status_str(code: int) -> str:
    return load_library().polylla_status_str(code).decode()


def mesh_create_host(n_vertices: int, n_tri: int) -> int:
    h = ctypes.c_void_p()
    _check(load_library().polylla_mesh_create_host(n_vertices, n_tri, ctypes.byref(h)),
           "polylla_mesh_create_host")
    return h.value


def run_host(mesh: int, xy: torch.Tensor, tri: torch.Tensor, twin: torch.Tensor,
             off_out: torch.Tensor, vtx_out: torch.Tensor, stream=None):
    """polylla_run_host on (preferably pinned) CPU tensors; returns (n_poly, n_vtx)."""
    for t, name in ((xy, "xy"), (tri, "tri"), (twin, "twin"), (off_out, "off"), (vtx_out, "vtx")):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous host tensor")
    npoly, nv = ctypes.c_int64(), ctypes.c_int64()
    tw = None if twin is None else twin.data_ptr()
    _check(load_library().polylla_run_host(mesh, xy.data_ptr(), tri.data_ptr(), tw,
                                           off_out.data_ptr(), vtx_out.data_ptr(),
                                           ctypes.byref(npoly), ctypes.byref(nv),
                                           _stream(stream)), "polylla_run_host")
    return npoly.value, nv.value


def set_timing(mesh: int, enable: bool = True):
    _check(load_library().polylla_set_timing(mesh, int(enable)), "polylla_set_timing")


def kernel_times(mesh: int, reset: bool = True, cap: int = 1 << 16):
    """[(kernel name, ms)] of the launches timed since the last reset."""
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_float * cap)()
    k = load_library().polylla_kernel_times(mesh, names, ms, cap, int(reset))
    if k < 0:
        raise PolyllaError(5, "polylla_kernel_times")
    return [(names[i].decode(), float(ms[i])) for i in range(min(k, cap))]


def launch_count(mesh: int) -> int:
    return int(load_library().polylla_launch_count(mesh))


def label_seeds_noalloc(xy: torch.Tensor, tri: torch.Tensor, twin: torch.Tensor,
                        lab_out: torch.Tensor, seeds_out: torch.Tensor, n_seeds_out: torch.Tensor,
                        stream=None):
    """polylla_label_seeds_noalloc: label bytes, seed list and seed count written
    into caller-provided device tensors (uint8 [m], int32 [m], int64 [1]); the
    library allocates nothing.  For callers that cannot allocate device memory."""
    m = tri.numel() // 3
    if lab_out.numel() < m or seeds_out.numel() < m or n_seeds_out.numel() < 1:
        raise ValueError("output tensors are too small")
    _check(load_library().polylla_label_seeds_noalloc(
        _dptr(xy, torch.int64, "xy"), xy.numel() // 2, _dptr(tri, torch.int32, "tri"),
        _dptr(twin, torch.int32, "twin"), m, _dptr(lab_out, torch.uint8, "lab_out"),
        _dptr(seeds_out, torch.int32, "seeds_out"), _dptr(n_seeds_out, torch.int64, "n_seeds_out"),
        _stream(stream)), "polylla_label_seeds_noalloc")


def mesh_build_twin(mesh: int, stream=None):
    _check(load_library().polylla_mesh_build_twin(mesh, _stream(stream)), "polylla_mesh_build_twin")


def lepp(mesh: int, stream=None):
    _check(load_library().polylla_lepp(mesh, _stream(stream)), "polylla_lepp")


def get_lepp(mesh: int, m: int):
    """Views (region int32 [m], depth int32 [m]) of the longest-edge paths."""
    a, b = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load_library().polylla_get_lepp(mesh, ctypes.byref(a), ctypes.byref(b)),
           "polylla_get_lepp")
    return _view(a.value, m, "<i4", torch.int32), _view(b.value, m, "<i4", torch.int32)


SCHEDULE_TUNED = -1


def batch_create(xy: torch.Tensor, vtx_off: torch.Tensor, tri: torch.Tensor, twin: torch.Tensor,
                 tri_off: torch.Tensor, flags: int = VALIDATE, stream=None) -> int:
    """Concatenated meshes with local ids (see polylla_batch_create)."""
    out = ctypes.c_void_p()
    n = vtx_off.numel() - 1
    if tri_off.numel() - 1 != n:
        raise ValueError("vtx_off and tri_off must describe the same number of meshes")
    _check(load_library().polylla_batch_create(
        _dptr(xy, torch.int64, "xy"), _dptr(vtx_off, torch.int64, "vtx_off"),
        _dptr(tri, torch.int32, "tri"), _dptr(twin, torch.int32, "twin"),
        _dptr(tri_off, torch.int64, "tri_off"), n, flags, _stream(stream), ctypes.byref(out)),
        "polylla_batch_create")
    return out.value


def batch_schedules() -> int:
    return int(load_library().polylla_batch_schedules())


def batch_schedule_info(schedule: int) -> dict:
    cap, thr, ovl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().polylla_batch_schedule_info(schedule, ctypes.byref(cap),
                                                      ctypes.byref(thr), ctypes.byref(ovl)),
           "polylla_batch_schedule_info")
    return {"walk_cap": cap.value, "long_mode": thr.value, "overlap": ovl.value}


def batch_tune(batch: int, reps: int = 3, stream=None):
    """Time every schedule; returns (best, [ms per run for each schedule])."""
    k = batch_schedules()
    best = ctypes.c_int()
    ms = (ctypes.c_float * k)()
    _check(load_library().polylla_batch_tune(batch, reps, _stream(stream), ctypes.byref(best), ms),
           "polylla_batch_tune")
    return best.value, [float(x) for x in ms]


def batch_run(batch: int, schedule: int = SCHEDULE_TUNED, stream=None):
    _check(load_library().polylla_batch_run(batch, schedule, _stream(stream)), "polylla_batch_run")


def batch_get(batch: int, mesh: int):
    """Mesh `mesh`'s polygons: (off int64 [np+1], vtx int32 view of the whole batch);
    polygon k is vtx[off[k]:off[k+1]], ids into the concatenated xy."""
    po, pv = ctypes.c_void_p(), ctypes.c_void_p()
    npoly, nv = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().polylla_batch_get(batch, mesh, ctypes.byref(po), ctypes.byref(pv),
                                            ctypes.byref(npoly), ctypes.byref(nv)),
           "polylla_batch_get")
    off = torch.as_tensor(_DeviceArray(po.value, npoly.value + 1, "<i8"), device="cuda")
    end = int(off[-1].item()) if npoly.value >= 0 else 0
    return off, _view(pv.value, end, "<i4", torch.int32)


def batch_get_all(batch: int, n_meshes: int):
    """(off int64 [np+1], vtx int32 [nv], mesh_first int64 [n_meshes+1]) of the whole
    batch: mesh j owns polygons mesh_first[j] .. mesh_first[j+1]-1."""
    po, pv, pf = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    npoly, nv = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().polylla_batch_get_all(batch, ctypes.byref(po), ctypes.byref(pv),
                                                ctypes.byref(pf), ctypes.byref(npoly),
                                                ctypes.byref(nv)),
           "polylla_batch_get_all")
    off = torch.as_tensor(_DeviceArray(po.value, npoly.value + 1, "<i8"), device="cuda")
    first = torch.as_tensor(_DeviceArray(pf.value, n_meshes + 1, "<i8"), device="cuda")
    return off, _view(pv.value, nv.value, "<i4", torch.int32), first


def batch_stats(batch: int) -> dict:
    s = Stats()
    _check(load_library().polylla_batch_stats(batch, ctypes.byref(s)), "polylla_batch_stats")
    return s.as_dict()


def batch_mesh(batch: int) -> int:
    return load_library().polylla_batch_mesh(batch)


def batch_destroy(batch: int):
    _check(load_library().polylla_batch_destroy(batch), "polylla_batch_destroy")


def mesh_footprint(n_vertices: int, n_tri: int, owns_inputs: bool = False) -> int:
    return int(load_library().polylla_mesh_footprint(n_vertices, n_tri, 1 if owns_inputs else 0))


def mesh_set_size(mesh: int, n_vertices: int, n_tri: int):
    _check(load_library().polylla_mesh_set_size(mesh, n_vertices, n_tri), "polylla_mesh_set_size")


def mesh_inputs(mesh: int, n_vertices: int, n_tri: int):
    """Views (xy int64 [2n], tri int32 [3m], twin int32 [3m]) of a host-created handle's
    device inputs."""
    a, b, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load_library().polylla_mesh_inputs(mesh, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(c)), "polylla_mesh_inputs")
    return (_view(a.value, 2 * n_vertices, "<i8", torch.int64),
            _view(b.value, 3 * n_tri, "<i4", torch.int32),
            _view(c.value, 3 * n_tri, "<i4", torch.int32))


def get_polygons_async(mesh: int):
    """Raw device pointers (off, vtx, counts[2], error) of the latest CSR, no sync."""
    a, b, c, d = (ctypes.c_void_p() for _ in range(4))
    _check(load_library().polylla_get_polygons_async(mesh, ctypes.byref(a), ctypes.byref(b),
                                                     ctypes.byref(c), ctypes.byref(d)),
           "polylla_get_polygons_async")
    return a.value, b.value, c.value, d.value


def server_create(budget_bytes: int, max_slots: int) -> int:
    out = ctypes.c_void_p()
    _check(load_library().polylla_server_create(budget_bytes, max_slots, ctypes.byref(out)),
           "polylla_server_create")
    return out.value


def _hptr(t: torch.Tensor, dtype: torch.dtype, name: str) -> int:
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous host {dtype} tensor")
    return t.data_ptr()


def server_submit(server: int, xy: torch.Tensor, tri: torch.Tensor, twin: torch.Tensor,
                  off_out: torch.Tensor, vtx_out: torch.Tensor) -> int:
    """Queue one mesh (host tensors, pinned for overlap; kept alive by the caller until
    its result is polled); returns the request id."""
    rid = ctypes.c_int64()
    n, m = xy.numel() // 2, tri.numel() // 3
    if off_out.numel() < m + 1 or vtx_out.numel() < 3 * m:
        raise ValueError("output buffers need m + 1 offsets and 3m vertices")
    _check(load_library().polylla_server_submit(
        server, _hptr(xy, torch.int64, "xy"), n, _hptr(tri, torch.int32, "tri"),
        None if twin is None else _hptr(twin, torch.int32, "twin"), m,
        _hptr(off_out, torch.int64, "off_out"),
        _hptr(vtx_out, torch.int32, "vtx_out"), ctypes.byref(rid)), "polylla_server_submit")
    return rid.value


def server_poll(server: int, cap: int = 256, wait_us: int = 0) -> list:
    buf = (Result * cap)()
    k = load_library().polylla_server_poll(server, buf, cap, wait_us)
    if k < 0:
        raise PolyllaError(1, "polylla_server_poll")
    return [{f: getattr(buf[i], f) for f, _ in Result._fields_ if f != "reserved"}
            for i in range(k)]


def server_info(server: int) -> dict:
    s = ServerStats()
    _check(load_library().polylla_server_info(server, ctypes.byref(s)), "polylla_server_info")
    return s.as_dict()


def server_cancel(server: int, rid: int) -> bool:
    """Cancel a queued request; False when it was already admitted (it runs on)."""
    code = load_library().polylla_server_cancel(server, rid)
    if code == 7:  # POLYLLA_ERR_STATE
        return False
    _check(code, "polylla_server_cancel")
    return True


def debug_fail_alloc(k: int):
    """Failure injection for tests: the k-th device allocation from now on fails
    (k <= 0: off)."""
    load_library().polylla_debug_fail_alloc(k)


def debug_rare_paths(mesh: int, enable: bool = True):
    """Test switch: the reparation takes its repeated-vertex paths on every
    polygon (same polygons; see the header)."""
    _check(load_library().polylla_debug_rare_paths(mesh, int(enable)), "polylla_debug_rare_paths")


def set_one_block(mesh: int, max_triangles: int):
    """polylla_run meshes a mesh of at most max_triangles triangles in one thread
    block (0: always the multi-kernel path)."""
    _check(load_library().polylla_set_one_block(mesh, int(max_triangles)), "polylla_set_one_block")


def debug_split_by_pieces(mesh: int, enable: bool = True):
    """Test switch: the one-block path splits every polygon piece by piece (same
    polygons; see the header)."""
    _check(load_library().polylla_debug_split_by_pieces(mesh, int(enable)),
           "polylla_debug_split_by_pieces")


def one_block_limit() -> int:
    return int(load_library().polylla_one_block_limit())


def server_destroy(server: int):
    _check(load_library().polylla_server_destroy(server), "polylla_server_destroy")


# ------------------------------------------------------------------ convenience
class Mesh:
    """Owns a handle over device tensors (kept alive here) and runs the phases."""

    def __init__(self, xy: torch.Tensor, tri: torch.Tensor, twin: torch.Tensor,
                 validate: bool = True, stream=None):
        self.xy, self.tri, self.twin = xy, tri, twin
        self.m = tri.numel() // 3
        self.handle = mesh_create(xy, tri, twin, VALIDATE if validate else 0, stream)

    def label(self, stream=None):
        label(self.handle, stream)

    def seeds(self, stream=None):
        seeds(self.handle, stream)

    def traverse(self, stream=None):
        traverse(self.handle, stream)

    def repair(self, stream=None):
        repair(self.handle, stream)

    def repair_host(self, stream=None):
        repair_host(self.handle, stream)

    def run(self, stream=None):
        run(self.handle, stream)

    def set_one_block(self, max_triangles: int):
        set_one_block(self.handle, max_triangles)

    def labels(self) -> torch.Tensor:
        return get_labels(self.handle, self.m)

    def seed_list(self) -> torch.Tensor:
        return get_seeds(self.handle)

    def polygons(self):
        return get_polygons(self.handle)

    def lepp(self, stream=None):
        lepp(self.handle, stream)
        return get_lepp(self.handle, self.m)

    def stats(self) -> dict:
        return get_stats(self.handle)

    def close(self):
        if self.handle:
            mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns a batch handle over concatenated device tensors (kept alive here)."""

    def __init__(self, xy: torch.Tensor, vtx_off: torch.Tensor, tri: torch.Tensor,
                 twin: torch.Tensor, tri_off: torch.Tensor, validate: bool = True, stream=None):
        self.xy, self.vtx_off, self.tri, self.twin, self.tri_off = xy, vtx_off, tri, twin, tri_off
        self.n_meshes = vtx_off.numel() - 1
        self.handle = batch_create(xy, vtx_off, tri, twin, tri_off,
                                   VALIDATE if validate else 0, stream)

    def tune(self, reps: int = 3, stream=None):
        return batch_tune(self.handle, reps, stream)

    def run(self, schedule: int = SCHEDULE_TUNED, stream=None):
        batch_run(self.handle, schedule, stream)

    def polygons(self, mesh: int):
        return batch_get(self.handle, mesh)

    def all_polygons(self):
        return batch_get_all(self.handle, self.n_meshes)

    def stats(self) -> dict:
        return batch_stats(self.handle)

    def close(self):
        if self.handle:
            batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_from_numpy(cat: dict, device: str = "cuda", validate: bool = True, stream=None) -> Batch:
    """Upload concatenated meshes (xy, vtx_off, tri, tri_off, twin numpy arrays, ids local
    to each mesh) and create a batch handle."""
    def dev(a, dt):
        return torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
    return Batch(dev(cat["xy"], torch.int64), dev(cat["vtx_off"], torch.int64),
                 dev(cat["tri"], torch.int32), dev(cat["twin"], torch.int32),
                 dev(cat["tri_off"], torch.int64), validate=validate, stream=stream)


class Server:
    """A server handle; keeps each request's host tensors alive until it is polled."""

    def __init__(self, budget_bytes: int, max_slots: int = 32):
        self.handle = server_create(budget_bytes, max_slots)
        self.live = {}

    def submit(self, xy: torch.Tensor, tri: torch.Tensor, twin: torch.Tensor,
               off_out: torch.Tensor | None = None, vtx_out: torch.Tensor | None = None) -> int:
        m = tri.numel() // 3
        pin = torch.cuda.is_available()
        if off_out is None:
            off_out = torch.empty(m + 1, dtype=torch.int64, pin_memory=pin)
        if vtx_out is None:
            vtx_out = torch.empty(3 * m, dtype=torch.int32, pin_memory=pin)
        rid = server_submit(self.handle, xy, tri, twin, off_out, vtx_out)
        self.live[rid] = (xy, tri, twin, off_out, vtx_out)
        return rid

    def poll(self, cap: int = 256, wait_us: int = 0) -> list:
        """Completed results, each with its CSR (off, vtx) as host tensors."""
        out = server_poll(self.handle, cap, wait_us)
        for r in out:
            _, _, _, off, vtx = self.live.pop(r["id"])
            if r["status"] == 0:
                r["off"] = off[:r["n_poly"] + 1]
                r["vtx"] = vtx[:r["n_vtx"]]
        return out

    def cancel(self, rid: int) -> bool:
        return server_cancel(self.handle, rid)

    def info(self) -> dict:
        return server_info(self.handle)

    def close(self):
        if self.handle:
            server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_numpy(mesh: dict, device: str = "cuda", validate: bool = True, stream=None) -> Mesh:
    """Upload a generated mesh dict (xy, tri, twin numpy arrays) and create a handle."""
    xy = torch.as_tensor(mesh["xy"]).to(device=device, dtype=torch.int64).contiguous()
    tri = torch.as_tensor(mesh["tri"]).to(device=device, dtype=torch.int32).contiguous()
    twin = torch.as_tensor(mesh["twin"]).to(device=device, dtype=torch.int32).contiguous()
    return Mesh(xy, tri, twin, validate=validate, stream=stream)
