"""ctypes declarations of libalsub's C ABI (include/alsub.h). Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int32, c_int64, c_size_t, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
P = ctypes.POINTER
H = c_void_p  # opaque handles and raw pointers



ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_void_p)


class Allocator(ctypes.Structure):
    """alsub_allocator."""
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_void_p)]


class Request(ctypes.Structure):
    """alsub_request."""
    _fields_ = [("kind", c_int32), ("resident", c_int32), ("scheme", c_int32), ("levels", c_int32),
                ("num_verts", c_int32), ("num_faces", c_int32), ("face_offsets_host", c_void_p),
                ("face_verts_host", c_void_p), ("num_creases", c_int32), ("num_boundary_edges", c_int32),
                ("crease_verts_host", c_void_p),
                ("crease_sharpness_host", c_void_p), ("P0_host", c_void_p), ("PL_host", c_void_p)]


class Result(ctypes.Structure):
    """alsub_result."""
    _fields_ = [("status", c_int32), ("kind", c_int32), ("num_verts", c_int64), ("PL_host", c_void_p),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    """alsub_serve_stats."""
    _fields_ = [("completed", c_int64), ("failed", c_int64), ("queued", c_int64), ("in_flight", c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("throughput_rps", ctypes.c_double),
                ("hbm_budget", ctypes.c_uint64), ("hbm_in_use", ctypes.c_uint64), ("hbm_peak", ctypes.c_uint64),
                ("frames_operator", c_int64), ("frames_eval", c_int64), ("meshes", c_int64),
                ("host_start_ms_mean", ctypes.c_double), ("host_finish_ms_mean", ctypes.c_double),
                ("peak_in_flight", c_int64), ("device_overlap_peak", c_int64),
                ("host_start_frame_ms_mean", ctypes.c_double), ("host_start_mesh_ms_mean", ctypes.c_double)]


# name -> argtypes; every function returns alsub_status (int32) unless listed in _RESTYPE
SIGNATURES = {
    "alsub_last_error": [],
    "alsub_status_string": [c_int32],
    "alsub_copy": [c_void_p, c_void_p, c_size_t, c_void_p],
    "alsub_plan": [c_int32, c_int64, c_int64, c_int64, c_int32, P(c_int64)],
    "alsub_plan_open": [c_int32, c_int64, c_int64, c_int64, c_int64, c_int32, P(c_int64)],
    "alsub_mesh_boundary_edges": [c_void_p, P(c_int64)],
    "alsub_subdivide_host": [c_void_p, c_void_p, c_void_p, c_void_p],
    "alsub_topology_set_edits": [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p],
    "alsub_topology_regular_faces": [c_void_p, c_int32, c_void_p, P(c_int64), c_void_p],
    "alsub_topology_eval_patches": [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_void_p],
    "alsub_mesh_info": [c_void_p, P(c_int32), P(c_int64), P(c_int64), P(c_int64), P(c_int64)],
    "alsub_topology_extract": [c_void_p, c_int32, c_void_p, c_int32, c_void_p, P(c_void_p)],
    "alsub_mesh_reorder": [c_void_p, c_void_p, P(c_void_p), P(c_int32)],
    "alsub_mesh_arrays": [c_void_p, P(c_void_p), P(c_void_p), P(c_void_p), P(c_void_p)],
    "alsub_mesh_extract_maps": [c_void_p, P(c_void_p), P(c_void_p)],
    "alsub_mesh_gather": [c_void_p, c_void_p, c_void_p, c_void_p],
    "alsub_mesh_create": [c_int32, c_int32, c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                          c_void_p, P(H)],
    "alsub_mesh_create_ex": [c_int32, c_int32, c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                             P(Allocator), c_void_p, P(H)],
    "alsub_mesh_destroy": [H],
    "alsub_topology_create": [H, c_int32, c_void_p, P(H)],
    "alsub_refine_topology": [H, c_int32, c_void_p, P(H)],
    "alsub_topology_status": [H],
    "alsub_topology_level": [H, c_int32, P(c_int64), P(c_int64), P(c_int64), P(c_int64), P(c_void_p),
                             P(c_void_p)],
    "alsub_topology_creases": [H, c_int32, P(c_int32), P(c_void_p), P(c_void_p)],
    "alsub_topology_destroy": [H],
    "alsub_refine_vertices": [H, c_void_p, c_void_p, c_void_p, c_void_p],
    "alsub_refine_vertices_scratch_bytes": [H, P(c_size_t)],
    "alsub_subdivide": [H, c_void_p, c_void_p, c_void_p, c_void_p],
    "alsub_topology_set_timing": [H, c_int32],
    "alsub_topology_timings": [H, P(ctypes.c_double), P(c_int32), P(c_int64)],
    "alsub_refine_vertices_static": [H, c_void_p, c_void_p, c_void_p],
    "alsub_build_operator": [H, ctypes.c_uint32, c_void_p, P(H)],
    "alsub_build_adaptive_operator": [P(H), c_int32, ctypes.c_uint32, c_void_p, P(H)],
    "alsub_operator_info": [H, c_int32, P(c_int64), P(c_int64), P(c_int64), P(c_void_p), P(c_void_p),
                            P(c_void_p)],
    "alsub_apply_operator": [H, c_void_p, c_void_p, c_void_p],
    "alsub_apply_operator_transpose": [H, c_void_p, c_void_p, c_void_p],
    "alsub_operator_destroy": [H],
    "alsub_batch_create": [c_int32, c_void_p, c_void_p, c_void_p, P(H)],
    "alsub_batch_refine": [H, c_void_p],
    "alsub_batch_configure": [H, c_int32, c_int32],
    "alsub_batch_tune": [H, c_void_p, P(c_int32), P(c_int32), P(ctypes.c_float)],
    "alsub_batch_launches": [H, P(c_int64)],
    "alsub_batch_destroy": [H],
    "alsub_plan_bytes": [c_int32, c_int32, c_int32, c_int32, c_int32, c_int32, ctypes.c_float, c_int32,
                         P(c_size_t)],
    "alsub_topology_bytes": [H, P(c_size_t)],
    "alsub_operator_bytes": [H, P(c_size_t)],
    "alsub_serve_create": [c_size_t, c_int32, P(H)],
    "alsub_serve_register": [H, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                             c_int32, c_int32, P(c_int32)],
    "alsub_serve_submit": [H, P(Request), P(ctypes.c_uint64)],
    "alsub_serve_poll": [H, ctypes.c_uint64, c_int32, P(Result)],
    "alsub_serve_release": [H, ctypes.c_uint64],
    "alsub_serve_pause": [H, c_int32],
    "alsub_serve_stats_get": [H, P(ServeStats)],
    "alsub_serve_destroy": [H],
}
_RESTYPE = {"alsub_last_error": ctypes.c_char_p, "alsub_status_string": ctypes.c_char_p}

_lock = threading.Lock()
_lib = None


def load(build_if_stale: bool = True) -> ctypes.CDLL:
    """Load the in-tree libalsub.so (building it first if it is missing or stale).

    Raises RuntimeError when the library cannot be built or loaded: there is no fallback path.
    """
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_stale:
            try:
                path = _build.build()
            except Exception as e:  # noqa: BLE001 -- surface the compiler output
                if not os.path.exists(path):
                    raise RuntimeError(f"libalsub could not be built: {e}") from e
        if not os.path.exists(path):
            raise RuntimeError(f"libalsub not found at {path}; run paper_1809_06047_gb300.build")
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, c_int32)
        _lib = lib
        return lib
