"""Python binding of libalsub with the C ABI's names (argument marshalling only).

PyTorch provides device memory and streams; every step of the subdivision runs in libalsub's
CUDA kernels. Without a loadable libalsub.so every call raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

SCHEMES = {"cc": 0, "loop": 1, "sqrt3": 2, "catmull-clark": 0}


class AlsubError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib():
    return _lib.load()


def _check(st: int):
    if st:
        L = lib()
        raise AlsubError(st, L.alsub_last_error().decode() or L.alsub_status_string(st).decode())


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def plan(scheme: str, V: int, F: int, nnz: int, levels: int, boundary: int = 0) -> np.ndarray:
    """Closed-form (V, F, nnz, E) per level (host only); ``boundary`` = boundary edges of an open
    Catmull-Clark or Loop mesh (alsub_plan_open)."""
    out = np.zeros(4 * (levels + 1), dtype=np.int64)
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if boundary:
        _check(lib().alsub_plan_open(SCHEMES[scheme], V, F, nnz, boundary, levels, p))
    else:
        _check(lib().alsub_plan(SCHEMES[scheme], V, F, nnz, levels, p))
    return out.reshape(levels + 1, 4)


def plan_bytes(scheme: str, V: int, F: int, nnz: int, levels: int, creases: int = 0,
               sigma_max: float = 0.0, boundary: int = 0) -> int:
    """alsub_plan_bytes: device bytes alsub_topology_create allocates (host only)."""
    b = ctypes.c_size_t()
    _check(lib().alsub_plan_bytes(SCHEMES[scheme], V, F, nnz, boundary, creases, ctypes.c_float(sigma_max),
                                  levels, ctypes.byref(b)))
    return b.value


def copy_to_host(ptr: int, nbytes: int, dtype, count: int, stream=None) -> np.ndarray:
    out = np.empty(count, dtype=dtype)
    if nbytes:
        _check(lib().alsub_copy(out.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(ptr), nbytes,
                                ctypes.c_void_p(_stream(stream))))
    return out


class DeviceAllocator:
    """An alsub_allocator backed by PyTorch's caching allocator (blocks come from and go back to
    torch's pool on the stream the library names). Keeps count of the blocks it holds; it must
    outlive every handle made with it (the handles keep a reference)."""

    def __init__(self, fail: bool = False):
        self.live, self.allocs, self.frees, self.bytes_live, self.fail = {}, 0, 0, 0, fail

        def _alloc(nbytes, ctx, stream):
            if self.fail:
                return None
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=s)
            self.live[p] = int(nbytes)
            self.allocs += 1
            self.bytes_live += int(nbytes)
            return p

        def _free(ptr, ctx, stream):
            self.bytes_live -= self.live.pop(ptr)
            self.frees += 1
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_fn, self._free_fn = _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)
        self.struct = _lib.Allocator(self._alloc_fn, self._free_fn, None)


class Mesh:
    """alsub_mesh_create / alsub_mesh_create_ex / alsub_mesh_destroy."""

    def __init__(self, scheme: str, V: int, F: int, fv, off=None, crease_verts=None,
                 crease_sharp=None, stream=None, allocator: DeviceAllocator | None = None):
        self.scheme = scheme
        fv = np.ascontiguousarray(fv, dtype=np.int32)
        off = None if off is None else np.ascontiguousarray(off, dtype=np.int32)
        cv = np.ascontiguousarray(crease_verts if crease_verts is not None else np.zeros((0, 2)),
                                  dtype=np.int32).reshape(-1)
        cs = np.ascontiguousarray(crease_sharp if crease_sharp is not None else np.zeros(0),
                                  dtype=np.float32).reshape(-1)
        self.V, self.F, self.nnz = int(V), int(F), int(fv.size)
        self._h = ctypes.c_void_p()
        self._allocator = allocator
        _check(lib().alsub_mesh_create_ex(SCHEMES[scheme], self.V, self.F, _ptr(off), _ptr(fv),
                                          int(cs.size), _ptr(cv) if cs.size else None,
                                          _ptr(cs) if cs.size else None,
                                          ctypes.byref(allocator.struct) if allocator else None,
                                          ctypes.c_void_p(_stream(stream)), ctypes.byref(self._h)))
        b = ctypes.c_int64()
        _check(lib().alsub_mesh_boundary_edges(self._h, ctypes.byref(b)))
        self.boundary_edges = int(b.value)

    @classmethod
    def _wrap(cls, h: ctypes.c_void_p, allocator=None) -> "Mesh":
        """A Mesh object around a handle the library made (an extracted or reordered mesh)."""
        self = cls.__new__(cls)
        self._h = h
        self._allocator = allocator
        sch, V, F, nnz, K = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().alsub_mesh_info(h, ctypes.byref(sch), ctypes.byref(V), ctypes.byref(F), ctypes.byref(nnz),
                                     ctypes.byref(K)))
        self.scheme = {v: k for k, v in SCHEMES.items()}[sch.value]
        self.V, self.F, self.nnz, self.K = V.value, F.value, nnz.value, K.value
        b = ctypes.c_int64()
        _check(lib().alsub_mesh_boundary_edges(h, ctypes.byref(b)))
        self.boundary_edges = int(b.value)
        return self

    def reorder(self, stream=None) -> "Mesh":
        """alsub_mesh_reorder (Sec. 4.5): the same mesh with its vertices in reverse Cuthill-McKee
        order and its faces sorted by their least new vertex; maps() and gather() relate it to this
        one. The breadth-first levels it took are in `.rcm_levels`."""
        h, lv = ctypes.c_void_p(), ctypes.c_int32()
        _check(lib().alsub_mesh_reorder(self._h, ctypes.c_void_p(_stream(stream)), ctypes.byref(h), ctypes.byref(lv)))
        out = Mesh._wrap(h, self._allocator)
        out.rcm_levels = int(lv.value)
        return out

    def arrays(self, stream=None) -> dict:
        """alsub_mesh_arrays, copied to the host: off, fv, crease_verts (K x 2), crease_sharp."""
        o, f, cv, cs = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().alsub_mesh_arrays(self._h, ctypes.byref(o), ctypes.byref(f), ctypes.byref(cv), ctypes.byref(cs)))
        Kc = ctypes.c_int64()
        _check(lib().alsub_mesh_info(self._h, None, None, None, None, ctypes.byref(Kc)))
        K = int(Kc.value)
        return dict(V=self.V, F=self.F,
                    off=copy_to_host(o.value, 4 * (self.F + 1), np.int32, self.F + 1, stream),
                    fv=copy_to_host(f.value, 4 * self.nnz, np.int32, self.nnz, stream),
                    crease_verts=copy_to_host(cv.value, 8 * K, np.int32, 2 * K, stream).reshape(-1, 2),
                    crease_sharp=copy_to_host(cs.value, 4 * K, np.float32, K, stream))

    def maps(self):
        """(vertex map int32[V], face map int32[F]) of an extracted or reordered mesh: source vertex /
        face ids."""
        vm, fm = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().alsub_mesh_extract_maps(self._h, ctypes.byref(vm), ctypes.byref(fm)))
        return (copy_to_host(vm.value, 4 * self.V, np.int32, self.V),
                copy_to_host(fm.value, 4 * self.F, np.int32, self.F))

    def gather(self, P: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        """alsub_mesh_gather: this extracted or reordered mesh's rows of the source's positions."""
        assert P.is_cuda and P.dtype == torch.float32 and P.is_contiguous()
        if out is None:
            out = torch.empty((self.V, 3), dtype=torch.float32, device=P.device)
        _check(lib().alsub_mesh_gather(self._h, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(_stream(stream))))
        return out

    @classmethod
    def from_dict(cls, m: dict, scheme: str | None = None, stream=None, allocator=None) -> "Mesh":
        return cls(scheme or m.get("scheme", "cc"), m["V"], m["F"], m["fv"], m["off"],
                   m.get("crease_verts"), m.get("crease_sharp"), stream, allocator)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _check(lib().alsub_mesh_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass


class Topology:
    """A refined topology: alsub_topology_create / alsub_refine_topology and the per-level calls."""

    def __init__(self, mesh: Mesh, levels: int, build: bool = True, stream=None):
        self.mesh = mesh          # the mesh must outlive the topology
        self.levels = int(levels)
        self._h = ctypes.c_void_p()
        fn = lib().alsub_refine_topology if build else lib().alsub_topology_create
        _check(fn(mesh.handle, self.levels, ctypes.c_void_p(_stream(stream)), ctypes.byref(self._h)))
        self.counts = [self.level_counts(l) for l in range(self.levels + 1)]

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _check(lib().alsub_topology_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def status(self):
        _check(lib().alsub_topology_status(self._h))

    def level_counts(self, level: int) -> dict:
        V, F, nnz, E = (ctypes.c_int64() for _ in range(4))
        _check(lib().alsub_topology_level(self._h, level, ctypes.byref(V), ctypes.byref(F),
                                          ctypes.byref(nnz), ctypes.byref(E), None, None))
        return dict(V=V.value, F=F.value, nnz=nnz.value, E=E.value)

    def faces(self, level: int, stream=None) -> np.ndarray:
        """Face table of a level as int32[nnz] (host copy)."""
        off, fv = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().alsub_topology_level(self._h, level, None, None, None, None,
                                          ctypes.byref(off), ctypes.byref(fv)))
        n = self.counts[level]["nnz"]
        return copy_to_host(fv.value, 4 * n, np.int32, n, stream)

    def face_table_ptr(self, level: int) -> int:
        fv = ctypes.c_void_p()
        _check(lib().alsub_topology_level(self._h, level, None, None, None, None, None,
                                          ctypes.byref(fv)))
        return fv.value

    def creases(self, level: int, stream=None):
        """(int32[K, 2] endpoints, float32[K] sharpness) of a level (synchronises)."""
        K = ctypes.c_int32()
        cv, cs = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().alsub_topology_creases(self._h, level, ctypes.byref(K), ctypes.byref(cv),
                                            ctypes.byref(cs)))
        k = K.value
        if k == 0:
            return np.zeros((0, 2), np.int32), np.zeros(0, np.float32)
        return (copy_to_host(cv.value, 8 * k, np.int32, 2 * k, stream).reshape(k, 2),
                copy_to_host(cs.value, 4 * k, np.float32, k, stream))

    def scratch_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().alsub_refine_vertices_scratch_bytes(self._h, ctypes.byref(b)))
        return b.value

    def bytes(self) -> int:
        """alsub_topology_bytes: device bytes the handle holds."""
        b = ctypes.c_size_t()
        _check(lib().alsub_topology_bytes(self._h, ctypes.byref(b)))
        return b.value

    def _run(self, fn, P0: torch.Tensor, out, scratch, stream):
        assert P0.is_cuda and P0.dtype == torch.float32 and P0.is_contiguous()
        VL = self.counts[-1]["V"]
        if out is None:
            out = torch.empty((VL, 3), dtype=torch.float32, device=P0.device)
        assert out.is_contiguous() and out.numel() == 3 * VL
        sp = None if scratch is None else ctypes.c_void_p(scratch.data_ptr())
        _check(fn(self._h, ctypes.c_void_p(P0.data_ptr()), ctypes.c_void_p(out.data_ptr()), sp,
                  ctypes.c_void_p(_stream(stream))))
        return out

    def refine_vertices(self, P0: torch.Tensor, out=None, scratch=None, stream=None) -> torch.Tensor:
        """alsub_refine_vertices: eval of all levels on the built topology."""
        return self._run(lib().alsub_refine_vertices, P0, out, scratch, stream)

    def refine_vertices_static(self, P0: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        """alsub_refine_vertices_static: the same eval with the library's fixed scratch array."""
        assert P0.is_cuda and P0.dtype == torch.float32 and P0.is_contiguous()
        VL = self.counts[-1]["V"]
        if out is None:
            out = torch.empty((VL, 3), dtype=torch.float32, device=P0.device)
        assert out.is_contiguous() and out.numel() == 3 * VL
        _check(lib().alsub_refine_vertices_static(self._h, ctypes.c_void_p(P0.data_ptr()),
                                                  ctypes.c_void_p(out.data_ptr()),
                                                  ctypes.c_void_p(_stream(stream))))
        return out

    def set_timing(self, capacity: int):
        """alsub_topology_set_timing: record per-level CUDA events for the next `capacity` calls."""
        _check(lib().alsub_topology_set_timing(self._h, int(capacity)))

    def timings(self):
        """alsub_topology_timings -> (ms per stage [level-0 build, level 0..L-1], calls, launches)."""
        ms = np.zeros(self.levels + 1, np.float64)
        calls, launches = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().alsub_topology_timings(self._h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            ctypes.byref(calls), ctypes.byref(launches)))
        return ms, calls.value, launches.value

    def subdivide(self, P0: torch.Tensor, out=None, scratch=None, stream=None) -> torch.Tensor:
        """alsub_subdivide: rebuild the topology and refine the vertices, fused per level."""
        return self._run(lib().alsub_subdivide, P0, out, scratch, stream)

    def extract(self, level: int = 0, select: torch.Tensor | None = None, rings: int = 2, stream=None) -> Mesh:
        """alsub_topology_extract (selective subdivision, Sec. 3.4): the region of a level around
        the selected vertices (uint8 device mask; None: extraordinary vertices and crease ends)."""
        h = ctypes.c_void_p()
        sel = None if select is None else ctypes.c_void_p(select.data_ptr())
        if select is not None:
            assert select.is_cuda and select.dtype == torch.uint8 and select.numel() == self.counts[level]["V"]
        _check(lib().alsub_topology_extract(self._h, int(level), sel, int(rings), ctypes.c_void_p(_stream(stream)),
                                            ctypes.byref(h)))
        return Mesh._wrap(h, getattr(self.mesh, "_allocator", None))

    def regular_faces(self, level: int = 0, stream=None) -> torch.Tensor:
        """alsub_topology_regular_faces: uint8 device mask of the level's regular (bicubic) faces."""
        flags = torch.empty(self.counts[level]["F"], dtype=torch.uint8, device="cuda")
        n = ctypes.c_int64()
        _check(lib().alsub_topology_regular_faces(self._h, int(level), ctypes.c_void_p(flags.data_ptr()),
                                                  ctypes.byref(n), ctypes.c_void_p(_stream(stream))))
        return flags

    def eval_patches(self, level: int, faces: torch.Tensor, P: torch.Tensor, samples: int, out=None,
                     stream=None) -> torch.Tensor:
        """alsub_topology_eval_patches: float32[n, samples, samples, 3] samples of the bicubic patches
        of `faces` (int32 device tensor) from the level's positions P (device, packed xyz)."""
        assert faces.is_cuda and faces.dtype == torch.int32 and P.is_cuda and P.dtype == torch.float32
        n = faces.numel()
        if out is None:
            out = torch.empty((n, samples, samples, 3), dtype=torch.float32, device="cuda")
        _check(lib().alsub_topology_eval_patches(self._h, int(level), n, ctypes.c_void_p(faces.data_ptr()),
                                                 ctypes.c_void_p(P.data_ptr()), int(samples),
                                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream(stream))))
        return out

    def set_edits(self, level: int, vid=None, offsets=None, stream=None):
        """alsub_topology_set_edits: offsets added to vertices of `level` after it is refined
        (None clears the level's edits). vid int32[n], offsets float32[n, 3]; host or device."""
        if vid is None or len(vid) == 0:
            _check(lib().alsub_topology_set_edits(self._h, int(level), 0, None, None, ctypes.c_void_p(_stream(stream))))
            return

        def ptr(a, dt):
            if isinstance(a, torch.Tensor):
                assert a.dtype == dt and a.is_contiguous()
                return a, a.data_ptr()
            a = np.ascontiguousarray(a, dtype={torch.int32: np.int32, torch.float32: np.float32}[dt])
            return a, a.ctypes.data

        v, pv = ptr(vid, torch.int32)
        o, po = ptr(offsets, torch.float32)
        n = len(v)
        assert (o.numel() if isinstance(o, torch.Tensor) else o.size) == 3 * n
        _check(lib().alsub_topology_set_edits(self._h, int(level), n, ctypes.c_void_p(pv), ctypes.c_void_p(po),
                                              ctypes.c_void_p(_stream(stream))))

    def subdivide_host(self, P0, out=None, stream=None):
        """alsub_subdivide_host: host positions in, host positions out (CPU tensors or numpy
        arrays, float32, contiguous; page-locked tensors are copied by DMA). The result is in
        ``out`` once ``stream`` (default: torch's current stream) has completed."""
        VL = self.counts[-1]["V"]
        if out is None:
            out = torch.empty((VL, 3), dtype=torch.float32).pin_memory()
        for a in (P0, out):
            if isinstance(a, torch.Tensor):
                assert not a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()
            else:
                assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
        def size(a):
            return a.size if isinstance(a, np.ndarray) else a.numel()

        assert size(P0) == 3 * self.counts[0]["V"] and size(out) == 3 * VL

        def ptr(a):
            return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data

        _check(lib().alsub_subdivide_host(self._h, ctypes.c_void_p(ptr(P0)), ctypes.c_void_p(ptr(out)),
                                          ctypes.c_void_p(_stream(stream))))
        return out


class Operator:
    """alsub_build_operator and friends: R_l per level and/or the composite R = R_{L-1}...R_0."""

    CHAIN, COMPOSE, TRANSPOSE, MATRIX_FREE, STACKED = 1, 2, 4, 8, 16

    def __init__(self, topo: Topology, chain: bool = True, compose: bool = False,
                 transpose: bool = False, matrix_free: bool = False, stream=None):
        self.topo = topo          # the topology must outlive the operator
        flags = (self.CHAIN if chain else 0) | (self.COMPOSE if compose else 0) | \
            (self.TRANSPOSE if transpose else 0) | (self.MATRIX_FREE if matrix_free else 0)
        self._h = ctypes.c_void_p()
        _check(lib().alsub_build_operator(topo.handle, flags, ctypes.c_void_p(_stream(stream)),
                                          ctypes.byref(self._h)))

    def close(self):
        if self._h:
            _check(lib().alsub_operator_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _sizes(self):
        """(output points, control points)."""
        return self.topo.counts[-1]["V"], self.topo.counts[0]["V"]

    def bytes(self) -> int:
        """alsub_operator_bytes: device bytes the operator holds."""
        b = ctypes.c_size_t()
        _check(lib().alsub_operator_bytes(self._h, ctypes.byref(b)))
        return b.value

    def info(self, level: int = -1) -> dict:
        rows, cols, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().alsub_operator_info(self._h, level, ctypes.byref(rows), ctypes.byref(cols),
                                         ctypes.byref(nnz), None, None, None))
        return dict(rows=rows.value, cols=cols.value, nnz=nnz.value)

    def csr(self, level: int = -1, stream=None):
        """Host copies (rowptr int64[rows+1], col int32[nnz], w float32[nnz]) of one matrix."""
        rows, cols, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rp, cl, w = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().alsub_operator_info(self._h, level, ctypes.byref(rows), ctypes.byref(cols),
                                         ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(cl),
                                         ctypes.byref(w)))
        n, z = rows.value, nnz.value
        return (copy_to_host(rp.value, 8 * (n + 1), np.int64, n + 1, stream),
                copy_to_host(cl.value, 4 * z, np.int32, z, stream),
                copy_to_host(w.value, 4 * z, np.float32, z, stream))

    def apply(self, P0: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        """alsub_apply_operator: P_L = R P_0."""
        assert P0.is_cuda and P0.dtype == torch.float32 and P0.is_contiguous()
        VL = self._sizes()[0]
        if out is None:
            out = torch.empty((VL, 3), dtype=torch.float32, device=P0.device)
        _check(lib().alsub_apply_operator(self._h, ctypes.c_void_p(P0.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream(stream))))
        return out

    def apply_transpose(self, gL: torch.Tensor, out=None, stream=None) -> torch.Tensor:
        """alsub_apply_operator_transpose: g_0 = R^T g_L."""
        assert gL.is_cuda and gL.dtype == torch.float32 and gL.is_contiguous()
        V0 = self._sizes()[1]
        if out is None:
            out = torch.empty((V0, 3), dtype=torch.float32, device=gL.device)
        _check(lib().alsub_apply_operator_transpose(self._h, ctypes.c_void_p(gL.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()),
                                                    ctypes.c_void_p(_stream(stream))))
        return out


class AdaptiveOperator(Operator):
    """alsub_build_adaptive_operator: one SpMV from the control points to the points of a chain of
    selective refinement rounds, topos[k] built on a mesh extracted from the last level of
    topos[k - 1]; ``stacked`` stacks every round's last level. The topologies are read during the
    build only."""

    def __init__(self, topos, stacked: bool = False, transpose: bool = False, stream=None):
        self.topo = None
        hs = (ctypes.c_void_p * len(topos))(*[t.handle.value for t in topos])
        flags = (self.TRANSPOSE if transpose else 0) | (self.STACKED if stacked else 0)
        self._h = ctypes.c_void_p()
        _check(lib().alsub_build_adaptive_operator(hs, len(topos), flags, ctypes.c_void_p(_stream(stream)),
                                                   ctypes.byref(self._h)))
        i = self.info(-1)
        self.rows, self.cols = i["rows"], i["cols"]

    def _sizes(self):
        return self.rows, self.cols


class Batch:
    """alsub_batch_*: vertex refinement of many built topologies in one launch per level and
    kernel class, replayed from a CUDA graph."""

    def __init__(self, topos, P0s, PLs=None):
        self.topos = list(topos)
        self.P0s = list(P0s)
        self.PLs = PLs if PLs is not None else [
            torch.empty((t.counts[-1]["V"], 3), dtype=torch.float32, device=p.device)
            for t, p in zip(self.topos, self.P0s)]
        n = len(self.topos)
        th = (ctypes.c_void_p * n)(*[t.handle.value for t in self.topos])
        p0 = (ctypes.c_void_p * n)(*[p.data_ptr() for p in self.P0s])
        pl = (ctypes.c_void_p * n)(*[p.data_ptr() for p in self.PLs])
        self._h = ctypes.c_void_p()
        _check(lib().alsub_batch_create(n, th, p0, pl, ctypes.byref(self._h)))

    def refine(self, stream=None):
        _check(lib().alsub_batch_refine(self._h, ctypes.c_void_p(_stream(stream))))
        return self.PLs

    def configure(self, block: int, blocks_per_sm: int):
        _check(lib().alsub_batch_configure(self._h, block, blocks_per_sm))

    def tune(self, stream=None):
        b, p, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        _check(lib().alsub_batch_tune(self._h, ctypes.c_void_p(_stream(stream)), ctypes.byref(b),
                                      ctypes.byref(p), ctypes.byref(ms)))
        return dict(block=b.value, blocks_per_sm=p.value, ms=ms.value)

    def launches(self) -> int:
        n = ctypes.c_int64()
        _check(lib().alsub_batch_launches(self._h, ctypes.byref(n)))
        return n.value

    def close(self):
        if self._h:
            _check(lib().alsub_batch_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


# ---------------------------------------------------------------------------- serving loop

REQ_FRAME, REQ_MESH = 0, 1
OK, ERR_OOM, ERR_TIMEOUT, ERR_NOT_READY = 0, 4, 5, 8


def _mesh_arrays(m: dict):
    fv = np.ascontiguousarray(m["fv"], dtype=np.int32)
    off = None if m.get("off") is None else np.ascontiguousarray(m["off"], dtype=np.int32)
    cv = np.ascontiguousarray(m["crease_verts"] if m.get("crease_verts") is not None else np.zeros((0, 2)),
                              dtype=np.int32).reshape(-1)
    cs = np.ascontiguousarray(m["crease_sharp"] if m.get("crease_sharp") is not None else np.zeros(0),
                              dtype=np.float32).reshape(-1)
    return fv, off, cv, cs


class Server:
    """alsub_serve_*: the serving loop (admission by HBM budget, slots on their own CUDA streams,
    resident topologies and operators, latency percentiles)."""

    def __init__(self, budget_bytes: int, max_slots: int = 8):
        self._h = ctypes.c_void_p()
        self._keep = {}
        _check(lib().alsub_serve_create(int(budget_bytes), int(max_slots), ctypes.byref(self._h)))

    FRAMES = {"eval": 0, "operator": 1, "fastest": 2, "operator_mf": 3}

    def register(self, m: dict, scheme: str, levels: int, frames: str = "operator_mf") -> int:
        """alsub_serve_register: make `m` a resident topology of `levels` steps whose frames are
        served by the eval kernels ("eval"), the cached composite operator ("operator"), the faster
        of those two ("fastest") or a matrix-free operator ("operator_mf", the stencils of the eval
        kernels behind alsub_apply_operator)."""
        fv, off, cv, cs = _mesh_arrays(m)
        rid = ctypes.c_int32()
        _check(lib().alsub_serve_register(self._h, SCHEMES[scheme], int(m["V"]), int(m["F"]), _ptr(off),
                                          _ptr(fv), int(cs.size), _ptr(cv) if cs.size else None,
                                          _ptr(cs) if cs.size else None, int(levels), self.FRAMES[frames],
                                          ctypes.byref(rid)))
        return rid.value

    def submit_frame(self, resident: int, P0: np.ndarray, out: np.ndarray | None = None) -> int:
        P0 = np.ascontiguousarray(P0, dtype=np.float32)
        r = _lib.Request(kind=REQ_FRAME, resident=int(resident), P0_host=P0.ctypes.data,
                         PL_host=None if out is None else out.ctypes.data)
        return self._submit(r, (P0, out))

    def submit_mesh(self, m: dict, scheme: str, levels: int, P0: np.ndarray | None = None,
                    out: np.ndarray | None = None, boundary_edges: int = 0) -> int:
        """A one-off mesh; ``boundary_edges`` as Mesh.boundary_edges (0 for a closed mesh)."""
        fv, off, cv, cs = _mesh_arrays(m)
        P0 = np.ascontiguousarray(m["P"] if P0 is None else P0, dtype=np.float32)
        r = _lib.Request(kind=REQ_MESH, scheme=SCHEMES[scheme], levels=int(levels), num_verts=int(m["V"]),
                         num_faces=int(m["F"]), face_offsets_host=None if off is None else off.ctypes.data,
                         face_verts_host=fv.ctypes.data, num_creases=int(cs.size),
                         num_boundary_edges=int(boundary_edges), crease_verts_host=cv.ctypes.data if cs.size else None,
                         crease_sharpness_host=cs.ctypes.data if cs.size else None,
                         P0_host=P0.ctypes.data, PL_host=None if out is None else out.ctypes.data)
        return self._submit(r, (P0, out))

    def _submit(self, r, keep) -> int:
        t = ctypes.c_uint64()
        _check(lib().alsub_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        if keep[1] is not None:
            self._keep[t.value] = keep[1]      # the caller's output buffer stays alive until polled
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0):
        """alsub_serve_poll: None while the request is in flight, else a dict with status, the
        positions (float32[V_L, 3]; a copy of the server's buffer unless the caller gave one) and
        the timestamps. The finished request is released."""
        res = _lib.Result()
        st = lib().alsub_serve_poll(self._h, int(ticket), int(timeout_us), ctypes.byref(res))
        if st in (ERR_TIMEOUT, ERR_NOT_READY):
            return None
        _check(st)
        P = None
        if res.status == OK:
            out = self._keep.get(ticket)
            if out is not None:
                P = out.reshape(-1, 3)
            else:
                n = 3 * res.num_verts
                P = np.ctypeslib.as_array(ctypes.cast(res.PL_host, ctypes.POINTER(ctypes.c_float)),
                                          shape=(n,)).copy().reshape(-1, 3)
        d = dict(status=res.status, kind=res.kind, P=P, submit_s=res.submit_s, start_s=res.start_s,
                 done_s=res.done_s, latency_s=res.done_s - res.submit_s)
        self._keep.pop(ticket, None)
        _check(lib().alsub_serve_release(self._h, int(ticket)))
        return d

    def pause(self, paused: bool = True):
        _check(lib().alsub_serve_pause(self._h, int(bool(paused))))

    def stats(self) -> dict:
        s = _lib.ServeStats()
        _check(lib().alsub_serve_stats_get(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in _lib.ServeStats._fields_}

    def close(self):
        if self._h:
            _check(lib().alsub_serve_destroy(self._h))
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
