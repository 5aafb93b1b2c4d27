"""AlSub oracle -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``alsub_oracle.c``: a plain, serial FP64 half-edge subdivider written
from the paper's classical rules (Catmull-Clark Sec. 3.1, creases Sec. 3.3, sqrt(3) Appendix A,
Loop Appendix B, boundaries Sec. 3.1/3.2), plus plain numpy restatements of selective subdivision
(Sec. 3.4: extraction, regular patches), hierarchical edits (Sec. 3.5) and mesh reordering
(Sec. 4.5: reverse Cuthill-McKee). Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import this package. It shares no code with the CUDA path and never calls it.

Every function follows its passage as cited in the C source. One part is "parity unpinned": the
crease vertex/edge rule reading (the paper delegates the rules to DeRose et al. 1998 and prints no
example); it is pinned only by its limit cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alsub_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCHEMES = {"cc": 0, "loop": 1, "sqrt3": 2}
ERRORS = {1: "invalid argument", 2: "non-manifold", 3: "boundary (open mesh)", 4: "out of memory",
          5: "invalid crease"}


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so FP32 crease arithmetic is exact)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            lib.or_run.argtypes = [ctypes.c_int] * 6 + [ctypes.c_int, ctypes.c_int, i32p, i32p, f64p,
                                                        ctypes.c_int, i32p, f32p,
                                                        ctypes.POINTER(ctypes.c_void_p)]
            lib.or_counts.argtypes = [ctypes.c_void_p, ctypes.c_int, np.ctypeslib.ndpointer(np.int64)]
            lib.or_faces.argtypes = [ctypes.c_void_p, ctypes.c_int, i32p, i32p]
            lib.or_positions.argtypes = [ctypes.c_void_p, ctypes.c_int, f64p]
            lib.or_creases.argtypes = [ctypes.c_void_p, ctypes.c_int, i32p, f32p]
            lib.or_operator.argtypes = [ctypes.c_void_p, ctypes.c_int, i32p, i32p, f64p]
            lib.or_free.argtypes = [ctypes.c_void_p]
            for f in ("or_run", "or_counts", "or_faces", "or_positions", "or_creases", "or_operator"):
                getattr(lib, f).restype = ctypes.c_int
            lib.or_free.restype = None
            _lib = lib
    return _lib


def subdivide(mesh: dict, levels: int, scheme: str | None = None, keep_all: bool = True,
              operator: bool = False, P0=None, patch: bool = False, start_level: int = 0) -> list[dict | None]:
    """Refine ``mesh`` ``levels`` times; returns one dict per level (None for levels not kept).

    Each dict holds V, F, nnz, E, K, off, fv, P (float64[V,3]), crease_verts, crease_sharp and,
    when ``operator`` is set and the level is below ``levels``, the operator R_l as COO
    (R_rows, R_cols, R_w) mapping level l to level l+1.

    ``patch``: the mesh is a patch cut out of a larger closed mesh (one level, any scheme); points
    whose rule reaches beyond the cut are NaN, every other point is the closed mesh's (the last
    level's E is not computed).

    ``start_level``: the level the input mesh is at (sqrt(3) alternates two kinds of step, the
    first of a pair from an even level).
    """
    lib = _load()
    scheme = scheme or mesh.get("scheme", "cc")
    off = np.ascontiguousarray(mesh["off"], dtype=np.int32)
    fv = np.ascontiguousarray(mesh["fv"], dtype=np.int32)
    P = np.ascontiguousarray(mesh["P"] if P0 is None else P0, dtype=np.float64).reshape(-1)
    cv = np.ascontiguousarray(mesh["crease_verts"], dtype=np.int32).reshape(-1)
    cs = np.ascontiguousarray(mesh["crease_sharp"], dtype=np.float32).reshape(-1)
    if cv.size == 0:
        cv = np.zeros(2, np.int32)
        cs_n = 0
        cs = np.zeros(1, np.float32)
    else:
        cs_n = cs.size
    h = ctypes.c_void_p()
    st = lib.or_run(SCHEMES[scheme], int(levels), int(keep_all), int(operator), int(patch), int(start_level),
                    int(mesh["V"]),
                    int(mesh["F"]), off, fv, P, cs_n, cv, cs, ctypes.byref(h))
    if st:
        raise OracleError(st)
    try:
        out = []
        for l in range(levels + 1):
            cnt = np.zeros(6, np.int64)
            if lib.or_counts(h, l, cnt):
                out.append(None)
                continue
            V, F, nnz, E, K, rnnz = (int(x) for x in cnt)
            d = dict(V=V, F=F, nnz=nnz, E=E, K=K)
            d["off"] = np.zeros(F + 1, np.int32)
            d["fv"] = np.zeros(max(nnz, 1), np.int32)
            lib.or_faces(h, l, d["off"], d["fv"])
            d["fv"] = d["fv"][:nnz]
            Pl = np.zeros(3 * V, np.float64)
            lib.or_positions(h, l, Pl)
            d["P"] = Pl.reshape(V, 3)
            cvl = np.zeros(2 * K + 2, np.int32)
            csl = np.zeros(K + 1, np.float32)
            lib.or_creases(h, l, cvl, csl)
            d["crease_verts"] = cvl[:2 * K].reshape(K, 2)
            d["crease_sharp"] = csl[:K]
            if operator and l < levels and rnnz > 0:
                rr = np.zeros(rnnz, np.int32)
                rc = np.zeros(rnnz, np.int32)
                rw = np.zeros(rnnz, np.float64)
                lib.or_operator(h, l, rr, rc, rw)
                d["R_rows"], d["R_cols"], d["R_w"] = rr, rc, rw
            out.append(d)
        return out
    finally:
        lib.or_free(h)


def operator_matrix(level: dict, n_cols: int):
    """The level's operator as a scipy.sparse CSR matrix (rows = next level's vertices)."""
    import scipy.sparse as sp
    n_rows = int(level["R_rows"].max()) + 1 if level["R_rows"].size else 0
    return sp.csr_matrix((level["R_w"], (level["R_rows"], level["R_cols"])), shape=(n_rows, n_cols))


def extract(mesh: dict, select=None, rings: int = 1, scheme: str = "cc") -> dict:
    """Extraction of selective subdivision (Sec. 3.4), written from its definition.

    The selected vertices x_0 (bool[V]; default: the extraordinary vertices, valence != 4 for
    Catmull-Clark or != 6 for Loop / sqrt(3) with valence = corners at the vertex, Eq. vo, among the
    vertices on no boundary edge, and both ends of every crease with sigma > 0) are propagated ``rings`` times: q_i = M^T x_i marks the faces
    with a selected vertex, x_{i+1} = M q_i the vertices of those faces. The extracted mesh keeps
    the faces of the last q (X-ring, columns of the identity: fmap, increasing) and their vertices
    (X, rows of the identity: vmap, increasing), M' = X M X-ring with the vertices renumbered, P' = X P.
    Where the region touches itself at a vertex only (two fans of kept faces there), every face
    around that vertex is kept too, repeatedly, so the extracted mesh is a manifold.
    A crease is kept when every face around both its ends is kept (so none touches the cut).
    """
    V, F = int(mesh["V"]), int(mesh["F"])
    off = np.asarray(mesh["off"], dtype=np.int64)
    fv = np.asarray(mesh["fv"], dtype=np.int64)
    cv = np.asarray(mesh.get("crease_verts", np.zeros((0, 2))), dtype=np.int64).reshape(-1, 2)
    cs = np.asarray(mesh.get("crease_sharp", np.zeros(0)), dtype=np.float32).reshape(-1)
    valence = np.bincount(fv, minlength=V)
    if select is None:
        # vertices on a boundary edge (an edge whose reverse direction is in no face) are not
        # extraordinary in this sense
        nxt = np.arange(1, fv.size + 1)
        nxt[off[1:] - 1] = off[:-1]
        a, b = fv, fv[nxt]
        fwd = set(zip(a.tolist(), b.tolist()))
        on_bnd = np.zeros(V, dtype=bool)
        for u, w in fwd:
            if (w, u) not in fwd:
                on_bnd[u] = on_bnd[w] = True
        x = (valence != (4 if scheme == "cc" else 6)) & ~on_bnd
        live = cs > 0
        x[cv[live, 0]] = True
        x[cv[live, 1]] = True
    else:
        x = np.asarray(select).astype(bool).copy()
    face_of = np.repeat(np.arange(F), np.diff(off))
    nxt = np.arange(1, fv.size + 1)
    nxt[off[1:] - 1] = off[:-1]
    q = np.zeros(F, dtype=bool)
    for _ in range(rings):
        q = np.zeros(F, dtype=bool)
        q[face_of[x[fv]]] = True                    # q = M^T x
        x = np.zeros(V, dtype=bool)
        x[fv[q[face_of]]] = True                    # x = M q
    # a vertex where the region touches itself (two or more fans of kept faces: as many boundary
    # edges of the region leave it) takes all its faces, until no such vertex is left
    while True:
        kc = np.flatnonzero(q[face_of])
        fwd = set(zip(fv[kc].tolist(), fv[nxt[kc]].tolist()))
        out_b = np.zeros(V, dtype=np.int64)
        for u, w in fwd:
            if (w, u) not in fwd:
                out_b[u] += 1
        pinch = out_b >= 2
        if not pinch.any():
            break
        q[face_of[pinch[fv]]] = True
    x = np.zeros(V, dtype=bool)
    x[fv[q[face_of]]] = True
    fmap = np.flatnonzero(q)
    vmap = np.flatnonzero(x)
    new_id = np.full(V, -1, dtype=np.int64)
    new_id[vmap] = np.arange(vmap.size)
    corners = np.flatnonzero(q[face_of])
    noff = np.zeros(fmap.size + 1, dtype=np.int64)
    noff[1:] = np.cumsum(np.diff(off)[fmap])
    kept_faces_at = np.bincount(fv[corners], minlength=V)
    inner = kept_faces_at == valence
    keep_c = (cs > 0) & inner[cv[:, 0]] & inner[cv[:, 1]] if cs.size else np.zeros(0, dtype=bool)
    out = dict(V=int(vmap.size), F=int(fmap.size), off=noff.astype(np.int32),
               fv=new_id[fv[corners]].astype(np.int32), vmap=vmap.astype(np.int32), fmap=fmap.astype(np.int32),
               crease_verts=new_id[cv[keep_c]].astype(np.int32).reshape(-1, 2), crease_sharp=cs[keep_c])
    if "P" in mesh:
        out["P"] = np.asarray(mesh["P"])[vmap]
    return out


def adaptive_operator(mesh: dict, rounds: int, rings: int = 2, scheme: str = "cc", stacked: bool = False):
    """The feature-adaptive subdivision operator as one matrix (Sec. 3.4, Fig. module_selective:
    the extraction matrices act on the vertex data before each refinement; composed into a single
    SpMV as Eq. singleSpMV does for uniform refinement and Sec. 5 "Adaptive Subdivision" evaluates
    it). Each round extracts ``rings`` rings around the selected vertices of the previous round's
    refined level (``extract`` with its default selection; its vmap gives X, row i = e_vmap[i])
    and refines them one level (the oracle's R_0 of the extracted mesh), so
        R = R^(n) X^(n) ... R^(1) X^(1)
    as scipy sparse products. ``stacked``: the identity of the control mesh, then every round's
    rows, stacked in round order. Returns a scipy CSR matrix over the control points."""
    import scipy.sparse as sp
    cur = dict(mesh, P=np.asarray(mesh["P"], dtype=np.float64))
    C = sp.identity(int(mesh["V"]), dtype=np.float64, format="csr")
    blocks = [C]
    for _ in range(rounds):
        e = extract(cur, None, rings, scheme=scheme)
        X = sp.csr_matrix((np.ones(e["V"]), (np.arange(e["V"]), e["vmap"])), shape=(e["V"], int(cur["V"])))
        lv = subdivide(e, 1, scheme, operator=True)
        R = sp.csr_matrix((lv[0]["R_w"], (lv[0]["R_rows"], lv[0]["R_cols"])), shape=(lv[1]["V"], e["V"]))
        C = (R @ (X @ C)).tocsr()
        cur = lv[1]
        blocks.append(C)
    return sp.vstack(blocks).tocsr() if stacked else C


def subdivide_edits(mesh: dict, levels: int, scheme: str, edits: dict) -> list[dict]:
    """Refinement with hierarchical edits (Sec. 3.5 "Other effects"): one level at a time, the
    offsets edits[l] = (vertex ids, float[n, 3]) added to level l's positions once it is refined,
    before the next level is computed from them. Returns the levels 0 .. levels."""
    cur = dict(mesh, P=np.asarray(mesh["P"], dtype=np.float64))
    out = [dict(cur, **subdivide(cur, 0, scheme)[0])]
    for l in range(1, levels + 1):
        nxt = subdivide(cur, 1, scheme)[1]
        if l in edits:
            vid, off = edits[l]
            P = nxt["P"].copy()
            P[np.asarray(vid)] += np.asarray(off, dtype=np.float64).reshape(-1, 3)
            nxt["P"] = P
        out.append(nxt)
        cur = nxt
    return out


def _cubic_bspline(t):
    """The uniform cubic B-spline N (support [0, 4], integer knots) by the Cox-de Boor recursion."""
    t = np.asarray(t, dtype=np.float64)

    def n(i, k):
        if k == 1:
            return ((t >= i) & (t < i + 1)).astype(np.float64)
        return ((t - i) / (k - 1)) * n(i, k - 1) + ((i + k - t) / (k - 1)) * n(i + 1, k - 1)
    return n(0, 4)


def regular_patches(level: dict, samples: int):
    """Regular faces of a Catmull-Clark level and their bicubic B-spline patches (Sec. 3.4: faces
    whose vertices all have valence 4 are bicubic patches whose limit surface is evaluated
    directly), written from the definitions.

    A face is regular when it is a quad, its 3 x 3 block of faces (the faces sharing a vertex with
    it) is 9 quads around 4 interior valence-4 vertices, and no crease with sigma > 0 has an end
    among the 16 vertices of the block. The control net: the face [v0, v1, v2, v3] spans grid
    cells (1..2, 1..2) with u along v0 -> v1 and v along v0 -> v3; every other vertex of the block
    gets its grid position from the faces it shares edges with. Returns (flags bool[F], {face:
    float[samples, samples, 3]}) with sample (b, a) = S(a / (s - 1), b / (s - 1)) and
    S(u, v) = sum_ij N(u + 3 - i) N(v + 3 - j) P_ij (N evaluated just inside its support at 1).
    """
    off = np.asarray(level["off"], dtype=np.int64)
    fv = np.asarray(level["fv"], dtype=np.int64)
    P = np.asarray(level["P"], dtype=np.float64)
    F, V = int(level["F"]), int(level["V"])
    faces = [list(fv[off[r]:off[r + 1]]) for r in range(F)]
    vfaces = [[] for _ in range(V)]
    for r, f in enumerate(faces):
        for v in f:
            vfaces[v].append(r)
    edge_faces = {}
    for r, f in enumerate(faces):
        for j in range(len(f)):
            edge_faces.setdefault(frozenset((f[j], f[(j + 1) % len(f)])), []).append(r)
    crease_v = set()
    cv = np.asarray(level.get("crease_verts", np.zeros((0, 2))), dtype=np.int64).reshape(-1, 2)
    cs = np.asarray(level.get("crease_sharp", np.zeros(0)), dtype=np.float32).reshape(-1)
    for (a, b), s in zip(cv, cs):
        if s > 0:
            crease_v.update((int(a), int(b)))
    flags = np.zeros(F, dtype=bool)
    grids = {}
    t = np.linspace(0.0, 1.0, samples)
    t[-1] = 1.0 - 1e-12                               # the support of N is half open
    B = np.stack([_cubic_bspline(t + 3 - i) for i in range(4)], axis=1)   # [samples, 4]
    for r, f in enumerate(faces):
        if len(f) != 4:
            continue
        block = sorted({q for v in f for q in vfaces[v]})
        if len(block) != 9 or any(len(faces[q]) != 4 for q in block):
            continue
        if any(len(vfaces[v]) != 4 for v in f):
            continue
        if any(len(edge_faces[frozenset((f[j], f[(j + 1) % 4]))]) != 2 for j in range(4)):
            continue
        # grid positions: the face's own vertices, then repeatedly a vertex of a block face whose
        # three other vertices are placed (the fourth corner of a unit square)
        pos = {f[0]: (1, 1), f[1]: (2, 1), f[2]: (2, 2), f[3]: (1, 2)}
        changed = True
        while changed:
            changed = False
            for q in block:
                g = faces[q]
                known = [v for v in g if v in pos]
                if len(known) == 3 and len(g) == 4:
                    miss = [v for v in g if v not in pos][0]
                    k = g.index(miss)
                    a, b, c = g[(k + 1) % 4], g[(k + 2) % 4], g[(k + 3) % 4]   # b is opposite miss
                    pa, pb, pc = np.array(pos[a]), np.array(pos[b]), np.array(pos[c])
                    pos[miss] = tuple(int(x) for x in pa + pc - pb)
                    changed = True
                elif len(known) == 2 and len(g) == 4:
                    # an edge p -> q of g is placed: g = [p, q, x, y] is the unit square on its left
                    for k in range(4):
                        p_, q_ = g[k], g[(k + 1) % 4]
                        if p_ in pos and q_ in pos:
                            d = np.array(pos[q_]) - np.array(pos[p_])
                            left = np.array([-d[1], d[0]])
                            pos[g[(k + 2) % 4]] = tuple(int(x) for x in np.array(pos[q_]) + left)
                            pos[g[(k + 3) % 4]] = tuple(int(x) for x in np.array(pos[p_]) + left)
                            changed = True
                            break
        if len(pos) != 16 or sorted(pos.values()) != [(i, j) for i in range(4) for j in range(4)]:
            continue
        if crease_v.intersection(pos.keys()):
            continue
        ctrl = np.zeros((4, 4, 3))
        for v, (i, j) in pos.items():
            ctrl[i, j] = P[v]
        flags[r] = True
        grids[r] = np.einsum("ai,bj,ijd->bad", B, B, ctrl)
    return flags, grids


def vertex_graph(mesh: dict) -> list[list[int]]:
    """The graph of the mesh Laplacian (Sec. 4.5): vertices u, w adjacent when an edge of some face
    joins them; each list increasing, without repeats."""
    V = int(mesh["V"])
    off = np.asarray(mesh["off"], dtype=np.int64)
    fv = np.asarray(mesh["fv"], dtype=np.int64)
    nbr = [set() for _ in range(V)]
    for f in range(len(off) - 1):
        ring = fv[off[f]:off[f + 1]].tolist()
        for i, u in enumerate(ring):
            w = ring[(i + 1) % len(ring)]
            if u != w:
                nbr[u].add(w)
                nbr[w].add(u)
    return [sorted(s) for s in nbr]


def cuthill_mckee(adj: list[list[int]]) -> np.ndarray:
    """Cuthill-McKee order (Cuthill and McKee 1969) of a graph: order[k] = the vertex labelled k.

    Each connected component starts at its unlabelled vertex of least degree (least index on ties);
    the labelled vertices are visited in label order, and each labels its unlabelled neighbours in
    increasing (degree, index). Components follow one another in the order their start vertices
    are found."""
    V = len(adj)
    deg = [len(a) for a in adj]
    label = [-1] * V
    order = []
    by_degree = sorted(range(V), key=lambda v: (deg[v], v))
    for s in by_degree:
        if label[s] >= 0:
            continue
        label[s] = len(order)
        order.append(s)
        head = label[s]
        while head < len(order):
            u = order[head]
            head += 1
            fresh = sorted((w for w in adj[u] if label[w] < 0), key=lambda w: (deg[w], w))
            for w in fresh:
                label[w] = len(order)
                order.append(w)
    return np.asarray(order, dtype=np.int64)


def bandwidth(adj: list[list[int]], new_id=None) -> int:
    """max |new_id[u] - new_id[w]| over the edges (the bandwidth of the Laplacian)."""
    b = 0
    for u, a in enumerate(adj):
        for w in a:
            b = max(b, abs(int(new_id[u] if new_id is not None else u) - int(new_id[w] if new_id is not None else w)))
    return b


def rcm_reorder(mesh: dict) -> dict:
    """Mesh reordering of Sec. 4.5: reverse Cuthill-McKee (George 1971: the Cuthill-McKee order
    reversed) on the graph of the mesh Laplacian permutes the vertices (the rows of M); the faces
    (the columns) are then sorted by their first non-zero row, i.e. by the least new index among
    their vertices, faces with the same least vertex keeping their input order. Each face keeps its
    corners in their cyclic order from the same first corner; creases keep their order with their
    ends renamed. vmap[new vertex] = old vertex, fmap[new face] = old face."""
    V, F = int(mesh["V"]), int(mesh["F"])
    off = np.asarray(mesh["off"], dtype=np.int64)
    fv = np.asarray(mesh["fv"], dtype=np.int64)
    order = cuthill_mckee(vertex_graph(mesh))
    vmap = order[::-1].copy()
    new_id = np.empty(V, dtype=np.int64)
    new_id[vmap] = np.arange(V)
    first = np.array([new_id[fv[off[f]:off[f + 1]]].min() for f in range(F)], dtype=np.int64)
    fmap = np.argsort(first, kind="stable")
    sizes = np.diff(off)[fmap]
    noff = np.zeros(F + 1, dtype=np.int64)
    noff[1:] = np.cumsum(sizes)
    nfv = np.concatenate([new_id[fv[off[f]:off[f + 1]]] for f in fmap]) if F else np.zeros(0, np.int64)
    cv = np.asarray(mesh.get("crease_verts", np.zeros((0, 2))), dtype=np.int64).reshape(-1, 2)
    cs = np.asarray(mesh.get("crease_sharp", np.zeros(0)), dtype=np.float32).reshape(-1)
    out = dict(V=V, F=F, off=noff.astype(np.int32), fv=nfv.astype(np.int32), vmap=vmap.astype(np.int32),
               fmap=fmap.astype(np.int32), crease_verts=new_id[cv].astype(np.int32).reshape(-1, 2),
               crease_sharp=cs.copy())
    if "P" in mesh:
        out["P"] = np.asarray(mesh["P"])[vmap]
    return out
