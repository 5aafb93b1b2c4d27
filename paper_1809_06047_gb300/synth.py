"""Seeded synthetic control meshes (inputs only).

This module builds the input meshes that both the CUDA path and the CPU oracle consume. It holds
none of the subdivision arithmetic: it only places vertices on a torus, edits the connectivity of
the control mesh (quad merges, quad splits, triangle edge flips), tags crease edges and draws
jitter. Every random number comes from one counter-based splitmix64 stream (Steele, Lea and Flood
2014, as published by Vigna), so a draw is a pure function of (seed, counter).

The meshes stand in for the production models of the paper's result tables (Sec. 5, Tables
mesh_info_CC, mesh_info_L, mesh_info_S), which are not available:

* ``torus_cc_plain``  -- closed quad torus, all valence 4, no creases.
* ``torus_cc_mixed``  -- quad torus with quad pairs merged into hexagons, quads split into
  triangle pairs (valences 3..6) and a share of edges tagged with FP32 crease sharpness.
* ``torus_tri``       -- triangulated torus with a share of edges flipped (valences 4..8) and a
  share of edges infinitely sharp.
* ``tube_cc``, ``sheet_cc``, ``holed_cc_mixed`` -- open Catmull-Clark meshes (boundary loops,
  valence-2 corners, holes cut into the mixed torus) for the boundary rules; ``triangulate`` turns
  any of them into a Loop mesh (each n-gon a fan from its first corner).

A mesh is a dict with ``V``, ``F``, ``off`` (int32[F+1]), ``fv`` (int32[nnz], faces in CCW cyclic
order), ``P`` (float32[V,3]), ``crease_verts`` (int32[K,2]) and ``crease_sharp`` (float32[K]).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 0x180906047
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based splitmix64: draw i is mix(seed + (i + 1) * gamma)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.ctr = 0

    def next_u64(self, n: int) -> np.ndarray:
        i = np.arange(self.ctr + 1, self.ctr + 1 + n, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            z = self.seed + i * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) from the top 53 bits of each draw."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def permutation(self, n: int) -> np.ndarray:
        """A seeded permutation of range(n): stable argsort of n uniform keys."""
        return np.argsort(self.uniform(n), kind="stable").astype(np.int64)


def _torus_points(N: int, M: int, R: float, r: float) -> np.ndarray:
    """Vertex (i, j) -> index i*M + j at u = 2 pi i / N, v = 2 pi j / M (FP64)."""
    i = np.repeat(np.arange(N, dtype=np.float64), M)
    j = np.tile(np.arange(M, dtype=np.float64), N)
    u = 2.0 * math.pi * i / N
    v = 2.0 * math.pi * j / M
    x = (R + r * np.cos(v)) * np.cos(u)
    y = (R + r * np.cos(v)) * np.sin(u)
    z = r * np.sin(v)
    return np.stack([x, y, z], axis=1)


def _torus_quads(N: int, M: int) -> list[list[int]]:
    """Quad (i, j) = [(i,j), (i+1,j), (i+1,j+1), (i,j+1)], indices mod N, M; CCW seen from outside."""
    def vid(i, j):
        return (i % N) * M + (j % M)
    return [[vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)]
            for i in range(N) for j in range(M)]


def _jitter(P: np.ndarray, amp: float, rng: SplitMix64) -> np.ndarray:
    d = (rng.uniform(P.size).reshape(P.shape) * 2.0 - 1.0) * amp
    return (P + d).astype(np.float32)  # one rounding FP64 -> FP32


def _pack(faces: list[list[int]], P: np.ndarray, cverts, csharp) -> dict:
    off = np.zeros(len(faces) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(f) for f in faces])
    fv = np.fromiter((v for f in faces for v in f), dtype=np.int32, count=int(off[-1]))
    return dict(V=int(P.shape[0]), F=len(faces), off=off.astype(np.int32), fv=fv,
                P=np.ascontiguousarray(P, dtype=np.float32),
                crease_verts=np.asarray(cverts, dtype=np.int32).reshape(-1, 2),
                crease_sharp=np.asarray(csharp, dtype=np.float32).reshape(-1))


def _undirected_edges(faces: list[list[int]]) -> np.ndarray:
    """Unique undirected edges (min, max), sorted lexicographically (an input-side listing)."""
    lens = np.fromiter((len(f) for f in faces), dtype=np.int64, count=len(faces))
    fv = np.fromiter((v for f in faces for v in f), dtype=np.int64, count=int(lens.sum()))
    off = np.zeros(len(faces) + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    nxt = np.arange(1, fv.size + 1)
    nxt[off[1:] - 1] = off[:-1]                     # the last corner of a face wraps to its first
    a, b = fv, fv[nxt]
    e = np.stack([np.minimum(a, b), np.maximum(a, b)], axis=1)
    return np.unique(e, axis=0).reshape(-1, 2)      # unique rows, lexicographic order


def _tag_creases(faces, rng: SplitMix64, frac: float, mode: str):
    """Tag round(frac * E) edges chosen by a seeded permutation.

    mode "mixed": first half integer sharpness max(1, round(u)), second half fractional u,
    u ~ U[0, 4). mode "inf": sharpness +inf.
    """
    edges = _undirected_edges(faces)
    k = int(math.floor(frac * len(edges) + 0.5))
    perm = rng.permutation(len(edges))[:k]
    sel = edges[perm]
    if mode == "inf":
        sharp = np.full(k, np.inf, dtype=np.float32)
    else:
        u = rng.uniform(k) * 4.0
        sharp = u.copy()
        half = k // 2
        sharp[:half] = np.maximum(1.0, np.floor(u[:half] + 0.5))
        sharp = sharp.astype(np.float32)
        # a fractional draw that rounds to 0 in FP32 carries no crease; keep it strictly positive
        sharp[sharp <= 0] = np.float32(1e-3)
    return sel.astype(np.int32), sharp


def torus_cc_plain(N: int = 16, M: int = 16, jitter: float = 0.01, seed: int = SEED_BASE + 1,
                   R: float = 1.0, r: float = 0.3) -> dict:
    """Closed N x M quad torus, all valence 4, no creases."""
    rng = SplitMix64(seed)
    faces = _torus_quads(N, M)
    P = _jitter(_torus_points(N, M, R, r), jitter, rng)
    return _pack(faces, P, np.zeros((0, 2)), np.zeros(0))


def torus_cc_mixed(N: int = 96, M: int = 96, merge_frac: float = 0.08, split_frac: float = 0.04,
                   crease_frac: float = 0.05, jitter: float = 0.02, seed: int = SEED_BASE + 2,
                   R: float = 1.0, r: float = 0.3, creases: bool = True) -> dict:
    """Quad torus with hexagon merges, triangle splits and semi-sharp creases.

    1. round(merge_frac * F) quads are merged in disjoint pairs: a seeded permutation of the
       shared edges is scanned and an edge is removed when both its quads are still unused and
       neither endpoint lies on an already removed edge (so every valence stays >= 3).
    2. round(split_frac * F) of the remaining quads are split along a seeded diagonal, scanning a
       seeded permutation of the unused quads and skipping a split that would push a diagonal
       endpoint above valence 6.
    3. round(crease_frac * E) edges get sharpness: half integer, half fractional, in [0, 4].
    4. Positions are jittered by U(-jitter, jitter) per coordinate, then rounded once to FP32.
    """
    rng = SplitMix64(seed)
    quads = _torus_quads(N, M)
    F0 = len(quads)
    n_pairs = int(math.floor(merge_frac * F0 + 0.5)) // 2
    n_split = int(math.floor(split_frac * F0 + 0.5))
    # shared edges between quads: right neighbour (i+1, j) and top neighbour (i, j+1)
    shared = []
    for i in range(N):
        for j in range(M):
            a = i * M + j
            shared.append((a, ((i + 1) % N) * M + j, 1))   # quad a's edge k=1 is b's edge k=3
            shared.append((a, i * M + (j + 1) % M, 2))     # quad a's edge k=2 is b's edge k=0
    perm = rng.permutation(len(shared))
    used_face = np.zeros(F0, dtype=bool)
    used_vert = np.zeros(N * M, dtype=bool)
    merged_into = {}   # face a -> hexagon
    removed = set()
    for idx in perm:
        if len(merged_into) >= n_pairs:
            break
        a, b, k = shared[idx]
        qa = quads[a]
        e0, e1 = qa[k], qa[(k + 1) % 4]
        if used_face[a] or used_face[b] or used_vert[e0] or used_vert[e1]:
            continue
        qb = quads[b]
        kb = qb.index(e1)
        assert qb[(kb + 1) % 4] == e0
        # hexagon: walk qa from its vertex after the shared edge around to e0, then qb's far side
        hexa = [qa[(k + 1 + t) % 4] for t in range(4)] + [qb[(kb + 2) % 4], qb[(kb + 3) % 4]]
        # rotate so that quad a's first vertex leads
        s = hexa.index(qa[0])
        hexa = hexa[s:] + hexa[:s]
        merged_into[a] = hexa
        removed.add(b)
        used_face[a] = used_face[b] = True
        used_vert[e0] = used_vert[e1] = True
    # valence (incident faces) after the merges
    val = np.zeros(N * M, dtype=np.int64)
    for f in range(F0):
        if f in removed:
            continue
        for v in (merged_into[f] if f in merged_into else quads[f]):
            val[v] += 1
    remaining = np.array([f for f in range(F0) if not used_face[f]], dtype=np.int64)
    perm2 = rng.permutation(len(remaining))
    diag = rng.uniform(len(remaining))
    split = {}
    for t in perm2:
        if len(split) >= n_split:
            break
        f = int(remaining[t])
        q = quads[f]
        if diag[t] < 0.5:
            d0, d1 = q[0], q[2]
            tris = [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
        else:
            d0, d1 = q[1], q[3]
            tris = [[q[1], q[2], q[3]], [q[1], q[3], q[0]]]
        if val[d0] + 1 > 6 or val[d1] + 1 > 6:
            continue
        val[d0] += 1
        val[d1] += 1
        split[f] = tris
    faces = []
    for f in range(F0):
        if f in removed:
            continue
        if f in merged_into:
            faces.append(merged_into[f])
        elif f in split:
            faces.extend(split[f])
        else:
            faces.append(quads[f])
    if creases:
        cv, cs = _tag_creases(faces, rng, crease_frac, "mixed")
    else:
        cv, cs = np.zeros((0, 2)), np.zeros(0)
    P = _jitter(_torus_points(N, M, R, r), jitter, rng)
    return _pack(faces, P, cv, cs)


def torus_tri(N: int = 128, M: int = 128, flip_frac: float = 0.10, sharp_frac: float = 0.02,
              jitter: float = 0.01, seed: int = SEED_BASE + 3, R: float = 1.0, r: float = 0.3,
              creases: bool = True) -> dict:
    """Triangulated N x M torus with seeded edge flips and infinitely sharp edges.

    Every quad [q0, q1, q2, q3] becomes [q0, q1, q2], [q0, q2, q3]. Then the first
    round(flip_frac * E) edges of a seeded permutation are flipped in that order; a flip is
    skipped when the new edge already exists or a valence would leave [4, 8]. Finally
    round(sharp_frac * E) edges of a seeded permutation are made infinitely sharp.
    """
    rng = SplitMix64(seed)
    tris = []
    for q in _torus_quads(N, M):
        tris.append([q[0], q[1], q[2]])
        tris.append([q[0], q[2], q[3]])
    V = N * M
    val = np.zeros(V, dtype=np.int64)
    for t in tris:
        for v in t:
            val[v] += 1
    # directed edge -> triangle
    dmap = {}
    for ti, t in enumerate(tris):
        for j in range(3):
            dmap[(t[j], t[(j + 1) % 3])] = ti
    edges = _undirected_edges(tris)
    n_flip = int(math.floor(flip_frac * len(edges) + 0.5))
    perm = rng.permutation(len(edges))[:n_flip]
    for idx in perm:
        a, b = int(edges[idx][0]), int(edges[idx][1])
        if (a, b) not in dmap:
            continue  # this edge was flipped away already
        t1, t2 = dmap[(a, b)], dmap[(b, a)]
        T1, T2 = tris[t1], tris[t2]
        c = T1[(T1.index(b) + 1) % 3]   # T1 = (a, b, c)
        d = T2[(T2.index(a) + 1) % 3]   # T2 = (b, a, d)
        if c == d or (c, d) in dmap or (d, c) in dmap:
            continue
        if val[a] - 1 < 4 or val[b] - 1 < 4 or val[c] + 1 > 8 or val[d] + 1 > 8:
            continue
        for T in (T1, T2):
            for j in range(3):
                del dmap[(T[j], T[(j + 1) % 3])]
        n1, n2 = [c, a, d], [d, b, c]
        tris[t1], tris[t2] = n1, n2
        for ti, T in ((t1, n1), (t2, n2)):
            for j in range(3):
                dmap[(T[j], T[(j + 1) % 3])] = ti
        val[a] -= 1
        val[b] -= 1
        val[c] += 1
        val[d] += 1
    if creases:
        cv, cs = _tag_creases(tris, rng, sharp_frac, "inf")
    else:
        cv, cs = np.zeros((0, 2)), np.zeros(0)
    P = _jitter(_torus_points(N, M, R, r), jitter, rng)
    return _pack(tris, P, cv, cs)


# --- named workloads ---------------------------------------------------------------------------

def workload(name: str) -> dict:
    """The named synthetic workloads (sizes fixed here, recipe in the module docstring)."""
    if name == "cc_torus16_L3":
        m = torus_cc_plain(16, 16, 0.01, SEED_BASE + 1)
        m.update(scheme="cc", levels=3)
    elif name == "cc_creased_torus96_L6":
        m = torus_cc_mixed(96, 96, seed=SEED_BASE + 2)
        m.update(scheme="cc", levels=6)
    elif name == "loop_tri_torus128_L6":
        m = torus_tri(128, 128, seed=SEED_BASE + 3)
        m.update(scheme="loop", levels=6)
    elif name == "sqrt3_tri_torus128_L8":
        m = torus_tri(128, 128, seed=SEED_BASE + 3)
        m.update(scheme="sqrt3", levels=8)
    elif name == "sqrt3_tri_torus128_L8_smooth":
        # the same mesh without its sharp edges: the closed-mesh sqrt(3) kernels
        m = torus_tri(128, 128, seed=SEED_BASE + 3)
        m.update(scheme="sqrt3", levels=8, crease_verts=np.zeros((0, 2), np.int32),
                 crease_sharp=np.zeros(0, np.float32))
    elif name == "cc_creased_torus144_L4":
        m = torus_cc_mixed(144, 144, seed=SEED_BASE + 5)
        m.update(scheme="cc", levels=4)
    else:
        raise KeyError(name)
    m["name"] = name
    return m


def cube() -> dict:
    """Unit cube with vertices (+-1, +-1, +-1), six CCW quads (outward normals)."""
    P = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], dtype=np.float32)

    def vid(x, y, z):
        return ((x > 0) << 2) | ((y > 0) << 1) | (z > 0)
    faces = [
        [vid(-1, -1, -1), vid(-1, -1, 1), vid(-1, 1, 1), vid(-1, 1, -1)],   # x = -1
        [vid(1, -1, -1), vid(1, 1, -1), vid(1, 1, 1), vid(1, -1, 1)],       # x = +1
        [vid(-1, -1, -1), vid(1, -1, -1), vid(1, -1, 1), vid(-1, -1, 1)],   # y = -1
        [vid(-1, 1, -1), vid(-1, 1, 1), vid(1, 1, 1), vid(1, 1, -1)],       # y = +1
        [vid(-1, -1, -1), vid(-1, 1, -1), vid(1, 1, -1), vid(1, -1, -1)],   # z = -1
        [vid(-1, -1, 1), vid(1, -1, 1), vid(1, 1, 1), vid(-1, 1, 1)],       # z = +1
    ]
    return _pack(faces, P, np.zeros((0, 2)), np.zeros(0))


def octahedron() -> dict:
    """Octahedron with vertices +-e_x, +-e_y, +-e_z, eight CCW triangles (valence 4)."""
    P = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float32)
    X, x, Y, y, Z, z = range(6)
    faces = [[X, Y, Z], [Y, x, Z], [x, y, Z], [y, X, Z],
             [Y, X, z], [x, Y, z], [y, x, z], [X, y, z]]
    return _pack(faces, P, np.zeros((0, 2)), np.zeros(0))


def tetrahedron() -> dict:
    """Regular tetrahedron (valence 3), CCW triangles."""
    P = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float32)
    faces = [[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]]
    return _pack(faces, P, np.zeros((0, 2)), np.zeros(0))


def pillow(n: int = 6) -> dict:
    """Two n-gons glued along their boundary: closed, manifold, every vertex of valence 2."""
    t = 2.0 * math.pi * np.arange(n) / n
    P = np.stack([np.cos(t), np.sin(t), 0.1 * np.cos(3 * t)], axis=1).astype(np.float32)
    faces = [list(range(n)), list(range(n - 1, -1, -1))]
    return _pack(faces, P, np.zeros((0, 2)), np.zeros(0))


def prism(n: int = 12, h: float = 0.7) -> dict:
    """Closed n-gon prism: two n-gon caps (faces of n corners) and n side quads; valence 3."""
    t = 2.0 * math.pi * np.arange(n) / n
    top = np.stack([np.cos(t), np.sin(t), np.full(n, h)], axis=1)
    bot = np.stack([np.cos(t), np.sin(t), np.full(n, -h)], axis=1)
    P = np.concatenate([top, bot]).astype(np.float32)
    faces = [list(range(n)),                                      # top, CCW seen from +z
             [n + i for i in range(n - 1, -1, -1)]]               # bottom, CCW seen from -z
    faces += [[n + i, n + (i + 1) % n, (i + 1) % n, i] for i in range(n)]
    return _pack(faces, P, np.zeros((0, 2)), np.zeros(0))


def tube_cc(N: int = 16, M: int = 9, jitter: float = 0.05, z_step: float = 0.25,
            seed: int = SEED_BASE + 6) -> dict:
    """Open quad cylinder: N vertices around, M vertex rows, M - 1 rows of quads, two boundary
    loops (rows 0 and M - 1). Vertex (i, j) -> index j*N + i at angle 2 pi i / N; the radius is
    jittered by U(-jitter, jitter) per vertex, z = j * z_step exactly (a power of two keeps z
    exact in FP32). Face (i, j) = [(i,j), (i+1,j), (i+1,j+1), (i,j+1)], face index j*N + i."""
    rng = SplitMix64(seed)
    i = np.tile(np.arange(N, dtype=np.float64), M)
    j = np.repeat(np.arange(M, dtype=np.float64), N)
    u = 2.0 * math.pi * i / N
    rad = 1.0 + (rng.uniform(N * M) * 2.0 - 1.0) * jitter
    P = np.stack([rad * np.cos(u), rad * np.sin(u), j * z_step], axis=1).astype(np.float32)
    faces = [[jj * N + ii, jj * N + (ii + 1) % N, (jj + 1) * N + (ii + 1) % N, (jj + 1) * N + ii]
             for jj in range(M - 1) for ii in range(N)]
    return _pack(faces, P, np.zeros((0, 2)), np.zeros(0))


def sheet_cc(NX: int = 12, NY: int = 9, split_frac: float = 0.1, jitter: float = 0.02,
             seed: int = SEED_BASE + 7) -> dict:
    """Open planar NX x NY grid of quads (one boundary loop with four valence-2 corners), a share
    of quads split into triangle pairs, xy jittered and z a seeded bump. Vertex (i, j) -> j*(NX+1)+i."""
    rng = SplitMix64(seed)
    W = NX + 1
    faces = []
    split = rng.uniform(NX * NY)
    for jj in range(NY):
        for ii in range(NX):
            q = [jj * W + ii, jj * W + ii + 1, (jj + 1) * W + ii + 1, (jj + 1) * W + ii]
            if split[jj * NX + ii] < split_frac:
                faces += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
            else:
                faces.append(q)
    x = np.tile(np.arange(W, dtype=np.float64), NY + 1) / NX
    y = np.repeat(np.arange(NY + 1, dtype=np.float64), W) / NY
    d = (rng.uniform(2 * W * (NY + 1)).reshape(-1, 2) * 2.0 - 1.0) * jitter
    z = 0.2 * np.sin(3.0 * x) * np.cos(2.0 * y)
    P = np.stack([x + d[:, 0], y + d[:, 1], z], axis=1).astype(np.float32)
    return _pack(faces, P, np.zeros((0, 2)), np.zeros(0))


def triangulate(m: dict) -> dict:
    """The same mesh with every face of order c > 3 split into the fan of c - 2 triangles from its
    corner 0 (a quad [a, b, c, d] -> [a, b, c], [a, c, d]); vertices, positions and creases kept."""
    off, fv = np.asarray(m["off"]), np.asarray(m["fv"])
    faces = []
    for r in range(len(off) - 1):
        f = fv[off[r]:off[r + 1]].tolist()
        faces += [[f[0], f[k], f[k + 1]] for k in range(1, len(f) - 1)]
    out = _pack(faces, np.asarray(m["P"]), np.asarray(m.get("crease_verts", np.zeros((0, 2)))).reshape(-1, 2),
                np.asarray(m.get("crease_sharp", np.zeros(0))).reshape(-1))
    return out


def open_box() -> dict:
    """The unit cube without its z = +1 face: one boundary loop of four valence-3 vertices."""
    m = cube()
    return _pack([list(m["fv"][4 * r:4 * r + 4]) for r in range(5)], m["P"], np.zeros((0, 2)), np.zeros(0))


def polygon(n: int = 4) -> dict:
    """A single n-gon (one face, all vertices on the boundary, each in one face only)."""
    t = 2.0 * math.pi * np.arange(n) / n
    P = np.stack([np.cos(t), 0.8 * np.sin(t), 0.2 * np.sin(2 * t)], axis=1).astype(np.float32)
    return _pack([list(range(n))], P, np.zeros((0, 2)), np.zeros(0))


def holed_cc_mixed(N: int = 32, M: int = 24, holes: int = 6, seed: int = SEED_BASE + 8,
                   creases: bool = True) -> dict:
    """``torus_cc_mixed`` with ``holes`` faces cut out (each hole one boundary loop). The removed
    faces are drawn from a seeded permutation, skipping any face that shares a vertex with a face
    already removed (so every vertex keeps a single fan); creases touching a hole are dropped."""
    m = torus_cc_mixed(N, M, seed=seed, creases=creases)
    off, fv = m["off"], m["fv"]
    rng = SplitMix64(seed ^ 0x5EED)
    used = np.zeros(m["V"], dtype=bool)
    gone = []
    for f in rng.permutation(m["F"]):
        if len(gone) >= holes:
            break
        vs = fv[off[f]:off[f + 1]]
        if used[vs].any():
            continue
        used[vs] = True
        gone.append(int(f))
    gone_set = set(gone)
    faces = [list(fv[off[f]:off[f + 1]]) for f in range(m["F"]) if f not in gone_set]
    cv, cs = m["crease_verts"], m["crease_sharp"]
    keep = ~(used[cv[:, 0]] | used[cv[:, 1]]) if len(cs) else np.zeros(0, dtype=bool)
    return _pack(faces, m["P"], cv[keep], cs[keep])


def serving_requests(n_requests: int = 512, rate_hz: float = 2000.0, n_resident: int = 32,
                     seed: int = SEED_BASE + 4, fmin: float = 1e3, fmax: float = 6e4,
                     frac_frame: float = 0.70) -> dict:
    """Request stream for the serving loop (arrival times, meshes, schemes, levels).

    32 resident topologies are drawn first (scheme 60/25/15 CC/Loop/sqrt3, levels uniform in
    2..5, face target log-uniform in [fmin, fmax]); then each request is, with probability
    frac_frame, a new frame of a uniformly chosen resident topology (positions re-jittered by
    +-0.05), else a fresh mesh drawn like a resident one. Arrivals are Poisson at rate_hz.
    """
    rng = SplitMix64(seed)

    def draw_mesh(sub_seed):
        u = rng.uniform(3)
        target = math.exp(math.log(fmin) + u[0] * (math.log(fmax) - math.log(fmin)))
        scheme = "cc" if u[1] < 0.60 else ("loop" if u[1] < 0.85 else "sqrt3")
        levels = 2 + min(3, int(u[2] * 4))
        if scheme == "cc":
            n = max(4, int(round(math.sqrt(target))))
            m = torus_cc_mixed(n, n, seed=sub_seed)
        else:
            n = max(4, int(round(math.sqrt(target / 2.0))))
            m = torus_tri(n, n, seed=sub_seed)
        m.update(scheme=scheme, levels=levels)
        return m

    resident = [draw_mesh(seed * 1000 + i) for i in range(n_resident)]
    gaps = -np.log(1.0 - rng.uniform(n_requests)) / rate_hz
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for q in range(n_requests):
        u = rng.uniform(2)
        if u[0] < frac_frame:
            rid = min(n_resident - 1, int(u[1] * n_resident))
            base = resident[rid]
            P = (base["P"].astype(np.float64)
                 + (rng.uniform(base["P"].size).reshape(base["P"].shape) * 2 - 1) * 0.05)
            reqs.append(dict(kind="frame", resident=rid, P=P.astype(np.float32),
                             arrival=float(arrivals[q])))
        else:
            m = draw_mesh(seed * 1000 + n_resident + q)
            reqs.append(dict(kind="mesh", mesh=m, arrival=float(arrivals[q])))
    return dict(resident=resident, requests=reqs)
