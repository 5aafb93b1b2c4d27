"""Patches of a large mesh for sampled parity checks (test infrastructure, plain numpy).

A patch is the set of faces within two vertex-adjacency rings of some sampled faces, with its
vertices renumbered in increasing order (so every sum the oracle forms runs in the same order as on
the whole mesh). One refinement step of the patch in the oracle's patch mode gives, for the sampled
faces, exactly the children the whole mesh would give: each child point's stencil reaches at most
one ring beyond its face.

Children of face r of a level (Sec. 3.2 layouts): Catmull-Clark quads off[r] .. off[r+1]-1 (one per
corner), Loop triangles 4r .. 4r+3, sqrt(3) triangles 3r .. 3r+2 (one per corner).
"""
from __future__ import annotations

import numpy as np

ARITY = {"cc": 4, "loop": 3, "sqrt3": 3}


def sample_faces(F: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.unique(rng.choice(F, size=min(n, F), replace=False))


def _face_mask(off: np.ndarray, fv: np.ndarray, vmark: np.ndarray) -> np.ndarray:
    """Faces with at least one marked vertex."""
    hit = vmark[fv].astype(np.int64)
    c = np.concatenate([[0], np.cumsum(hit)])
    return (c[off[1:]] - c[off[:-1]]) > 0


def extract(level: dict, faces: np.ndarray, rings: int = 2, creases: bool = True) -> tuple[dict, np.ndarray]:
    """The patch around `faces` of `level` (dict with V, F, off, fv, P, crease_verts, crease_sharp).

    Returns the patch mesh and, for each sampled face, its index in the patch."""
    off = np.asarray(level["off"], dtype=np.int64)
    fv = np.asarray(level["fv"], dtype=np.int64)
    V = int(level["V"])
    fmask = np.zeros(len(off) - 1, dtype=bool)
    fmask[faces] = True
    for _ in range(rings):
        vmark = np.zeros(V, dtype=bool)
        vmark[fv[np.repeat(fmask, np.diff(off))]] = True
        fmask = _face_mask(off, fv, vmark)
    keep = np.flatnonzero(fmask)
    counts = off[keep + 1] - off[keep]
    corners = np.flatnonzero(np.repeat(fmask, np.diff(off)))
    verts = np.unique(fv[corners])                       # increasing: the sums keep their order
    remap = np.full(V, -1, dtype=np.int64)
    remap[verts] = np.arange(verts.size)
    poff = np.zeros(keep.size + 1, dtype=np.int64)
    poff[1:] = np.cumsum(counts)
    pm = dict(V=int(verts.size), F=int(keep.size), off=poff.astype(np.int32),
              fv=remap[fv[corners]].astype(np.int32), P=np.asarray(level["P"])[verts])
    cv = np.asarray(level.get("crease_verts", np.zeros((0, 2))), dtype=np.int64).reshape(-1, 2)
    cs = np.asarray(level.get("crease_sharp", np.zeros(0)), dtype=np.float32).reshape(-1)
    if creases and cs.size:
        inside = (remap[cv[:, 0]] >= 0) & (remap[cv[:, 1]] >= 0)
        pm["crease_verts"] = remap[cv[inside]].astype(np.int32).reshape(-1, 2)
        pm["crease_sharp"] = cs[inside]
    else:
        pm["crease_verts"] = np.zeros((0, 2), np.int32)
        pm["crease_sharp"] = np.zeros(0, np.float32)
    local = np.searchsorted(keep, faces)
    return pm, local


def child_corners(scheme: str, off: np.ndarray, r: int) -> np.ndarray:
    """Corner indices (into the next level's flat face table) of the children of face r."""
    k = ARITY[scheme]
    if scheme == "cc":
        first, n = int(off[r]), int(off[r + 1] - off[r])
    elif scheme == "loop":
        first, n = 4 * r, 4
    else:
        first, n = 3 * r, 3
    return np.arange(k * first, k * (first + n))
