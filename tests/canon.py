"""Canonical relabelling and comparison of two refinement results (test infrastructure).

Both sides follow the refined-mesh layout of Sec. 3.2: old vertices keep their ids, face points
follow at |v| + r, edge points after them; children of a face follow in corner order. The one
freedom is the edge numbering (Sec. 3.2 only asks for a unique enumeration of the upper
triangle of E). This module recovers, level by level, the map from one side's edge ids to the
other's from the edge points' slots in the child face tables, checks that the map is a
bijection, and then requires the relabelled face tables to be equal integer for integer. The
vertex map of level l+1 is [map of level l | identity on face points | edge map].

It imports neither the oracle nor the CUDA binding.
"""
from __future__ import annotations

import numpy as np

ARITY = {"cc": 4, "loop": 3, "sqrt3": 3}


class Mismatch(AssertionError):
    pass


def _edge_map(a_ids: np.ndarray, b_ids: np.ndarray, E: int, level: int) -> np.ndarray:
    """Map edge ids of side A to side B from paired occurrences; must be a consistent bijection."""
    if a_ids.min(initial=0) < 0 or a_ids.max(initial=-1) >= E or b_ids.min(initial=0) < 0 \
            or b_ids.max(initial=-1) >= E:
        raise Mismatch(f"level {level}: edge id out of range")
    emap = np.full(E, -1, dtype=np.int64)
    emap[a_ids] = b_ids
    if not np.array_equal(emap[a_ids], b_ids):
        raise Mismatch(f"level {level}: an edge of A maps to two edges of B")
    if (emap < 0).any():
        raise Mismatch(f"level {level}: {int((emap < 0).sum())} edges of A never appear")
    if np.unique(emap).size != E:
        raise Mismatch(f"level {level}: two edges of A map to one edge of B")
    return emap


def vertex_maps(scheme: str, faces_a: list, faces_b: list, counts: list) -> list:
    """Vertex maps A -> B for levels 0..L (faces_*[l]: flat int arrays of level l).

    counts[l] = dict(V, F, E) of level l (identical on both sides). Raises Mismatch when the face
    tables differ after relabelling.
    """
    k = ARITY[scheme]
    L = len(faces_a) - 1
    pi = [np.arange(counts[0]["V"], dtype=np.int64)]
    if not np.array_equal(np.asarray(faces_a[0]), np.asarray(faces_b[0])):
        raise Mismatch("level 0 face tables differ")
    for l in range(L):
        V, F, E = counts[l]["V"], counts[l]["F"], counts[l]["E"]
        A = np.asarray(faces_a[l + 1], dtype=np.int64).reshape(-1, k)
        B = np.asarray(faces_b[l + 1], dtype=np.int64).reshape(-1, k)
        if A.shape != B.shape:
            raise Mismatch(f"level {l + 1}: face counts differ {A.shape} vs {B.shape}")
        if scheme == "cc":
            base = V + F
            emap = _edge_map(A[:, 1] - base, B[:, 1] - base, E, l + 1)
        elif scheme == "loop":
            base = V
            emap = _edge_map(A[:, 1] - base, B[:, 1] - base, E, l + 1)
        else:
            base, emap = None, None
        if scheme == "sqrt3":
            # face points (and the feature-edge points in the triangles' slots), then the second
            # points of boundary edges split on a second step (ranked alike on both sides)
            nxt = np.concatenate([pi[l], np.arange(V, counts[l + 1]["V"])])
        elif scheme == "cc":
            nxt = np.concatenate([pi[l], np.arange(V, V + F), base + emap])
        else:
            nxt = np.concatenate([pi[l], base + emap])
        if A.min() < 0 or A.max() >= nxt.size:
            raise Mismatch(f"level {l + 1}: vertex id out of range")
        mapped = nxt[A]
        if not np.array_equal(mapped, B):
            bad = np.argwhere(mapped != B)
            raise Mismatch(f"level {l + 1}: {len(bad)} face-table entries differ after relabelling, "
                           f"first at face {bad[0][0]} slot {bad[0][1]}: {mapped[bad[0][0]]} vs "
                           f"{B[bad[0][0]]}")
        pi.append(nxt)
    return pi


def compare_creases(pi: np.ndarray, cv_a, cs_a, cv_b, cs_b, level: int):
    """Crease lists equal as sets of (relabelled undirected edge, FP32 sharpness), bit for bit."""
    cv_a = np.asarray(cv_a, dtype=np.int64).reshape(-1, 2)
    cv_b = np.asarray(cv_b, dtype=np.int64).reshape(-1, 2)
    if cv_a.shape != cv_b.shape:
        raise Mismatch(f"level {level}: {len(cv_a)} vs {len(cv_b)} creases")
    if cv_a.size == 0:
        return

    def keyed(cv, cs):
        lo, hi = np.minimum(cv[:, 0], cv[:, 1]), np.maximum(cv[:, 0], cv[:, 1])
        bits = np.asarray(cs, dtype=np.float32).view(np.uint32).astype(np.int64)
        order = np.lexsort((bits, hi, lo))
        return np.stack([lo, hi, bits], axis=1)[order]

    ka = keyed(pi[cv_a], cs_a)
    kb = keyed(cv_b, cs_b)
    if not np.array_equal(ka, kb):
        bad = np.argwhere((ka != kb).any(axis=1))[0][0]
        raise Mismatch(f"level {level}: crease lists differ, first at {ka[bad]} vs {kb[bad]}")


def position_error(pi: np.ndarray, P_a, P_b) -> tuple[float, float]:
    """(max |P_a - P_b[pi]| over all xyz, bounding-box diagonal of P_b)."""
    P_a = np.asarray(P_a, dtype=np.float64).reshape(-1, 3)
    P_b = np.asarray(P_b, dtype=np.float64).reshape(-1, 3)
    Pb_on_a = np.empty_like(P_b)
    Pb_on_a[:] = P_b[pi]
    err = float(np.abs(P_a - Pb_on_a).max()) if P_a.size else 0.0
    diag = float(np.linalg.norm(P_b.max(axis=0) - P_b.min(axis=0))) if P_b.size else 0.0
    return err, diag


def relabel(scheme: str, levels: list, seed: int) -> list:
    """Renumber the edges of every level of an oracle result with a random permutation (old vertex
    ids kept, face points kept), as another valid implementation could. For testing this module."""
    rng = np.random.default_rng(seed)
    k = ARITY[scheme]
    out = [dict(levels[0])]
    perm = np.arange(levels[0]["V"])
    for l in range(len(levels) - 1):
        a, b = levels[l], levels[l + 1]
        V, F, E = a["V"], a["F"], a["E"]
        ep = rng.permutation(E)
        if scheme == "cc":
            nperm = np.concatenate([perm, np.arange(V, V + F), V + F + ep])
        elif scheme == "loop":
            nperm = np.concatenate([perm, V + ep])
        else:
            nperm = np.concatenate([perm, np.arange(V, b["V"])])
        d = dict(b)
        d["fv"] = nperm[np.asarray(b["fv"], dtype=np.int64)].astype(np.int32)
        P = np.empty_like(b["P"])
        P[nperm] = b["P"]
        d["P"] = P
        d["crease_verts"] = nperm[np.asarray(b["crease_verts"], dtype=np.int64)].astype(np.int32)
        out.append(d)
        perm = nperm
    return out
