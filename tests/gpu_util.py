"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and compare with the
oracle level by level (topology bit-exact after canonical relabelling, crease lists bit-exact,
positions within 2e-6 x bounding-box diagonal per level)."""
from __future__ import annotations

import numpy as np

from tests import canon

POS_TOL = 2e-6        # x bounding-box diagonal of the oracle's level-l positions


def gpu_run(mesh: dict, scheme: str, levels: int, mode: str = "static", per_level: bool = True):
    """Face tables, crease lists and positions of every level from the CUDA path."""
    import torch
    from paper_1809_06047_gb300 import alsub
    M = alsub.Mesh.from_dict(mesh, scheme)
    T = alsub.Topology(M, levels, build=(mode == "static"))
    P0 = torch.from_numpy(np.ascontiguousarray(mesh["P"], dtype=np.float32)).cuda()
    PL = T.refine_vertices(P0) if mode == "static" else T.subdivide(P0)
    torch.cuda.synchronize()
    T.status()
    out = []
    for l in range(levels + 1):
        d = dict(T.counts[l])
        d["fv"] = T.faces(l)
        d["crease_verts"], d["crease_sharp"] = T.creases(l)
        out.append(d)
    out[-1]["P"] = PL.cpu().numpy()
    out[0]["P"] = mesh["P"]
    if per_level:
        for l in range(1, levels):
            Tl = alsub.Topology(M, l, build=True)
            out[l]["P"] = Tl.refine_vertices(P0).cpu().numpy()
            Tl.status()
            Tl.close()
    T.close()
    M.close()
    return out


def compare(scheme: str, gpu: list, ref: list, pos_levels=None):
    counts = [dict(V=r["V"], F=r["F"], E=r["E"]) for r in ref]
    for g, r in zip(gpu, ref):
        assert (g["V"], g["F"]) == (r["V"], r["F"])
    pi = canon.vertex_maps(scheme, [g["fv"] for g in gpu], [r["fv"] for r in ref], counts)
    errs = []
    for l in range(len(ref)):
        canon.compare_creases(pi[l], gpu[l]["crease_verts"], gpu[l]["crease_sharp"],
                              ref[l]["crease_verts"], ref[l]["crease_sharp"], l)
        if "P" in gpu[l] and (pos_levels is None or l in pos_levels):
            err, diag = canon.position_error(pi[l], gpu[l]["P"], ref[l]["P"])
            assert err <= POS_TOL * diag, f"level {l}: max err {err:.3e} > {POS_TOL} x {diag:.3f}"
            errs.append(err / diag)
    return errs
