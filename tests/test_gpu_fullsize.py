"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (one
alsub_subdivide call on the dynamic path), on sampled outputs.

The oracle cannot refine the full meshes, but it can compute any child point from a patch of the
level above (tests/patch.py: two rings around the sampled faces, oracle patch mode). For the
Catmull-Clark workload the level above is the oracle's own level 5 (so the check covers all six
levels end to end); for Loop and sqrt(3) it is the CUDA path's level L-1, for the timed last step
(Loop level 6, sqrt(3) level 8) and for every level between it and the largest level the oracle
refines whole (Loop 5, sqrt(3) 6 and 7). Every child point of 4096 sampled faces must agree within
2e-6 x the bounding-box diagonal.
"""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util, patch

pytestmark = pytest.mark.gpu

N_SAMPLES = 4096


def _compare(scheme, parent, child, faces, level=0):
    pm, local = patch.extract(parent, faces)
    part = oracle.subdivide(pm, 1, scheme, patch=True, start_level=level)[1]
    diag = float(np.linalg.norm(child["P"].max(0) - child["P"].min(0)))
    worst = 0.0
    for r, q in zip(faces, local):
        a = child["fv"][patch.child_corners(scheme, parent["off"], int(r))]
        b = part["fv"][patch.child_corners(scheme, pm["off"], int(q))]
        assert np.all(b >= 0)
        ref = part["P"][b]
        assert np.all(np.isfinite(ref)), f"face {r}: a sampled child reaches beyond the patch"
        worst = max(worst, float(np.abs(child["P"][a] - ref).max()))
    assert worst <= gpu_util.POS_TOL * diag, f"max err {worst:.3e} > {gpu_util.POS_TOL} x {diag:.3f}"
    return worst / diag


def test_cc_creased_torus96_L6_sampled():
    """Config of the headline: six levels of the creased mixed torus (37.75 M quads) against the
    oracle's level 5 and one patch step."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.workload("cc_creased_torus96_L6")
    ref5 = oracle.subdivide(m, 5, "cc", keep_all=False)[5]
    M = alsub.Mesh.from_dict(m, "cc")
    T = alsub.Topology(M, 6, build=False)
    P0 = torch.from_numpy(m["P"]).cuda()
    PL = torch.empty((T.counts[-1]["V"], 3), dtype=torch.float32, device="cuda")
    T.subdivide(P0, out=PL)
    torch.cuda.synchronize()
    T.status()
    child = dict(fv=T.faces(6), P=PL.cpu().numpy().astype(np.float64))
    T.close()
    faces = patch.sample_faces(ref5["F"], N_SAMPLES, seed=71)
    _compare("cc", ref5, child, faces)


@pytest.mark.parametrize("name,scheme", [("loop_tri_torus128_L6", "loop"), ("sqrt3_tri_torus128_L8", "sqrt3")])
def test_triangle_schemes_last_step_sampled(name, scheme):
    """Loop level 6 (134.2 M triangles) and sqrt(3) level 8 (215.0 M triangles): the timed last
    step, from the CUDA path's level L-1, against one oracle patch step."""
    _triangle_step_sampled(name, scheme, synth.workload(name)["levels"])


@pytest.mark.parametrize("name,scheme,L", [("loop_tri_torus128_L6", "loop", 5),
                                           ("sqrt3_tri_torus128_L8", "sqrt3", 6),
                                           ("sqrt3_tri_torus128_L8", "sqrt3", 7)])
def test_triangle_schemes_middle_levels_sampled(name, scheme, L):
    """The levels between the oracle's whole-mesh limit (Loop 4, sqrt(3) 5) and the last one, at the
    benchmark's full size: level L from the CUDA path's level L - 1 against one oracle patch step."""
    _triangle_step_sampled(name, scheme, L)


def _triangle_step_sampled(name, scheme, L):
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.workload(name)
    M = alsub.Mesh.from_dict(m, scheme)
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda()
    T = alsub.Topology(M, L - 1, build=True)
    P = T.refine_vertices(P0)
    torch.cuda.synchronize()
    T.status()
    c = T.counts[-1]
    parent = dict(V=c["V"], F=c["F"], fv=T.faces(L - 1), off=np.arange(c["F"] + 1, dtype=np.int64) * 3,
                  P=P.cpu().numpy().astype(np.float64))
    # Loop creases, and sqrt(3)'s infinitely sharp ones (feature edges)
    parent["crease_verts"], parent["crease_sharp"] = T.creases(L - 1)
    T.close()
    del P
    T = alsub.Topology(M, L, build=False)
    PL = torch.empty((T.counts[-1]["V"], 3), dtype=torch.float32, device="cuda")
    T.subdivide(P0, out=PL)
    torch.cuda.synchronize()
    T.status()
    child = dict(fv=T.faces(L), P=PL.cpu().numpy().astype(np.float64))
    T.close()
    faces = patch.sample_faces(parent["F"], N_SAMPLES, seed=72)
    _compare(scheme, parent, child, faces, level=L - 1)
