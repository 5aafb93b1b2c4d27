"""Ragged batches: many topologies of uneven sizes, mixed schemes and level counts, refined with
one launch per level per kernel class (CUDA graph replay). Every member must equal its own
alsub_refine_vertices result within the parity tolerance, and the oracle: topology from each
member's handle (bit-exact after relabelling), positions from the batch output."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu

TOL = 2e-6


def _members():
    return [
        ("cc", synth.torus_cc_mixed(20, 24, seed=81), 3),
        ("cc", synth.torus_cc_plain(9, 7, jitter=0.02, seed=82), 4),
        ("cc", synth.cube(), 2),
        ("cc", synth.torus_cc_mixed(31, 17, crease_frac=0.1, seed=83), 1),
        ("loop", synth.torus_tri(13, 11, seed=84), 3),
        ("loop", synth.octahedron(), 4),
        ("sqrt3", synth.torus_tri(12, 9, seed=85, creases=False), 4),
        ("sqrt3", synth.tetrahedron(), 2),
        ("cc", synth.torus_cc_mixed(12, 12, seed=86), 0),
    ]


def _oracle_refs():
    return [oracle.subdivide(m, lv, scheme, keep_all=True) for scheme, m, lv in _members()]


def _check_oracle(topos, outs, refs):
    """Each member's face tables and creases from its own handle, its last level's positions from
    the batch output, against the oracle."""
    for (scheme, m, lv), T, got, ref in zip(_members(), topos, outs, refs):
        gpu = []
        for l in range(lv + 1):
            d = dict(T.counts[l])
            d["fv"] = T.faces(l)
            d["crease_verts"], d["crease_sharp"] = T.creases(l)
            gpu.append(d)
        gpu[-1]["P"] = got.cpu().numpy()
        gpu_util.compare(scheme, gpu, ref, pos_levels={lv})


def _build():
    import torch
    from paper_1809_06047_gb300 import alsub
    keep, topos, P0s = [], [], []
    for scheme, m, lv in _members():
        M = alsub.Mesh.from_dict(m, scheme)
        T = alsub.Topology(M, lv)
        keep.append(M)
        topos.append(T)
        P0s.append(torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda())
    return keep, topos, P0s


def _check(topos, P0s, outs):
    for T, P0, got in zip(topos, P0s, outs):
        want = T.refine_vertices(P0)
        diag = float((want.max(0).values - want.min(0).values).norm())
        assert float((got - want).abs().max()) <= TOL * max(diag, 1e-3)


def test_batch_matches_members_and_replays():
    import torch
    from paper_1809_06047_gb300 import alsub
    keep, topos, P0s = _build()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B = alsub.Batch(topos, P0s)
        first = [x.clone() for x in B.refine(stream=s)]          # captures the graph
        second = [x.clone() for x in B.refine(stream=s)]         # replays it
    torch.cuda.synchronize()
    for a, b in zip(first, second):
        assert torch.equal(a, b)
    _check(topos, P0s, first)
    refs = _oracle_refs()
    _check_oracle(topos, first, refs)
    _check_oracle(topos, second, refs)
    # new positions written into the bound inputs are picked up by the replay
    for P in P0s:
        P.mul_(1.5).add_(0.25)
    with torch.cuda.stream(s):
        third = [x.clone() for x in B.refine(stream=s)]
    torch.cuda.synchronize()
    _check(topos, P0s, third)
    per_call = B.launches() // 3
    assert per_call >= 4          # a handful of launches for nine meshes and four levels
    for T in topos:
        T.status()


def test_batch_autotune_keeps_results():
    import torch
    from paper_1809_06047_gb300 import alsub
    keep, topos, P0s = _build()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B = alsub.Batch(topos, P0s)
        best = B.tune(stream=s)
        outs = [x.clone() for x in B.refine(stream=s)]
    torch.cuda.synchronize()
    assert best["block"] in (128, 256, 512) and best["ms"] > 0
    _check(topos, P0s, outs)
    _check_oracle(topos, outs, _oracle_refs())
    B.configure(128, 0)
    outs = [x.clone() for x in B.refine()]
    torch.cuda.synchronize()
    _check(topos, P0s, outs)
