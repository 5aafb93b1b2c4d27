"""Ragged batches: many topologies of uneven sizes, mixed schemes and level counts, refined with
one launch per level per kernel class (CUDA graph replay). Every member must equal its own
alsub_refine_vertices result within the parity tolerance."""
import numpy as np
import pytest

from paper_1809_06047_gb300 import synth

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
    B.configure(128, 0)
    outs = [x.clone() for x in B.refine()]
    torch.cuda.synchronize()
    _check(topos, P0s, outs)
