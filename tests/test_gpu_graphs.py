"""Repeated refine calls replay a CUDA graph the library captures: the first call with new pointers
launches kernels directly, the second is captured, later ones replay. Every way must give the same
bits, pick up new input values written behind the same pointers, count the same kernels, and keep
the per-level timing events working."""
import numpy as np
import pytest

from paper_1809_06047_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme,mesh,levels", [
    ("cc", lambda: synth.torus_cc_mixed(18, 14, seed=61), 4),
    ("loop", lambda: synth.torus_tri(12, 10, seed=62), 3),
    ("sqrt3", lambda: synth.torus_tri(10, 8, seed=63, creases=False), 4),
])
def test_replay_matches_direct(scheme, mesh, levels):
    import torch
    from paper_1809_06047_gb300 import alsub
    m = mesh()
    M = alsub.Mesh.from_dict(m, scheme)
    T = alsub.Topology(M, levels, build=False)
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda()
    PL = torch.empty((T.counts[-1]["V"], 3), dtype=torch.float32, device="cuda")
    outs, launches = [], []
    T.timings()
    for _ in range(4):                       # direct, captured, replayed, replayed
        T.subdivide(P0, out=PL)
        torch.cuda.synchronize()
        outs.append(PL.clone())
        launches.append(T.timings()[2])
    T.status()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    assert len(set(launches)) == 1 and launches[0] > 0
    # new values behind the same pointer
    P0.mul_(0.5).add_(1.0)
    T.subdivide(P0, out=PL)
    ref = alsub.Topology(M, levels).refine_vertices(P0)       # a fresh handle: direct launches
    torch.cuda.synchronize()
    assert torch.equal(PL, ref)
    # the static path too: direct, captured, replayed
    R = alsub.Topology(M, levels)
    got = [R.refine_vertices(P0, out=torch.empty_like(PL)) for _ in range(1)]
    out = torch.empty_like(PL)
    for _ in range(3):
        R.refine_vertices(P0, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out, got[0])


def test_timing_events_inside_graphs():
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_mixed(24, 20, seed=64)
    M = alsub.Mesh.from_dict(m, "cc")
    T = alsub.Topology(M, 4, build=False)
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda()
    PL = torch.empty((T.counts[-1]["V"], 3), dtype=torch.float32, device="cuda")
    T.subdivide(P0, out=PL)
    T.subdivide(P0, out=PL)                  # untimed graph captured
    T.set_timing(5)
    for _ in range(5):                       # first timed call is captured with event nodes
        T.subdivide(P0, out=PL)
    ms, calls, launches = T.timings()
    assert calls == 5 and launches > 0
    assert np.all(ms > 0)
    # beyond the capacity the read fails but nothing breaks
    for _ in range(7):
        T.subdivide(P0, out=PL)
    with pytest.raises(alsub.AlsubError):
        T.timings()
    T.set_timing(0)
    T.subdivide(P0, out=PL)
    torch.cuda.synchronize()
    T.status()
