"""alsub_subdivide_host: host buffers in and out, the next call's upload and eval overlapping the
previous call's download. Every call's result must equal alsub_subdivide on device buffers bit for
bit, whatever the inputs of the calls around it, with page-locked and pageable host memory."""
import numpy as np
import pytest

from paper_1809_06047_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme,mesh,levels", [
    ("cc", lambda: synth.torus_cc_mixed(20, 16, seed=81), 4),
    ("cc", lambda: synth.holed_cc_mixed(16, 12, holes=3, seed=82), 3),
    ("loop", lambda: synth.torus_tri(12, 10, seed=83), 3),
])
def test_host_calls_match_device_calls(scheme, mesh, levels):
    import torch
    from paper_1809_06047_gb300 import alsub
    m = mesh()
    M = alsub.Mesh.from_dict(m, scheme)
    H = alsub.Topology(M, levels, build=False)
    D = alsub.Topology(M, levels, build=False)
    VL = H.counts[-1]["V"]
    rng = np.random.default_rng(5)
    frames = [(m["P"] + rng.uniform(-0.05, 0.05, m["P"].shape)).astype(np.float32) for _ in range(6)]
    # pinned: many calls in flight into two alternating outputs, read after one sync
    outs = [torch.empty((VL, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    got = []
    for k, P in enumerate(frames):
        o = outs[k & 1]
        H.subdivide_host(torch.from_numpy(P).pin_memory(), out=o)
        if k & 1:
            torch.cuda.current_stream().synchronize()
            got += [outs[0].clone(), outs[1].clone()]
    torch.cuda.synchronize()
    H.status()
    for P, g in zip(frames, got):
        ref = D.subdivide(torch.from_numpy(P).cuda())
        torch.cuda.synchronize()
        assert torch.equal(g, ref.cpu())
    # pageable numpy in and out, the input buffer overwritten right after the call
    P = frames[0].copy()
    out = np.empty((VL, 3), np.float32)
    H.subdivide_host(P, out=out)
    P[:] = 0.0
    torch.cuda.current_stream().synchronize()
    ref = D.subdivide(torch.from_numpy(frames[0]).cuda()).cpu().numpy()
    np.testing.assert_array_equal(out, ref)
    D.status()
