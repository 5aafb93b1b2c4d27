"""alsub_refine_vertices_static: the vertex refinement entry point that allocates nothing.

It serves callers that cannot allocate device memory when they refine (and cannot pass scratch of
their own); it keeps the intermediate levels in a fixed array inside the library. These tests call
it through the C ABI and check it against alsub_refine_vertices, within the position tolerance the
parity tests use (2e-6 x bounding-box diagonal), on two calls in a row. The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

from paper_1809_06047_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 2e-6


def _both(mesh, scheme, levels):
    import torch
    from paper_1809_06047_gb300 import alsub
    M = alsub.Mesh.from_dict(mesh, scheme)
    T = alsub.Topology(M, levels, build=True)
    P0 = torch.from_numpy(np.ascontiguousarray(mesh["P"], dtype=np.float32)).cuda()
    ref = T.refine_vertices(P0).cpu().numpy()
    outs = []
    for _ in range(2):                                 # two calls in a row share the array
        outs.append(T.refine_vertices_static(P0).cpu().numpy())
    torch.cuda.synchronize()
    T.status()
    return ref, outs, T, M


@pytest.mark.parametrize("scheme,mesh,levels", [
    ("cc", synth.workload("cc_torus16_L3"), 3),
    ("cc", synth.torus_cc_mixed(40, 40, seed=51), 3),
    ("loop", synth.torus_tri(24, 24, seed=52), 3),
    ("sqrt3", synth.torus_tri(24, 24, seed=53, creases=False), 4),
])
def test_static_scratch_matches_refine_vertices(scheme, mesh, levels):
    ref, outs, T, M = _both(mesh, scheme, levels)
    diag = float(np.linalg.norm(ref.max(axis=0) - ref.min(axis=0)))
    for out in outs:
        assert out.shape == ref.shape
        assert float(np.abs(out - ref).max()) <= TOL * diag


def test_static_scratch_rejects_too_large():
    """Intermediate levels beyond the fixed 32 MiB array are refused with a clear error."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.workload("cc_creased_torus96_L6")
    M = alsub.Mesh.from_dict(m, "cc")
    T = alsub.Topology(M, 5, build=True)
    assert T.scratch_bytes() > 32 << 20
    P0 = torch.from_numpy(m["P"]).cuda()
    with pytest.raises(alsub.AlsubError) as e:
        T.refine_vertices_static(P0)
    assert e.value.status == 3 and "32 MiB" in str(e.value)
