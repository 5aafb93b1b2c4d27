"""alsub_refine_vertices_static: the vertex refinement entry point that allocates nothing.

It serves callers that cannot allocate device memory when they refine (code inside another
allocator's callback, a host that forbids device allocation after start-up) and cannot pass scratch
of their own: it keeps the intermediate levels in a fixed array inside the library and launches its
kernels directly, never through a CUDA graph. These tests call it through the C ABI and check it
against alsub_refine_vertices and the oracle, within the position tolerance the parity tests use
(2e-6 x bounding-box diagonal), on two calls in a row and on repeated calls into the same output
buffer, which must leave the device's free memory unchanged. The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

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
    return ref, outs, T, M, P0


CASES = [
    ("cc", synth.workload("cc_torus16_L3"), 3),
    ("cc", synth.torus_cc_mixed(40, 40, seed=51), 3),
    ("loop", synth.torus_tri(24, 24, seed=52), 3),
    ("sqrt3", synth.torus_tri(24, 24, seed=53, creases=False), 4),
]


@pytest.mark.parametrize("scheme,mesh,levels", CASES)
def test_static_scratch_matches_refine_vertices(scheme, mesh, levels):
    ref, outs, T, M, _ = _both(mesh, scheme, levels)
    diag = float(np.linalg.norm(ref.max(axis=0) - ref.min(axis=0)))
    for out in outs:
        assert out.shape == ref.shape
        assert float(np.abs(out - ref).max()) <= TOL * diag


@pytest.mark.parametrize("scheme,mesh,levels", CASES[1:])
def test_static_scratch_repeated_calls_match_oracle_and_allocate_nothing(scheme, mesh, levels):
    """Repeated calls into the same buffers: results equal the oracle's, free memory stays put."""
    import torch
    from paper_1809_06047_gb300 import alsub
    M = alsub.Mesh.from_dict(mesh, scheme)
    T = alsub.Topology(M, levels, build=True)
    P0 = torch.from_numpy(np.ascontiguousarray(mesh["P"], dtype=np.float32)).cuda()
    out = torch.empty((T.counts[-1]["V"], 3), dtype=torch.float32, device="cuda")
    T.refine_vertices_static(P0, out=out)              # set-up call (loads the array's module)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):                                 # the same pointers every time
        T.refine_vertices_static(P0, out=out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    T.status()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    gpu = gpu_util.gpu_run(mesh, scheme, levels, mode="static", per_level=False)
    gpu[-1]["P"] = out.cpu().numpy()
    ref = oracle.subdivide(mesh, levels, scheme, keep_all=True)
    gpu_util.compare(scheme, gpu, ref, pos_levels={levels})


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
