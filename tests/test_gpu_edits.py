"""Hierarchical edits between levels (Sec. 3.5 "Other effects") on the CUDA path against the
oracle's level-by-level refinement with the same offsets (vertex ids translated by the canonical
relabelling), through the static, dynamic (graph-replayed) and host-buffer calls."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import canon, gpu_util

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme,mesh", [
    ("cc", lambda: synth.torus_cc_mixed(12, 10, crease_frac=0.1, seed=101)),
    ("cc", lambda: synth.holed_cc_mixed(14, 12, holes=3, seed=102)),
    ("loop", lambda: synth.torus_tri(9, 8, seed=103)),
])
def test_edits_match_oracle(scheme, mesh):
    import torch
    from paper_1809_06047_gb300 import alsub
    m = mesh()
    L = 3
    ref_plain = oracle.subdivide(m, L, scheme, keep_all=True)
    M = alsub.Mesh.from_dict(m, scheme)
    T = alsub.Topology(M, L, build=True)
    D = alsub.Topology(M, L, build=False)
    counts = [dict(V=r["V"], F=r["F"], E=r["E"]) for r in ref_plain]
    pi = canon.vertex_maps(scheme, [T.faces(l) for l in range(L + 1)], [r["fv"] for r in ref_plain], counts)
    rng = np.random.default_rng(9)
    edits_gpu, edits_ref = {}, {}
    for l in (1, 2, 3):
        vid = rng.choice(T.counts[l]["V"], 7, replace=False).astype(np.int32)
        off = (0.05 * rng.standard_normal((7, 3))).astype(np.float32)
        edits_gpu[l] = (vid, off)
        edits_ref[l] = (pi[l][vid], off.astype(np.float64))
        T.set_edits(l, torch.from_numpy(vid).cuda(), torch.from_numpy(off).cuda())
        D.set_edits(l, vid, off)                     # host arrays
    ref = oracle.subdivide_edits(m, L, scheme, edits_ref)
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"])).cuda()
    outs = [T.refine_vertices(P0) for _ in range(3)]                  # direct, captured, replayed
    PL = torch.empty_like(outs[0])
    dyn = []
    for _ in range(3):
        D.subdivide(P0, out=PL)
        torch.cuda.synchronize()
        dyn.append(PL.clone())
    host = D.subdivide_host(torch.from_numpy(np.ascontiguousarray(m["P"])).pin_memory())
    torch.cuda.synchronize()
    T.status()
    D.status()
    for o in outs[1:] + dyn + [host.cuda()]:
        assert torch.equal(o.cuda(), outs[0])
    err, diag = canon.position_error(pi[L], outs[0].cpu().numpy(), ref[L]["P"])
    assert err <= gpu_util.POS_TOL * diag
    plain = ref_plain[L]["P"]
    assert canon.position_error(pi[L], outs[0].cpu().numpy(), plain)[0] > 10 * err   # the edits show
    # clearing the edits gives plain refinement again
    for l in (1, 2, 3):
        T.set_edits(l)
    err0, _ = canon.position_error(pi[L], T.refine_vertices(P0).cpu().numpy(), plain)
    assert err0 <= gpu_util.POS_TOL * diag


def test_edit_out_of_range_is_latched():
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.cube()
    M = alsub.Mesh.from_dict(m, "cc")
    T = alsub.Topology(M, 2, build=True)
    T.set_edits(2, np.array([10 ** 6], np.int32), np.zeros((1, 3), np.float32))
    T.refine_vertices(torch.from_numpy(np.ascontiguousarray(m["P"])).cuda())
    with pytest.raises(alsub.AlsubError) as e:
        T.status()
    assert e.value.status == 1
    with pytest.raises(alsub.AlsubError):
        T.set_edits(0, np.array([0], np.int32), np.zeros((1, 3), np.float32))   # level 0: the caller's P0
