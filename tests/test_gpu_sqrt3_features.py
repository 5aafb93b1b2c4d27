"""sqrt(3) with feature edges on the CUDA path: boundaries and infinitely sharp creases (Appendix A
gives neither; the oracle follows Kobbelt 2000: feature edges are not flipped on the first step of
each pair and split in three on the second, along the ternary cubic B-spline curve). Parity with the
oracle as for closed meshes (topology bit-exact after canonical relabelling, crease lists bit-exact,
positions within 2e-6 x bounding-box diagonal at every level) over both kinds of step, static and
dynamic, graph replay, the host-buffer call and the allocation-free entry point; the calls that have
no feature path refuse such meshes."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _corner_mesh():
    m = synth.torus_tri(8, 8, flip_frac=0.0, creases=False, jitter=0.04, seed=71)
    v = 3 * 8 + 3
    return dict(m, crease_verts=np.array([[v, v + 8], [v, v + 1], [v, v - 8], [v + 8, v + 16]], np.int32),
                crease_sharp=np.full(4, np.inf, np.float32))


FEATURES = [
    ("tube", lambda: synth.triangulate(synth.tube_cc(12, 7, seed=72)), 4),
    ("sheet", lambda: synth.triangulate(synth.sheet_cc(9, 7, seed=73)), 5),
    ("holes", lambda: synth.triangulate(synth.holed_cc_mixed(20, 16, holes=4, seed=74)), 4),
    ("triangle", lambda: synth.polygon(3), 5),
    ("creased_torus", lambda: synth.torus_tri(16, 14, seed=75), 5),
    ("corner_dart", _corner_mesh, 4),
    ("mixed_sharpness", lambda: synth.torus_tri(12, 10, seed=76, sharp_frac=0.1), 3),
    ("sheet_L1", lambda: synth.triangulate(synth.sheet_cc(5, 4, seed=77)), 1),
]


@pytest.mark.parametrize("name,fn,levels", FEATURES, ids=[c[0] for c in FEATURES])
@pytest.mark.parametrize("mode", ["static", "dynamic"])
def test_sqrt3_features_parity(name, fn, levels, mode):
    mesh = fn()
    if name == "mixed_sharpness":          # finite sharpness is ignored, infinite kept
        cs = mesh["crease_sharp"].copy()
        cs[::2] = 1.5
        mesh = dict(mesh, crease_sharp=cs)
    ref = oracle.subdivide(mesh, levels, "sqrt3", keep_all=True)
    gpu = gpu_util.gpu_run(mesh, "sqrt3", levels, mode=mode)
    gpu_util.compare("sqrt3", gpu, ref)


def test_sqrt3_features_graph_host_and_static_entry():
    """Repeated calls (captured and replayed), the host-buffer call and the allocation-free entry
    point give the bits of a one-off call; the counts are the closed forms with boundary edges."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.triangulate(synth.holed_cc_mixed(16, 12, holes=3, seed=78))
    m["crease_verts"], m["crease_sharp"] = np.zeros((0, 2), np.int32), np.zeros(0, np.float32)
    L = 4
    M = alsub.Mesh.from_dict(m, "sqrt3")
    B = M.boundary_edges
    plan = alsub.plan("sqrt3", m["V"], m["F"], len(m["fv"]), L, boundary=B)
    T = alsub.Topology(M, L, build=False)
    P0 = torch.from_numpy(m["P"]).cuda()
    outs = [T.subdivide(P0).clone() for _ in range(3)]
    Ts = alsub.Topology(M, L, build=True)
    a = Ts.refine_vertices(P0)
    b = Ts.refine_vertices(P0)
    c = Ts.refine_vertices_static(P0)
    h = T.subdivide_host(P0.cpu().pin_memory())
    torch.cuda.synchronize()
    T.status(); Ts.status()
    for x in outs[1:] + [a, b, c, h.cuda()]:
        assert torch.equal(x, outs[0])
    # closed-form counts: V + F (+ B on a second step), F x 3, boundary edges x 3 per pair
    Bl = B
    for l in range(L):
        cur, nxt = T.counts[l], T.counts[l + 1]
        extra = Bl if l % 2 == 1 else 0
        assert (nxt["V"], nxt["F"], nxt["E"]) == (cur["V"] + cur["F"] + extra, 3 * cur["F"],
                                                  cur["E"] + 3 * cur["F"] + extra)
        Bl = 3 * Bl if l % 2 == 1 else Bl
    assert [tuple(int(x) for x in r) for r in plan] == [tuple(T.counts[l][k] for k in ("V", "F", "nnz", "E"))
                                                        for l in range(L + 1)]


def test_sqrt3_features_refused_where_no_path():
    from paper_1809_06047_gb300 import alsub
    import torch
    m = synth.torus_tri(10, 8, seed=79)
    M = alsub.Mesh.from_dict(m, "sqrt3")
    T = alsub.Topology(M, 2)
    with pytest.raises(alsub.AlsubError) as e:
        alsub.Operator(T, chain=True)
    assert e.value.status == 3
    with pytest.raises(alsub.AlsubError) as e:
        alsub.Operator(T, chain=False, matrix_free=True, transpose=True)
    assert e.value.status == 3
    # the matrix-free operator needs no rows: it is the feature path's eval kernels
    op = alsub.Operator(T, chain=False, matrix_free=True)
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"], np.float32)).cuda()
    assert torch.equal(op.apply(P0), T.refine_vertices(P0))
    T.status()
    with pytest.raises(alsub.AlsubError) as e:
        alsub.Batch([T], [torch.from_numpy(m["P"]).cuda()])
    assert e.value.status == 3
