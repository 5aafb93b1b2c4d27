"""Open Catmull-Clark and Loop meshes (Sec. 3.1 and 3.2 "Boundaries") on the CUDA path.

The boundary edge points are midpoints and the boundary vertices follow Eq. CC_boundary, written
by the repair step after the smooth eval (build and repair, Fig. module_boundary); Loop, for which
Appendix B gives no boundary rule, takes the same two rules (the oracle's reading, pinned by the
cubic B-spline boundary curves). Parity with the
oracle as for closed meshes: topology bit-exact after canonical relabelling, positions within
2e-6 x bounding-box diagonal at every level; the operator, its transpose, the dynamic and graph
paths and the server are checked on the same inputs.
"""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu

OPEN = [
    ("tube16x9", lambda: synth.tube_cc(16, 9, seed=51), 4),
    ("tube3x2", lambda: synth.tube_cc(3, 2, seed=52), 4),
    ("sheet", lambda: synth.sheet_cc(12, 9, seed=53), 4),
    ("holes", lambda: synth.holed_cc_mixed(24, 20, holes=6, seed=54), 4),
    ("box", synth.open_box, 5),
    ("quad", lambda: synth.polygon(4), 5),
    ("heptagon", lambda: synth.polygon(7), 4),
    ("sheet_L0", lambda: synth.sheet_cc(6, 5, seed=60), 0),
    ("box_L1", synth.open_box, 1),
]


def _boundary_edges(mesh):
    """Edges of one face, counted from the directed edges (a plain set computation)."""
    off, fv = mesh["off"], mesh["fv"]
    d = set()
    for r in range(mesh["F"]):
        f = fv[off[r]:off[r + 1]]
        for j in range(len(f)):
            d.add((int(f[j]), int(f[(j + 1) % len(f)])))
    return sum((b, a) not in d for a, b in d)


@pytest.mark.parametrize("name,fn,levels", OPEN, ids=[c[0] for c in OPEN])
@pytest.mark.parametrize("mode", ["static", "dynamic"])
def test_open_parity(name, fn, levels, mode):
    mesh = fn()
    ref = oracle.subdivide(mesh, levels, "cc", keep_all=True)
    gpu = gpu_util.gpu_run(mesh, "cc", levels, mode=mode)
    gpu_util.compare("cc", gpu, ref)


def test_boundary_count_and_plan_open():
    from paper_1809_06047_gb300 import alsub
    for _, fn, levels in OPEN:
        mesh = fn()
        M = alsub.Mesh.from_dict(mesh, "cc")
        B = _boundary_edges(mesh)
        assert M.boundary_edges == B > 0
        T = alsub.Topology(M, levels, build=True)
        T.status()
        plan = alsub.plan("cc", mesh["V"], mesh["F"], len(mesh["fv"]), levels, boundary=B)
        for l in range(levels + 1):
            c = T.counts[l]
            assert (c["V"], c["F"], c["nnz"], c["E"]) == tuple(int(x) for x in plan[l])
        T.close()
        M.close()
    M = alsub.Mesh.from_dict(synth.cube(), "cc")
    assert M.boundary_edges == 0


def test_open_repeated_calls_replay_graphs():
    """Repeated dynamic calls (direct, captured, replayed) give identical bits, equal to the static
    path."""
    import torch
    from paper_1809_06047_gb300 import alsub
    mesh = synth.holed_cc_mixed(20, 16, holes=4, seed=55)
    M = alsub.Mesh.from_dict(mesh, "cc")
    T = alsub.Topology(M, 4, build=False)
    S = alsub.Topology(M, 4, build=True)
    P0 = torch.from_numpy(np.ascontiguousarray(mesh["P"], dtype=np.float32)).cuda()
    PL = torch.empty((T.counts[-1]["V"], 3), dtype=torch.float32, device="cuda")
    outs = []
    for _ in range(4):
        T.subdivide(P0, out=PL)
        torch.cuda.synchronize()
        outs.append(PL.clone())
    ref = S.refine_vertices(P0)
    torch.cuda.synchronize()
    T.status()
    S.status()
    for o in outs:
        assert torch.equal(o, ref)


OP_CASES = [
    ("sheet", "cc", lambda: synth.sheet_cc(5, 4, seed=56), 3),
    ("holes", "cc", lambda: synth.holed_cc_mixed(10, 10, holes=3, seed=57), 3),
    ("box", "cc", synth.open_box, 3),
    ("quad", "cc", lambda: synth.polygon(4), 3),
    ("loop_sheet", "loop", lambda: synth.triangulate(synth.sheet_cc(5, 4, seed=68)), 3),
    ("loop_holes_creased", "loop", lambda: synth.triangulate(synth.holed_cc_mixed(10, 10, holes=3, seed=69)), 3),
    ("loop_box", "loop", lambda: synth.triangulate(synth.open_box()), 3),
]


@pytest.mark.parametrize("name,scheme,fn,levels", OP_CASES, ids=[c[0] for c in OP_CASES])
def test_open_operator(name, scheme, fn, levels):
    """Per-level rows equal the oracle's R_l entry by entry; chain, composite and their
    transposes reproduce the positions and the oracle's R^T g."""
    import scipy.sparse as sp
    import torch
    from paper_1809_06047_gb300 import alsub
    from tests import canon
    mesh = fn()
    ref = oracle.subdivide(mesh, levels, scheme, keep_all=True, operator=True)
    M = alsub.Mesh.from_dict(mesh, scheme)
    T = alsub.Topology(M, levels, build=True)
    P0 = torch.from_numpy(np.ascontiguousarray(mesh["P"], dtype=np.float32)).cuda()
    counts = [dict(V=r["V"], F=r["F"], E=r["E"]) for r in ref]
    pi = canon.vertex_maps(scheme, [T.faces(l) for l in range(levels + 1)], [r["fv"] for r in ref], counts)
    chain = alsub.Operator(T, chain=True, transpose=True)
    comp = alsub.Operator(T, chain=False, compose=True, transpose=True)
    T.status()
    Rs = []
    for l in range(levels):
        shape = (ref[l + 1]["V"], ref[l]["V"])
        rp, col, w = chain.csr(l)
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        G = sp.csr_matrix((w.astype(np.float64), (pi[l + 1][rows], pi[l][col.astype(np.int64)])), shape=shape)
        O = sp.csr_matrix((ref[l]["R_w"], (ref[l]["R_rows"], ref[l]["R_cols"])), shape=shape)
        assert (G != 0).nnz == (O != 0).nnz == G.nnz
        assert abs(G - O).max() <= 1e-6
        Rs.append(O)
    Rc = Rs[0]
    for l in range(1, levels):
        Rc = Rs[l] @ Rc
    for opx in (chain, comp):
        got = opx.apply(P0).cpu().numpy()
        err, diag = canon.position_error(pi[levels], got, ref[levels]["P"])
        assert err <= gpu_util.POS_TOL * diag
    rng = np.random.default_rng(7)
    gL = rng.standard_normal((ref[levels]["V"], 3)).astype(np.float32)
    want = Rc.T @ gL[np.argsort(pi[levels])].astype(np.float64)
    for opx in (chain, comp):
        g0 = opx.apply_transpose(torch.from_numpy(gL).cuda()).cpu().numpy()
        np.testing.assert_allclose(g0, want, atol=1e-4 * np.abs(want).max())


def test_open_mesh_errors():
    from paper_1809_06047_gb300 import alsub
    box = synth.open_box()
    rim = box["fv"][:4]                         # face x = -1: edge (0, 1) ends on the rim (z = +1)
    cre = dict(box, crease_verts=np.array([[rim[0], rim[1]]], np.int32),
               crease_sharp=np.array([2.0], np.float32))
    with pytest.raises(alsub.AlsubError) as e:     # a crease meets the boundary
        alsub.Mesh.from_dict(cre, "cc")
    assert e.value.status == 3
    o = synth.octahedron()
    open_tri = dict(o, F=6, off=o["off"][:7], fv=o["fv"][:18])
    # sqrt(3): Kobbelt's boundary treatment (the feature path); a sharp crease at its boundary is
    # refused as for the other schemes
    M = alsub.Mesh.from_dict(open_tri, "sqrt3")
    assert M.boundary_edges == 4
    M.close()
    t = synth.triangulate(box)
    with pytest.raises(alsub.AlsubError) as e:
        alsub.Mesh.from_dict(dict(t, crease_verts=np.array([[rim[0], rim[1]]], np.int32),
                                  crease_sharp=np.array([np.inf], np.float32)), "sqrt3")
    assert e.value.status == 3
    M = alsub.Mesh.from_dict(open_tri, "loop")     # Loop: the rules of Eq. CC_boundary
    assert M.boundary_edges == 4
    M.close()
    # two squares sharing one vertex: two fans there
    bow = dict(V=7, F=2, off=np.array([0, 4, 8], np.int32), fv=np.array([0, 1, 2, 3, 0, 4, 5, 6], np.int32),
               P=np.random.default_rng(1).standard_normal((7, 3)).astype(np.float32),
               crease_verts=np.zeros((0, 2), np.int32), crease_sharp=np.zeros(0, np.float32))
    M = alsub.Mesh.from_dict(bow, "cc")
    with pytest.raises(alsub.AlsubError) as e:
        T = alsub.Topology(M, 2, build=True)
        T.status()
    assert e.value.status == 2
    # ragged batches have no repair step
    M = alsub.Mesh.from_dict(synth.sheet_cc(4, 3, seed=58), "cc")
    T = alsub.Topology(M, 2, build=True)
    import torch
    P0 = torch.zeros((M.V, 3), device="cuda")
    PL = torch.empty((T.counts[-1]["V"], 3), device="cuda")
    with pytest.raises(alsub.AlsubError) as e:
        alsub.Batch([T], [P0], [PL])
    assert e.value.status == 3


def test_open_mesh_served():
    """A one-off open mesh through the server equals a direct subdivide; a wrong boundary count
    in the request fails that request only."""
    import torch
    from paper_1809_06047_gb300 import alsub
    mesh = synth.holed_cc_mixed(16, 12, holes=3, seed=59)
    M = alsub.Mesh.from_dict(mesh, "cc")
    T = alsub.Topology(M, 3, build=True)
    ref = T.refine_vertices(torch.from_numpy(np.ascontiguousarray(mesh["P"])).cuda()).cpu().numpy()
    T.status()
    S = alsub.Server(1 << 30, 2)
    try:
        good = S.submit_mesh(mesh, "cc", 3, boundary_edges=M.boundary_edges)
        bad = S.submit_mesh(mesh, "cc", 3, boundary_edges=M.boundary_edges + 2)
        r = None
        while r is None:
            r = S.poll(good, 100000)
        assert r["status"] == 0
        np.testing.assert_array_equal(r["P"], ref)
        r = None
        while r is None:
            r = S.poll(bad, 100000)
        assert r["status"] == 1
    finally:
        S.close()


def _triangle():
    return dict(V=3, F=1, off=np.array([0, 3], np.int32), fv=np.array([0, 1, 2], np.int32),
                P=np.array([[0, 0, 0], [1, 0, 0.2], [0.3, 1, -0.1]], np.float32),
                crease_verts=np.zeros((0, 2), np.int32), crease_sharp=np.zeros(0, np.float32))


OPEN_LOOP = [
    ("tube16x9", lambda: synth.triangulate(synth.tube_cc(16, 9, seed=61)), 4),
    ("tube3x2", lambda: synth.triangulate(synth.tube_cc(3, 2, seed=62)), 4),
    ("sheet", lambda: synth.triangulate(synth.sheet_cc(12, 9, seed=63)), 4),
    ("holes_creased", lambda: synth.triangulate(synth.holed_cc_mixed(24, 20, holes=6, seed=64)), 4),
    ("box", lambda: synth.triangulate(synth.open_box()), 4),
    ("triangle", _triangle, 4),
    ("sheet_L1", lambda: synth.triangulate(synth.sheet_cc(6, 5, seed=65)), 1),
    ("sheet_L0", lambda: synth.triangulate(synth.sheet_cc(6, 5, seed=66)), 0),
]


@pytest.mark.parametrize("name,fn,levels", OPEN_LOOP, ids=[c[0] for c in OPEN_LOOP])
@pytest.mark.parametrize("mode", ["static", "dynamic"])
def test_open_loop_parity(name, fn, levels, mode):
    """Open Loop meshes: every level against the oracle (topology after canonical relabelling,
    creases, positions within 2e-6 x diagonal), and the boundary count and level counts."""
    from paper_1809_06047_gb300 import alsub
    mesh = fn()
    B = _boundary_edges(mesh)
    M = alsub.Mesh.from_dict(mesh, "loop")
    assert M.boundary_edges == B > 0
    plan = alsub.plan("loop", mesh["V"], mesh["F"], len(mesh["fv"]), levels, boundary=B)
    M.close()
    ref = oracle.subdivide(mesh, levels, "loop", keep_all=True)
    for l in range(levels + 1):
        assert (ref[l]["V"], ref[l]["F"], ref[l]["E"]) == (int(plan[l][0]), int(plan[l][1]), int(plan[l][3]))
    gpu = gpu_util.gpu_run(mesh, "loop", levels, mode=mode)
    gpu_util.compare("loop", gpu, ref)


def test_open_loop_repeated_calls_replay_graphs():
    import torch
    from paper_1809_06047_gb300 import alsub
    mesh = synth.triangulate(synth.holed_cc_mixed(20, 16, holes=4, seed=67))
    M = alsub.Mesh.from_dict(mesh, "loop")
    T = alsub.Topology(M, 4, build=False)
    S = alsub.Topology(M, 4, build=True)
    P0 = torch.from_numpy(np.ascontiguousarray(mesh["P"], dtype=np.float32)).cuda()
    PL = torch.empty((T.counts[-1]["V"], 3), dtype=torch.float32, device="cuda")
    outs = []
    for _ in range(4):
        T.subdivide(P0, out=PL)
        torch.cuda.synchronize()
        outs.append(PL.clone())
    ref = S.refine_vertices(P0)
    torch.cuda.synchronize()
    T.status()
    S.status()
    for o in outs:
        assert torch.equal(o, ref)
