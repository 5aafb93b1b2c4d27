"""Selective subdivision (Sec. 3.4): extraction on the device against the oracle's extraction
(face tables, vertex and face maps, creases bit-exact), from the control mesh and from refined
levels, and feature-adaptive refinement (extract around the extraordinary vertices, refine one
level, repeat) against the same chain in the oracle, compared face corner by face corner."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _sparse(seed, n=20, m=16, creases=0.0):
    return synth.torus_cc_mixed(n, m, merge_frac=0.03, split_frac=0.02, crease_frac=creases, seed=seed)


def _gpu_mesh_dict(sub):
    """Face table, maps and creases of an extracted mesh handle (read through a level-0 topology)."""
    from paper_1809_06047_gb300 import alsub
    T = alsub.Topology(sub, 0, build=True)
    T.status()
    cv, cs = T.creases(0)
    vmap, fmap = sub.maps()
    d = dict(V=sub.V, F=sub.F, fv=T.faces(0), crease_verts=cv, crease_sharp=cs, vmap=vmap, fmap=fmap)
    T.close()
    return d


def _same(got, ref):
    assert (got["V"], got["F"]) == (ref["V"], ref["F"])
    np.testing.assert_array_equal(got["fv"], ref["fv"])
    np.testing.assert_array_equal(got["vmap"], ref["vmap"])
    np.testing.assert_array_equal(got["fmap"], ref["fmap"])
    # a crease list is read back with each edge oriented from its owner corner: compare edges
    gv = np.sort(np.asarray(got["crease_verts"]).reshape(-1, 2), axis=1)
    rv = np.sort(np.asarray(ref["crease_verts"]).reshape(-1, 2), axis=1)
    np.testing.assert_array_equal(gv, rv)
    np.testing.assert_array_equal(got["crease_sharp"], ref["crease_sharp"])


@pytest.mark.parametrize("name,mesh,rings,select", [
    ("sparse_evs_r1", lambda: _sparse(91), 1, None),
    ("sparse_evs_r2", lambda: _sparse(92), 2, None),
    ("sparse_evs_creases_r2", lambda: _sparse(93, creases=0.04), 2, None),
    ("holes_mask_r3", lambda: synth.holed_cc_mixed(20, 16, holes=4, seed=94), 3, "mask"),
    ("mixed_dense_r1", lambda: synth.torus_cc_mixed(16, 16, seed=95), 1, None),
])
def test_extract_control_mesh(name, mesh, rings, select):
    import torch
    from paper_1809_06047_gb300 import alsub
    m = mesh()
    M = alsub.Mesh.from_dict(m, "cc")
    T = alsub.Topology(M, 1, build=True)
    sel_np = None
    sel = None
    if select == "mask":
        sel_np = np.zeros(m["V"], np.uint8)
        sel_np[np.random.default_rng(3).choice(m["V"], 6, replace=False)] = 1
        sel = torch.from_numpy(sel_np).cuda()
    sub = T.extract(0, sel, rings)
    got = _gpu_mesh_dict(sub)
    ref = oracle.extract(m, None if sel_np is None else sel_np.astype(bool), rings)
    _same(got, ref)
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"])).cuda()
    np.testing.assert_array_equal(sub.gather(P0).cpu().numpy(), m["P"][ref["vmap"]])


def test_extract_refined_level():
    """Extraction from level 2 of a built topology: the oracle extracts from the same level (the
    CUDA path's own numbering), so the result must agree bit for bit."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = _sparse(96, 12, 10, creases=0.05)
    M = alsub.Mesh.from_dict(m, "cc")
    T = alsub.Topology(M, 3, build=True)
    P = T.refine_vertices(torch.from_numpy(np.ascontiguousarray(m["P"])).cuda())
    torch.cuda.synchronize()
    T.status()
    for l in (1, 2):
        c = T.counts[l]
        cv, cs = T.creases(l)
        lvl = dict(V=c["V"], F=c["F"], off=np.arange(c["F"] + 1, dtype=np.int32) * 4, fv=T.faces(l),
                   crease_verts=cv, crease_sharp=cs)
        sub = T.extract(l, None, 2)
        _same(_gpu_mesh_dict(sub), oracle.extract(lvl, None, 2))


def test_feature_adaptive_chain():
    """Three rounds of (extract two rings around the extraordinary vertices, refine one level) on
    the device and in the oracle: the same faces in the same order, positions within 2e-6 x the
    bounding-box diagonal corner by corner."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = _sparse(97, 18, 14)
    levels = 3
    # device chain: the source of each round is level 1 of the previous round's topology
    M = alsub.Mesh.from_dict(m, "cc")
    P = torch.from_numpy(np.ascontiguousarray(m["P"])).cuda()
    T = alsub.Topology(M, 0, build=True)
    keep, lvl = [M, T], 0
    for _ in range(levels):
        sub = T.extract(lvl, None, 2)
        Ps = sub.gather(P)
        T = alsub.Topology(sub, 1, build=True)
        P = T.refine_vertices(Ps)
        torch.cuda.synchronize()
        T.status()
        keep += [sub, T]
        lvl = 1
    gfv, gP = T.faces(1), P.cpu().numpy()
    # oracle chain
    cur = dict(m, P=m["P"].astype(np.float64))
    for _ in range(levels):
        e = oracle.extract(cur, None, 2)
        cur = oracle.subdivide(e, 1, "cc")[1]
    assert len(gfv) == len(cur["fv"])
    a, b = gP[gfv], cur["P"][cur["fv"]]
    diag = float(np.linalg.norm(b.max(0) - b.min(0)))
    assert float(np.abs(a - b).max()) <= gpu_util.POS_TOL * diag


def _loop_mesh(seed):
    return synth.torus_tri(32, 24, flip_frac=0.01, sharp_frac=0.004, seed=seed)


@pytest.mark.parametrize("rings", [1, 2])
def test_extract_loop_control_mesh(rings):
    """Loop: extraction around the valence != 6 vertices and the crease ends, bit-exact against the
    oracle; the extracted mesh is open and refines with the boundary rules."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = _loop_mesh(110 + rings)
    M = alsub.Mesh.from_dict(m, "loop")
    T = alsub.Topology(M, 1, build=True)
    sub = T.extract(0, None, rings)
    got = _gpu_mesh_dict(sub)
    ref = oracle.extract(m, None, rings, scheme="loop")
    _same(got, ref)
    assert sub.boundary_edges > 0
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"])).cuda()
    np.testing.assert_array_equal(sub.gather(P0).cpu().numpy(), m["P"][ref["vmap"]])


def test_extract_loop_refined_level():
    import torch
    from paper_1809_06047_gb300 import alsub
    m = _loop_mesh(113)
    M = alsub.Mesh.from_dict(m, "loop")
    T = alsub.Topology(M, 2, build=True)
    T.refine_vertices(torch.from_numpy(np.ascontiguousarray(m["P"])).cuda())
    torch.cuda.synchronize()
    T.status()
    for l in (1, 2):
        c = T.counts[l]
        cv, cs = T.creases(l)
        lvl = dict(V=c["V"], F=c["F"], off=np.arange(c["F"] + 1, dtype=np.int32) * 3, fv=T.faces(l),
                   crease_verts=cv, crease_sharp=cs)
        sub = T.extract(l, None, 2)
        _same(_gpu_mesh_dict(sub), oracle.extract(lvl, None, 2, scheme="loop"))


def test_loop_feature_adaptive_chain():
    """Three rounds of (extract two rings, refine one Loop level) on the device and in the oracle:
    the same faces, positions within 2e-6 x the bounding-box diagonal corner by corner."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = _loop_mesh(114)
    M = alsub.Mesh.from_dict(m, "loop")
    P = torch.from_numpy(np.ascontiguousarray(m["P"])).cuda()
    T = alsub.Topology(M, 0, build=True)
    keep, lvl = [M, T], 0
    for _ in range(3):
        sub = T.extract(lvl, None, 2)
        Ps = sub.gather(P)
        T = alsub.Topology(sub, 1, build=True)
        P = T.refine_vertices(Ps)
        torch.cuda.synchronize()
        T.status()
        keep += [sub, T]
        lvl = 1
    gfv, gP = T.faces(1), P.cpu().numpy()
    cur = dict(m, P=m["P"].astype(np.float64))
    for _ in range(3):
        e = oracle.extract(cur, None, 2, scheme="loop")
        cur = oracle.subdivide(e, 1, "loop")[1]
    assert len(gfv) == len(cur["fv"])
    a, b = gP[gfv], cur["P"][cur["fv"]]
    diag = float(np.linalg.norm(b.max(0) - b.min(0)))
    assert float(np.abs(a - b).max()) <= gpu_util.POS_TOL * diag
