"""Mesh reordering (Sec. 4.5) on the device against the oracle's reverse Cuthill-McKee: vertex and
face maps, face table and creases bit-exact (the order is unique: ties go by degree, then index;
faces with the same least vertex keep their input order), positions gathered exactly, and the
reordered mesh refined by the CUDA path against the oracle's refinement of the oracle's reordering."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _shuffled(m, seed):
    rng = np.random.default_rng(seed)
    pv = rng.permutation(m["V"])
    order = rng.permutation(m["F"])
    off, fv = np.asarray(m["off"]), np.asarray(m["fv"])
    faces = [pv[fv[off[r]:off[r + 1]]] for r in order]
    noff = np.zeros(m["F"] + 1, np.int32)
    noff[1:] = np.cumsum([len(f) for f in faces])
    out = dict(m, off=noff, fv=np.concatenate(faces).astype(np.int32),
               P=np.ascontiguousarray(np.asarray(m["P"])[np.argsort(pv)]))
    if "crease_verts" in m:
        out["crease_verts"] = pv[np.asarray(m["crease_verts"])].astype(np.int32).reshape(-1, 2)
    return out


def _two_components(a, b):
    """Disjoint union of two meshes (b's ids after a's)."""
    cv = [np.asarray(a.get("crease_verts", np.zeros((0, 2))), np.int32).reshape(-1, 2),
          np.asarray(b.get("crease_verts", np.zeros((0, 2))), np.int32).reshape(-1, 2) + a["V"]]
    cs = [np.asarray(a.get("crease_sharp", np.zeros(0)), np.float32).reshape(-1),
          np.asarray(b.get("crease_sharp", np.zeros(0)), np.float32).reshape(-1)]
    return dict(V=a["V"] + b["V"], F=a["F"] + b["F"],
                off=np.concatenate([a["off"][:-1], np.asarray(b["off"]) + a["off"][-1]]).astype(np.int32),
                fv=np.concatenate([a["fv"], np.asarray(b["fv"]) + a["V"]]).astype(np.int32),
                P=np.concatenate([a["P"], b["P"]]), crease_verts=np.concatenate(cv), crease_sharp=np.concatenate(cs))


def _live_creases(m):
    cs = np.asarray(m.get("crease_sharp", np.zeros(0)), np.float32).reshape(-1)
    cv = np.asarray(m.get("crease_verts", np.zeros((0, 2))), np.int32).reshape(-1, 2)
    return dict(m, crease_verts=cv[cs > 0], crease_sharp=cs[cs > 0])


def _soup(n, seed=9):
    """n disjoint quads (n components, every vertex of degree 2)."""
    fv = np.arange(4 * n, dtype=np.int32)
    P = np.random.default_rng(seed).standard_normal((4 * n, 3)).astype(np.float32)
    return dict(V=4 * n, F=n, off=np.arange(n + 1, dtype=np.int32) * 4, fv=fv, P=P,
                crease_verts=np.zeros((0, 2), np.int32), crease_sharp=np.zeros(0, np.float32))


def _one(k, seed=10):
    """A single k-gon."""
    P = np.random.default_rng(seed).standard_normal((k, 3)).astype(np.float32)
    return dict(V=k, F=1, off=np.array([0, k], np.int32), fv=np.arange(k, dtype=np.int32), P=P,
                crease_verts=np.zeros((0, 2), np.int32), crease_sharp=np.zeros(0, np.float32))


CASES = [
    ("single_triangle", "loop", lambda: _one(3)),
    ("single_quad", "cc", lambda: _one(4)),
    ("single_heptagon", "cc", lambda: _one(7)),
    ("seven_components", "cc", lambda: _shuffled(_soup(7), 11)),
    ("cc_mixed_creased", "cc", lambda: _shuffled(synth.torus_cc_mixed(20, 16, merge_frac=0.03, split_frac=0.02,
                                                                      crease_frac=0.05, seed=81), 1)),
    ("cc_holed", "cc", lambda: _shuffled(synth.holed_cc_mixed(20, 16, holes=4, seed=82), 2)),
    ("cc_two_components", "cc", lambda: _two_components(synth.torus_cc_mixed(8, 6, seed=83),
                                                        _shuffled(synth.torus_cc_plain(6, 5), 3))),
    ("cc_generator_order", "cc", lambda: synth.torus_cc_mixed(16, 12, seed=84)),
    ("loop_torus", "loop", lambda: _shuffled(synth.torus_tri(16, 12, seed=85), 4)),
    ("sqrt3_torus", "sqrt3", lambda: _shuffled(synth.torus_tri(12, 10, seed=86, creases=False), 5)),
    ("cc_bench_mesh_shuffled", "cc", lambda: _shuffled(synth.workload("cc_creased_torus96_L6"), 6)),
]


@pytest.mark.parametrize("name,scheme,mesh", CASES, ids=[c[0] for c in CASES])
def test_reorder_bit_exact(name, scheme, mesh):
    import torch
    from paper_1809_06047_gb300 import alsub
    m = _live_creases(mesh())
    if scheme == "sqrt3":
        m = dict(m, crease_verts=np.zeros((0, 2), np.int32), crease_sharp=np.zeros(0, np.float32))
    M = alsub.Mesh.from_dict(m, scheme)
    R = M.reorder()
    got = R.arrays()
    vmap, fmap = R.maps()
    ref = oracle.rcm_reorder(m)
    assert (R.V, R.F, R.nnz) == (ref["V"], ref["F"], len(ref["fv"]))
    assert R.boundary_edges == M.boundary_edges
    np.testing.assert_array_equal(vmap, ref["vmap"])
    np.testing.assert_array_equal(fmap, ref["fmap"])
    np.testing.assert_array_equal(got["off"], ref["off"])
    np.testing.assert_array_equal(got["fv"], ref["fv"])
    np.testing.assert_array_equal(got["crease_verts"], ref["crease_verts"])
    np.testing.assert_array_equal(got["crease_sharp"], ref["crease_sharp"])
    assert R.rcm_levels >= 1
    P = torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda()
    np.testing.assert_array_equal(R.gather(P).cpu().numpy(), np.asarray(m["P"], np.float32)[ref["vmap"]])
    R.close()
    M.close()


@pytest.mark.parametrize("scheme,mesh", [
    ("cc", lambda: _shuffled(synth.torus_cc_mixed(12, 10, crease_frac=0.06, seed=87), 7)),
    ("loop", lambda: _shuffled(synth.torus_tri(10, 8, seed=88), 8)),
])
def test_reordered_mesh_refines_like_the_oracle(scheme, mesh):
    """Three levels of the device-reordered mesh (refined from its own handle) on the CUDA path
    against three oracle levels of the oracle-reordered mesh (the same mesh, by the test above):
    topology equal after canonical relabelling, creases equal, level-3 positions within 2e-6 x the
    bounding-box diagonal."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = _live_creases(mesh())
    M = alsub.Mesh.from_dict(m, scheme)
    R = M.reorder()
    P = R.gather(torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda())
    T = alsub.Topology(R, 3, build=True)
    PL = T.refine_vertices(P)
    torch.cuda.synchronize()
    T.status()
    gpu = []
    for l in range(4):
        d = dict(T.counts[l])
        d["fv"] = T.faces(l)
        d["crease_verts"], d["crease_sharp"] = T.creases(l)
        gpu.append(d)
    gpu[3]["P"] = PL.cpu().numpy()
    T.close()
    R.close()
    M.close()
    ref = oracle.subdivide(oracle.rcm_reorder(m), 3, scheme)
    gpu_util.compare(scheme, gpu, ref, pos_levels={3})


def test_maps_of_a_plain_mesh_are_refused():
    from paper_1809_06047_gb300 import alsub
    M = alsub.Mesh.from_dict(synth.torus_cc_plain(4, 4), "cc")
    with pytest.raises(Exception):
        M.maps()
    M.close()
