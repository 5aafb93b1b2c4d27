"""The caller's allocator (alsub_mesh_create_ex, the boundary's allocator callback): a mesh made
with it, and every handle made from that mesh (topologies static and dynamic, host-buffer staging,
hierarchical edits, operators, extracted and reordered meshes), takes all of its device memory from
the callbacks and gives all of it back when destroyed; results are bit-identical to the default
allocator's. An allocator that has no memory makes the calls fail with OOM."""
import numpy as np
import pytest

from paper_1809_06047_gb300 import synth

pytestmark = pytest.mark.gpu


def _pair(m, scheme, A):
    from paper_1809_06047_gb300 import alsub
    return alsub.Mesh.from_dict(m, scheme, allocator=A), alsub.Mesh.from_dict(m, scheme)


@pytest.mark.parametrize("scheme,mesh,levels", [
    ("cc", synth.torus_cc_mixed(20, 20, crease_frac=0.1, seed=61), 4),
    ("cc", synth.holed_cc_mixed(16, 12, holes=2, seed=62), 3),
    ("loop", synth.torus_tri(12, 10, seed=63), 3),
    ("sqrt3", synth.torus_tri(12, 10, seed=64, creases=False), 3),
])
def test_caller_allocator_holds_everything_and_matches(scheme, mesh, levels):
    import torch
    from paper_1809_06047_gb300 import alsub
    A = alsub.DeviceAllocator()
    P0 = torch.from_numpy(np.ascontiguousarray(mesh["P"], dtype=np.float32)).cuda()
    M, MD = _pair(mesh, scheme, A)
    n_mesh = A.allocs
    assert n_mesh >= 2                         # face offsets and corners at least
    # static and dynamic topologies
    T, TD = alsub.Topology(M, levels), alsub.Topology(MD, levels)
    assert A.bytes_live >= T.bytes()
    assert torch.equal(T.refine_vertices(P0), TD.refine_vertices(P0))
    Tdyn, TDdyn = alsub.Topology(M, levels, build=False), alsub.Topology(MD, levels, build=False)
    assert torch.equal(Tdyn.subdivide(P0), TDdyn.subdivide(P0))
    # host-buffer staging
    hP0 = P0.cpu().pin_memory()
    a, b = Tdyn.subdivide_host(hP0), TDdyn.subdivide_host(hP0)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # hierarchical edits on level 1
    vid = np.arange(0, T.counts[1]["V"], 7, dtype=np.int32)
    off = np.full((len(vid), 3), 0.01, dtype=np.float32)
    T.set_edits(1, vid, off)
    TD.set_edits(1, vid, off)
    assert torch.equal(T.refine_vertices(P0), TD.refine_vertices(P0))
    T.set_edits(1)
    TD.set_edits(1)
    # operators (chain, composite, transposes)
    O = alsub.Operator(T, chain=True, compose=True, transpose=True)
    OD = alsub.Operator(TD, chain=True, compose=True, transpose=True)
    assert torch.equal(O.apply(P0), OD.apply(P0))
    gL = torch.ones((T.counts[-1]["V"], 3), dtype=torch.float32, device="cuda")
    assert torch.equal(O.apply_transpose(gL), OD.apply_transpose(gL))
    # extraction and reordering make meshes that keep the allocator
    extra = []
    if scheme != "sqrt3":
        E, ED = T.extract(1), TD.extract(1)
        assert E._allocator is A
        TE, TED = alsub.Topology(E, 2), alsub.Topology(ED, 2)
        T1 = alsub.Topology(M, 1)
        PE = E.gather(T1.refine_vertices(P0))
        assert torch.equal(TE.refine_vertices(PE), TED.refine_vertices(PE))
        extra += [TE, E, TED, ED, T1]
    R, RD = M.reorder(), MD.reorder()
    assert R._allocator is A
    TR, TRD = alsub.Topology(R, 2), alsub.Topology(RD, 2)
    PR = R.gather(P0)
    assert torch.equal(TR.refine_vertices(PR), TRD.refine_vertices(PR))
    torch.cuda.synchronize()
    for h in (T, TD, Tdyn, TDdyn):
        h.status()
    for h in [O, OD, TR, TRD, R, RD] + extra + [T, TD, Tdyn, TDdyn, M, MD]:
        h.close()
    torch.cuda.synchronize()
    assert A.allocs > n_mesh
    assert A.bytes_live == 0 and not A.live and A.frees == A.allocs


def test_handles_released_parent_first():
    """A handle's release reads nothing of the handle it was made from, so the mesh, then the
    topology, then its operators (matrix-free, chain and transposes) may be destroyed in that
    order, as Python's cycle collector may do; every byte goes back to the caller's allocator."""
    import torch
    from paper_1809_06047_gb300 import alsub
    A = alsub.DeviceAllocator()
    m = synth.torus_cc_mixed(12, 10, crease_frac=0.1, seed=65)
    M = alsub.Mesh.from_dict(m, "cc", allocator=A)
    T = alsub.Topology(M, 3)
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda()
    ops = [alsub.Operator(T, chain=False, matrix_free=True), alsub.Operator(T, chain=True, transpose=True)]
    want = T.refine_vertices(P0)
    assert torch.equal(ops[0].apply(P0), want)
    torch.cuda.synchronize()
    M.close()
    T.close()
    for o in ops:
        o.close()
    torch.cuda.synchronize()
    assert A.bytes_live == 0 and not A.live and A.frees == A.allocs


def test_allocator_without_memory_is_oom():
    from paper_1809_06047_gb300 import alsub
    A = alsub.DeviceAllocator(fail=True)
    with pytest.raises(alsub.AlsubError) as e:
        alsub.Mesh.from_dict(synth.cube(), "cc", allocator=A)
    assert e.value.status == 4
    # a mesh made while memory lasted: its topology's allocation fails cleanly
    A.fail = False
    M = alsub.Mesh.from_dict(synth.cube(), "cc", allocator=A)
    A.fail = True
    with pytest.raises(alsub.AlsubError) as e:
        alsub.Topology(M, 2)
    assert e.value.status == 4
    A.fail = False
    M.close()
    assert A.bytes_live == 0
