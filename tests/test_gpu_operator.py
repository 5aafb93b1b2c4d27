"""Parity of the subdivision operator (Sec. 3.6, single SpMV) with the oracle's operator.

R_l from the CUDA path is compared entry by entry with the oracle's R_l after canonical
relabelling of rows (level l+1 vertices) and columns (level l vertices): identical sparsity, FP32
weights within 1e-6 of the FP64 weights. Apply, composite and transpose are checked against the
oracle's positions and scipy products of the oracle's matrices.
"""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import canon, gpu_util

pytestmark = pytest.mark.gpu

W_TOL = 1e-6

CASES = [
    ("cc", lambda: synth.torus_cc_mixed(8, 10, crease_frac=0.2, seed=61), 3),
    ("cc", synth.cube, 3),
    ("cc", lambda: synth.pillow(5), 3),
    ("loop", lambda: synth.torus_tri(7, 6, seed=62), 3),
    ("loop", synth.octahedron, 3),
    ("sqrt3", lambda: synth.torus_tri(6, 7, seed=63, creases=False), 3),
]


def _setup(mesh, scheme, levels):
    import torch
    from paper_1809_06047_gb300 import alsub
    M = alsub.Mesh.from_dict(mesh, scheme)
    T = alsub.Topology(M, levels, build=True)
    P0 = torch.from_numpy(np.ascontiguousarray(mesh["P"], dtype=np.float32)).cuda()
    return M, T, P0


def _maps(scheme, T, ref):
    counts = [dict(V=r["V"], F=r["F"], E=r["E"]) for r in ref]
    return canon.vertex_maps(scheme, [T.faces(l) for l in range(len(ref))],
                             [r["fv"] for r in ref], counts)


def _coo(rowptr, col, w):
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    return rows, col.astype(np.int64), w.astype(np.float64)


@pytest.mark.parametrize("scheme,fn,levels", CASES)
def test_per_level_operator_entries(scheme, fn, levels):
    import scipy.sparse as sp
    from paper_1809_06047_gb300 import alsub
    mesh = fn()
    ref = oracle.subdivide(mesh, levels, scheme, keep_all=True, operator=True)
    M, T, P0 = _setup(mesh, scheme, levels)
    op = alsub.Operator(T, chain=True)
    T.status()
    pi = _maps(scheme, T, ref)
    for l in range(levels):
        rp, col, w = op.csr(l)
        assert np.all(np.diff(rp) > 0)
        r, c, wv = _coo(rp, col, w)
        # every row sorted by column, no duplicates
        assert np.all((np.diff(c) > 0) | (np.diff(r) != 0))
        shape = (ref[l + 1]["V"], ref[l]["V"])
        G = sp.csr_matrix((wv, (pi[l + 1][r], pi[l][c])), shape=shape)
        O = sp.csr_matrix((ref[l]["R_w"], (ref[l]["R_rows"], ref[l]["R_cols"])), shape=shape)
        assert (G != 0).nnz == (O != 0).nnz == G.nnz
        assert abs(G - O).max() <= W_TOL
        np.testing.assert_allclose(np.asarray(G.sum(axis=1)).ravel(), 1.0, atol=1e-5)


@pytest.mark.parametrize("scheme,fn,levels", CASES)
def test_apply_chain_composite_transpose(scheme, fn, levels):
    import scipy.sparse as sp
    import torch
    from paper_1809_06047_gb300 import alsub
    mesh = fn()
    ref = oracle.subdivide(mesh, levels, scheme, keep_all=True, operator=True)
    M, T, P0 = _setup(mesh, scheme, levels)
    pi = _maps(scheme, T, ref)
    chain = alsub.Operator(T, chain=True, transpose=True)
    comp = alsub.Operator(T, chain=False, compose=True, transpose=True)
    a = chain.apply(P0).cpu().numpy()
    b = comp.apply(P0).cpu().numpy()
    T.status()
    for got in (a, b):
        err, diag = canon.position_error(pi[levels], got, ref[levels]["P"])
        assert err <= gpu_util.POS_TOL * diag
    # the oracle's composite operator and its transpose
    Rs = [sp.csr_matrix((ref[l]["R_w"], (ref[l]["R_rows"], ref[l]["R_cols"])),
                        shape=(ref[l + 1]["V"], ref[l]["V"])) for l in range(levels)]
    Rc = Rs[0]
    for l in range(1, levels):
        Rc = Rs[l] @ Rc
    rp, col, w = comp.csr(-1)
    r, c, wv = _coo(rp, col, w)
    G = sp.csr_matrix((wv, (pi[levels][r], c)), shape=Rc.shape)
    assert abs(G - Rc).max() <= 1e-5
    rng = np.random.default_rng(3)
    gL = rng.standard_normal((ref[levels]["V"], 3)).astype(np.float32)
    # gradient of the GPU-numbered level L: permute into the oracle's numbering for the check
    want = Rc.T @ gL[np.argsort(pi[levels])].astype(np.float64)
    for opx in (chain, comp):
        g0 = opx.apply_transpose(torch.from_numpy(gL).cuda()).cpu().numpy()
        np.testing.assert_allclose(g0, want, atol=1e-4 * np.abs(want).max())


@pytest.mark.parametrize("scheme,fn,levels", CASES)
def test_matrix_free_apply_and_transpose(scheme, fn, levels):
    """ALSUB_OP_MATRIX_FREE: apply is the eval kernels' result bit for bit (and so within the
    tolerance of the oracle); with ALSUB_OP_TRANSPOSE the stored transposes give the chain's
    adjoint bit for bit; no forward matrix is stored. Without ALSUB_OP_TRANSPOSE a closed
    Catmull-Clark mesh applies R^T as a gather per coarse vertex: against the oracle's R_l^T chain
    (scipy, FP64); the other schemes refuse."""
    import scipy.sparse as sp
    import torch
    from paper_1809_06047_gb300 import alsub
    mesh = fn()
    ref = oracle.subdivide(mesh, levels, scheme, keep_all=True, operator=True)
    M, T, P0 = _setup(mesh, scheme, levels)
    pi = _maps(scheme, T, ref)
    ev = T.refine_vertices(P0).cpu().numpy()
    mf = alsub.Operator(T, chain=False, matrix_free=True, transpose=True)
    chain = alsub.Operator(T, chain=True, transpose=True)
    got = [mf.apply(P0).cpu().numpy() for _ in range(3)]   # a one-off call, then a graph replay
    T.status()
    for g in got:
        assert np.array_equal(g, ev)
    err, diag = canon.position_error(pi[levels], got[0], ref[levels]["P"])
    assert err <= gpu_util.POS_TOL * diag
    gL = torch.from_numpy(np.random.default_rng(5).standard_normal((ev.shape[0], 3)).astype(np.float32)).cuda()
    assert torch.equal(mf.apply_transpose(gL), chain.apply_transpose(gL))
    with pytest.raises(alsub.AlsubError) as e:
        mf.info(0)
    assert e.value.status == 1
    only = alsub.Operator(T, chain=False, matrix_free=True)
    assert only.bytes() < mf.bytes()
    if scheme != "cc":
        with pytest.raises(alsub.AlsubError) as e:
            only.apply_transpose(gL)
        assert e.value.status == 1
        return
    Rs = [sp.csr_matrix((ref[l]["R_w"], (ref[l]["R_rows"], ref[l]["R_cols"])),
                        shape=(ref[l + 1]["V"], ref[l]["V"])) for l in range(levels)]
    gl = gL.double().cpu().numpy()[np.argsort(pi[levels])]      # into the oracle's numbering
    for R in reversed(Rs):
        gl = R.T @ gl
    got = [only.apply_transpose(gL).cpu().numpy() for _ in range(2)]
    T.status()
    assert np.array_equal(got[0], got[1])                        # deterministic: no atomics
    np.testing.assert_allclose(got[0], gl, atol=1e-5 * np.abs(gl).max())
    np.testing.assert_allclose(got[0], chain.apply_transpose(gL).cpu().numpy(), atol=1e-5 * np.abs(gl).max())


def test_matrix_free_applies_on_many_streams():
    """Applies of one matrix-free operator issued on several streams share its scratch: each one
    waits for the previous, so every result equals the eval kernels' for its own input."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_mixed(24, 20, crease_frac=0.1, seed=66)
    M, T, P0 = _setup(m, "cc", 4)
    op = alsub.Operator(T, chain=False, matrix_free=True)
    streams = [torch.cuda.Stream() for _ in range(4)]
    ins = [P0 * (1.0 + 0.25 * k) + k for k in range(8)]
    torch.cuda.synchronize()
    outs = []
    for k, x in enumerate(ins):
        s = streams[k % 4]
        with torch.cuda.stream(s):
            outs.append(op.apply(x, stream=s))
    torch.cuda.synchronize()
    for x, y in zip(ins, outs):
        assert torch.equal(y, T.refine_vertices(x))
    T.status()


def test_operator_matches_refine_vertices_and_is_deterministic():
    """Config-2 mesh at level 4: R P0 (composite) equals the fused eval within tolerance; two
    builds give identical bits."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.workload("cc_creased_torus96_L6")
    M, T, P0 = _setup(m, "cc", 4)
    ev = T.refine_vertices(P0)
    op1 = alsub.Operator(T, chain=True, compose=True)
    op2 = alsub.Operator(T, chain=False, compose=True)
    y = op1.apply(P0)
    T.status()
    diag = float(torch.linalg.norm(ev.max(0).values - ev.min(0).values))
    assert float((y - ev).abs().max()) <= gpu_util.POS_TOL * diag
    for x, z in zip(op1.csr(-1), op2.csr(-1)):
        assert np.array_equal(x, z)
    assert op1.info(-1)["rows"] == ev.shape[0]
