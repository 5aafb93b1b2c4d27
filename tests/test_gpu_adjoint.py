"""Adjoint of vertex refinement (the transposed operator behind torch.autograd).

Workload: Catmull-Clark level 4 of the 144 x 144 creased torus (20,736 control faces, 5.3 M
refined quads). Loss L = sum |P_4 - T|^2 with the target T = refine_4(P_0 + d(P_0)),
d(p) = 0.05 (sin 2 pi p_y, sin 2 pi p_z, sin 2 pi p_x). The GPU gradient (autograd backward
through alsub_apply_operator_transpose) is checked against FP64 central differences (h = 1e-6) on
64 random control coordinates and against 2 R^T (R P_0 - T) from the oracle's FP64 operator.
Refinement is linear, so the oracle's positions at any perturbed P_0 are its operator chain applied
to that P_0 (pinned against its half-edge positions by the brute-force operator test).
"""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth

pytestmark = pytest.mark.gpu


def _chain(Rs, P):
    for R in Rs:
        P = R @ P
    return P


def _chain_t(Rs, g):
    for R in reversed(Rs):
        g = R.T @ g
    return g


def test_adjoint_config5_fd_and_oracle_transpose():
    import scipy.sparse as sp
    import torch
    from paper_1809_06047_gb300.autograd import Subdivider
    from tests import canon
    m = synth.workload("cc_creased_torus144_L4")
    L = 4
    ref = oracle.subdivide(m, L, "cc", keep_all=True, operator=True)
    Rs = [sp.csr_matrix((ref[l]["R_w"], (ref[l]["R_rows"], ref[l]["R_cols"])),
                        shape=(ref[l + 1]["V"], ref[l]["V"])) for l in range(L)]
    P0 = m["P"].astype(np.float64)
    d = 0.05 * np.stack([np.sin(2 * np.pi * P0[:, 1]), np.sin(2 * np.pi * P0[:, 2]),
                         np.sin(2 * np.pi * P0[:, 0])], axis=1)
    target = _chain(Rs, P0 + d)                      # oracle numbering
    PL = _chain(Rs, P0)
    g_ref = _chain_t(Rs, 2.0 * (PL - target))        # exact gradient, FP64

    sub = Subdivider(m, L, "cc")
    counts = [dict(V=r["V"], F=r["F"], E=r["E"]) for r in ref]
    pi = canon.vertex_maps("cc", [sub.topo.faces(l) for l in range(L + 1)],
                           [r["fv"] for r in ref], counts)[L]
    tgt_gpu = torch.from_numpy(target[pi].astype(np.float32)).cuda()   # GPU numbering
    P = torch.from_numpy(m["P"]).cuda().requires_grad_(True)
    loss = ((sub(P) - tgt_gpu) ** 2).sum()
    loss.backward()
    sub.topo.status()
    g = P.grad.double().cpu().numpy()

    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 1e-4 * scale

    rng = np.random.default_rng(2018)
    idx = rng.choice(P0.size, 64, replace=False)
    h = 1e-6

    def loss64(Pc):
        r = _chain(Rs, Pc) - target
        return float((r * r).sum())

    g_fd = np.empty(64)
    for t, k in enumerate(idx):
        Pp, Pm = P0.copy(), P0.copy()
        Pp.flat[k] += h
        Pm.flat[k] -= h
        g_fd[t] = (loss64(Pp) - loss64(Pm)) / (2 * h)
    assert np.abs(g.flat[idx] - g_fd).max() <= 1e-4 * np.abs(g_fd).max()


def test_backward_chain_small_matches_oracle():
    """A small creased mesh through three levels: autograd gradient == R^T g from the oracle."""
    import scipy.sparse as sp
    import torch
    from paper_1809_06047_gb300.autograd import Subdivider
    from tests import canon
    m = synth.torus_cc_mixed(10, 12, crease_frac=0.2, seed=71)
    L = 3
    ref = oracle.subdivide(m, L, "cc", keep_all=True, operator=True)
    Rs = [sp.csr_matrix((ref[l]["R_w"], (ref[l]["R_rows"], ref[l]["R_cols"])),
                        shape=(ref[l + 1]["V"], ref[l]["V"])) for l in range(L)]
    sub = Subdivider(m, L, "cc")
    counts = [dict(V=r["V"], F=r["F"], E=r["E"]) for r in ref]
    pi = canon.vertex_maps("cc", [sub.topo.faces(l) for l in range(L + 1)],
                           [r["fv"] for r in ref], counts)[L]
    rng = np.random.default_rng(5)
    w = rng.standard_normal((ref[L]["V"], 3))
    P = torch.from_numpy(m["P"]).cuda().requires_grad_(True)
    (sub(P) * torch.from_numpy(w.astype(np.float32)).cuda()).sum().backward()
    want = _chain_t(Rs, w[np.argsort(pi)])
    np.testing.assert_allclose(P.grad.double().cpu().numpy(), want, atol=1e-5 * np.abs(want).max())


@pytest.mark.parametrize("scheme,fn", [
    ("cc", lambda: synth.holed_cc_mixed(12, 10, holes=2, seed=73)),
    ("loop", lambda: synth.torus_tri(8, 7, seed=74)),
])
def test_backward_where_no_gather_matches_oracle(scheme, fn):
    """An open Catmull-Clark mesh and a Loop mesh have no matrix-free transpose: autograd takes
    their stored transposes, and the gradient is R^T g from the oracle's operator chain."""
    import scipy.sparse as sp
    import torch
    from paper_1809_06047_gb300.autograd import Subdivider
    from tests import canon
    m = fn()
    L = 3
    ref = oracle.subdivide(m, L, scheme, keep_all=True, operator=True)
    Rs = [sp.csr_matrix((ref[l]["R_w"], (ref[l]["R_rows"], ref[l]["R_cols"])),
                        shape=(ref[l + 1]["V"], ref[l]["V"])) for l in range(L)]
    sub = Subdivider(m, L, scheme)
    assert sub.op.bytes() > 0
    counts = [dict(V=r["V"], F=r["F"], E=r["E"]) for r in ref]
    pi = canon.vertex_maps(scheme, [sub.topo.faces(l) for l in range(L + 1)],
                           [r["fv"] for r in ref], counts)[L]
    rng = np.random.default_rng(9)
    w = rng.standard_normal((ref[L]["V"], 3))
    P = torch.from_numpy(np.ascontiguousarray(m["P"], np.float32)).cuda().requires_grad_(True)
    (sub(P) * torch.from_numpy(w.astype(np.float32)).cuda()).sum().backward()
    sub.topo.status()
    want = _chain_t(Rs, w[np.argsort(pi)])
    np.testing.assert_allclose(P.grad.double().cpu().numpy(), want, atol=1e-5 * np.abs(want).max())
