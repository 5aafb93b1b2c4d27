"""The feature-adaptive single-SpMV operator (Sec. 3.4 with Eq. singleSpMV: the extraction matrices
and one-level operators of a chain of selective refinement rounds composed into one matrix) against
the oracle's composition: every weight, the applied points and the transposed apply, stacked and
last round only, for Catmull-Clark with and without creases and for Loop; the full-size chain of
the benchmark's adaptive workload against the oracle's chain of points; and the chains the call
refuses."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu

W_TOL = 1e-6      # absolute, on weights in [0, 1] composed in FP32 over a few rounds


def _chain(m, scheme, rounds, rings=2):
    """Device topologies of `rounds` rounds (extract from the last level, refine one level) after a
    level-0 topology of the control mesh; every handle is returned so it outlives the build."""
    from paper_1809_06047_gb300 import alsub
    M = alsub.Mesh.from_dict(m, scheme)
    T = alsub.Topology(M, 0, build=True)
    topos, keep = [T], [M]
    for _ in range(rounds):
        sub = T.extract(T.levels, None, rings)
        T = alsub.Topology(sub, 1, build=True)
        T.status()
        topos.append(T)
        keep.append(sub)
    return topos, keep


def _oracle_faces(m, scheme, rounds, rings=2):
    """The oracle chain's face table of every round's refined level."""
    cur, fvs = dict(m, P=np.asarray(m["P"], dtype=np.float64)), []
    for _ in range(rounds):
        cur = oracle.subdivide(oracle.extract(cur, None, rings, scheme=scheme), 1, scheme)[1]
        fvs.append(np.asarray(cur["fv"]))
    return fvs


def _relabel(dev_fv, ref_fv, V):
    """Device vertex id of every oracle vertex id of one level: both sides emit the same faces in the
    same corner order and number their edges differently (so edge points and, through the
    extraction order, every vertex), so the face tables match corner by corner."""
    dev_fv, ref_fv = np.asarray(dev_fv), np.asarray(ref_fv)
    assert dev_fv.shape == ref_fv.shape
    perm = np.full(V, -1, dtype=np.int64)
    perm[ref_fv] = dev_fv
    assert np.array_equal(perm[ref_fv], dev_fv)            # one device id per oracle id
    assert (perm >= 0).all() and np.unique(perm).size == V  # a bijection
    return perm


def _dense(op):
    info = op.info(-1)
    rp, col, w = op.csr(-1)
    rows = np.repeat(np.arange(info["rows"]), np.diff(rp))
    A = np.zeros((info["rows"], info["cols"]))
    A[rows, col] = w
    assert np.all(np.diff(rp) >= 0) and rp[0] == 0 and rp[-1] == col.size
    return A


@pytest.mark.parametrize("name,scheme,mesh,rounds", [
    ("cc_evs", "cc", lambda: synth.torus_cc_mixed(18, 14, merge_frac=0.03, split_frac=0.02, crease_frac=0.0,
                                                  seed=201), 3),
    ("cc_creases", "cc", lambda: synth.torus_cc_mixed(16, 14, merge_frac=0.03, split_frac=0.02,
                                                      crease_frac=0.04, seed=202), 2),
    ("loop_evs", "loop", lambda: synth.torus_tri(16, 14, flip_frac=0.03, sharp_frac=0.0, seed=203), 3),
])
@pytest.mark.parametrize("stacked", [False, True])
def test_adaptive_operator_matches_oracle(name, scheme, mesh, rounds, stacked):
    import torch
    from paper_1809_06047_gb300 import alsub
    m = mesh()
    topos, keep = _chain(m, scheme, rounds)
    op = alsub.AdaptiveOperator(topos, stacked=stacked, transpose=True)
    ref = oracle.adaptive_operator(m, rounds, 2, scheme, stacked=stacked)
    # the rows in the oracle's vertex order: each round's level relabelled through its face table
    perms = [np.arange(m["V"])]
    for t, fv in zip(topos[1:], _oracle_faces(m, scheme, rounds)):
        perms.append(_relabel(t.faces(1), fv, t.counts[1]["V"]))
    if stacked:
        offs = np.cumsum([0] + [p.size for p in perms])
        perm = np.concatenate([o + p for o, p in zip(offs, perms)])
    else:
        perm = perms[-1]
    # every weight
    A = _dense(op)
    assert A.shape == ref.shape
    np.testing.assert_allclose(A[perm], ref.toarray(), rtol=0, atol=W_TOL)
    # the topologies may go once it is built
    for t in topos:
        t.close()
    # P = R P0 against the oracle's composition in FP64
    P0 = np.ascontiguousarray(m["P"], dtype=np.float32)
    got = op.apply(torch.from_numpy(P0).cuda()).cpu().numpy()
    want = ref @ P0.astype(np.float64)
    diag = float(np.linalg.norm(want.max(0) - want.min(0)))
    assert float(np.abs(got[perm] - want).max()) <= gpu_util.POS_TOL * diag
    # g0 = R^T gL
    g = np.random.default_rng(7).standard_normal((op.rows, 3)).astype(np.float32)
    gt = op.apply_transpose(torch.from_numpy(g).cuda()).cpu().numpy()
    gw = ref.T @ g[perm].astype(np.float64)
    scale = float(np.abs(gw).max())
    assert float(np.abs(gt - gw).max()) <= 1e-5 * scale
    torch.cuda.synchronize()
    op.close()


def test_adaptive_operator_of_the_benchmark_workload():
    """The benchmark's adaptive workload at its full size (96 x 96 mixed torus, six rounds of two
    rings): the last round's points from one SpMV against the oracle's chain of (extract, refine)
    evaluated in FP64, point by point."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_mixed(96, 96, merge_frac=0.01, split_frac=0.005, crease_frac=0.0, seed=synth.SEED_BASE + 10)
    rounds = 6
    topos, keep = _chain(m, "cc", rounds)
    op = alsub.AdaptiveOperator(topos)
    P = op.apply(torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda()).cpu().numpy()
    cur = dict(m, P=m["P"].astype(np.float64))
    for _ in range(rounds):
        cur = oracle.subdivide(oracle.extract(cur, None, 2), 1, "cc")[1]
    assert P.shape == cur["P"].shape
    gfv = topos[-1].faces(1)
    assert len(gfv) == len(cur["fv"])
    diag = float(np.linalg.norm(cur["P"].max(0) - cur["P"].min(0)))
    assert float(np.abs(P[gfv] - cur["P"][cur["fv"]]).max()) <= gpu_util.POS_TOL * diag
    # the same rows as refinement of the device chain's own levels
    Ps = torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda()
    for t in topos[1:]:
        Ps = t.refine_vertices(t.mesh.gather(Ps))
    np.testing.assert_allclose(P, Ps.cpu().numpy(), rtol=0, atol=gpu_util.POS_TOL * diag)
    op.close()


def test_adaptive_operator_refuses_broken_chains():
    """A round whose mesh was not extracted from the last level of the round before, a topology
    that is not built and flags other than TRANSPOSE and STACKED are INVALID_ARG (host checks)."""
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_mixed(12, 10, merge_frac=0.03, split_frac=0.02, crease_frac=0.0, seed=204)
    topos, keep = _chain(m, "cc", 2)
    with pytest.raises(alsub.AlsubError) as e:
        alsub.AdaptiveOperator([topos[0], topos[2]])
    assert e.value.status == 1
    with pytest.raises(alsub.AlsubError) as e:
        alsub.AdaptiveOperator([topos[1], topos[0]])
    assert e.value.status == 1
    # extracted from level 0 of a two-level topology: not its last level
    M2 = alsub.Mesh.from_dict(m, "cc")
    T2 = alsub.Topology(M2, 2, build=True)
    sub = T2.extract(0, None, 2)
    Ts = alsub.Topology(sub, 1, build=True)
    with pytest.raises(alsub.AlsubError) as e:
        alsub.AdaptiveOperator([T2, Ts])
    assert e.value.status == 1
    U = alsub.Topology(M2, 1, build=False)
    with pytest.raises(alsub.AlsubError) as e:
        alsub.AdaptiveOperator([U])
    assert e.value.status == 1
    import ctypes
    lib = alsub.lib
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(topos[0].handle.value)
    assert lib().alsub_build_adaptive_operator(arr, 1, alsub.Operator.COMPOSE, None, ctypes.byref(h)) == 1
    assert lib().alsub_build_adaptive_operator(arr, 0, 0, None, ctypes.byref(h)) == 1
    # a one-round chain of no levels is the identity
    op = alsub.AdaptiveOperator([topos[0]])
    A = _dense(op)
    np.testing.assert_array_equal(A, np.eye(m["V"]))
    op.close()


def test_adaptive_autograd_gradient_matches_oracle():
    """torch.autograd through the adaptive operator: loss = sum |P - target|^2 over the last round's
    points; the gradient equals 2 R^T (R P0 - target) with the oracle's composed R (rows relabelled
    through the face tables), and FP64 central differences of the oracle's chain of (extract,
    refine) eval steps on a few control coordinates."""
    import torch
    from paper_1809_06047_gb300.autograd import AdaptiveSubdivider
    m = synth.torus_cc_mixed(16, 14, merge_frac=0.03, split_frac=0.02, crease_frac=0.04, seed=205)
    rounds = 2
    sub = AdaptiveSubdivider(m, rounds)
    ref = oracle.adaptive_operator(m, rounds, 2, "cc")
    fv_ref = _oracle_faces(m, "cc", rounds)[-1]
    perm = _relabel(sub.faces, fv_ref, ref.shape[0])
    rng = np.random.default_rng(11)
    target = rng.standard_normal((ref.shape[0], 3))              # oracle vertex order
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"], dtype=np.float32)).cuda().requires_grad_(True)
    P = sub(P0)
    tgt = torch.from_numpy(target[np.argsort(perm)].astype(np.float32)).cuda()   # device order
    loss = ((P - tgt) ** 2).sum()
    loss.backward()
    g = P0.grad.cpu().numpy()
    P0d = m["P"].astype(np.float64)
    want = 2.0 * (ref.T @ (ref @ P0d - target))
    assert float(np.abs(g - want).max()) <= 1e-4 * float(np.abs(want).max())

    def f(Q):                                                # the oracle's chain of eval steps
        cur = dict(m, P=Q)
        for _ in range(rounds):
            cur = oracle.subdivide(oracle.extract(cur, None, 2), 1, "cc")[1]
        return float(((cur["P"] - target) ** 2).sum())
    h = 1e-6
    for (i, c) in [(0, 0), (7, 1), (m["V"] // 2, 2), (m["V"] - 1, 0)]:
        Qp, Qm = P0d.copy(), P0d.copy()
        Qp[i, c] += h
        Qm[i, c] -= h
        fd = (f(Qp) - f(Qm)) / (2 * h)
        assert abs(g[i, c] - fd) <= 1e-3 * max(1.0, abs(fd))


def test_adaptive_operator_of_one_topology_is_its_composite():
    """A chain of one topology with levels is R = R_{L-1} ... R_0: the same rows as the composite
    operator of alsub_build_operator, entry for entry; and a round after it composes with it."""
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_mixed(12, 10, merge_frac=0.03, split_frac=0.02, crease_frac=0.05, seed=206)
    M = alsub.Mesh.from_dict(m, "cc")
    T = alsub.Topology(M, 2, build=True)
    T.status()
    comp = alsub.Operator(T, chain=False, compose=True)
    ad = alsub.AdaptiveOperator([T])
    for x, y in zip(comp.csr(-1), ad.csr(-1)):
        np.testing.assert_array_equal(x, y)
    # one more round extracted from level 2: rows = R^(1) X^(1) R
    sub = T.extract(2, None, 2)
    T1 = alsub.Topology(sub, 1, build=True)
    T1.status()
    chain = alsub.AdaptiveOperator([T, T1])
    A = _dense(chain)
    R = _dense(ad)
    op1 = alsub.Operator(T1, chain=False, compose=True)
    R1 = _dense(op1)
    vmap, _ = sub.maps()
    np.testing.assert_allclose(A, R1 @ R[vmap], rtol=0, atol=W_TOL)
    for o in (comp, ad, chain, op1):
        o.close()
