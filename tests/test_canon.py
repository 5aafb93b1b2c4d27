"""The canonical comparison accepts any valid edge numbering and rejects planted mistakes."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import canon

CASES = [
    ("cc", synth.torus_cc_mixed(10, 10, seed=31)),
    ("loop", synth.torus_tri(8, 8, seed=32)),
    ("sqrt3", synth.torus_tri(8, 8, seed=33, creases=False)),
]


def _compare(scheme, A, B):
    counts = [dict(V=b["V"], F=b["F"], E=b["E"]) for b in B]
    pi = canon.vertex_maps(scheme, [a["fv"] for a in A], [b["fv"] for b in B], counts)
    for l in range(len(B)):
        canon.compare_creases(pi[l], A[l]["crease_verts"], A[l]["crease_sharp"],
                              B[l]["crease_verts"], B[l]["crease_sharp"], l)
        err, diag = canon.position_error(pi[l], A[l]["P"], B[l]["P"])
        assert err <= 1e-12 * max(diag, 1.0)
    return pi


@pytest.mark.parametrize("scheme,mesh", CASES)
def test_relabelled_oracle_matches(scheme, mesh):
    ref = oracle.subdivide(mesh, 3, scheme)
    _compare(scheme, canon.relabel(scheme, ref, seed=7), ref)


@pytest.mark.parametrize("scheme,mesh", CASES)
def test_planted_topology_mistake_is_caught(scheme, mesh):
    ref = oracle.subdivide(mesh, 2, scheme)
    bad = canon.relabel(scheme, ref, seed=8)
    fv = bad[2]["fv"].copy()
    k = canon.ARITY[scheme]
    fv[5 * k], fv[5 * k + 1] = fv[5 * k + 1], fv[5 * k]     # transpose two slots of one face
    bad[2] = dict(bad[2], fv=fv)
    with pytest.raises(canon.Mismatch):
        _compare(scheme, bad, ref)


def test_planted_edge_merge_is_caught():
    ref = oracle.subdivide(CASES[0][1], 1, "cc")
    bad = [dict(d) for d in ref]
    fv = bad[1]["fv"].copy().reshape(-1, 4)
    V, F = ref[0]["V"], ref[0]["F"]
    e_other = fv[1, 1]
    fv[0, 1] = e_other                     # two different edges get one edge point
    bad[1]["fv"] = fv.reshape(-1)
    with pytest.raises(canon.Mismatch):
        _compare("cc", bad, ref)


def test_planted_crease_and_position_mistakes_are_caught():
    scheme, mesh = CASES[0]
    ref = oracle.subdivide(mesh, 2, scheme)
    bad = canon.relabel(scheme, ref, seed=9)
    cs = bad[1]["crease_sharp"].copy()
    cs[0] = np.nextafter(cs[0], np.float32(np.inf))       # one ulp off
    bad[1] = dict(bad[1], crease_sharp=cs)
    with pytest.raises(canon.Mismatch):
        _compare(scheme, bad, ref)
    bad = canon.relabel(scheme, ref, seed=10)
    P = bad[2]["P"].copy()
    P[17, 1] += 1e-6
    bad[2] = dict(bad[2], P=P)
    with pytest.raises(AssertionError):
        _compare(scheme, bad, ref)
