"""Pins for the CPU oracle: closed forms, printed-rule special cases, invariants, brute force.

None of these re-types the oracle's own formulas: every expected value is either a hand-derived
closed form from the paper's equations (stored under tests/golden/ with its derivation), a
structural identity (counts, Euler characteristic), an invariant of linear subdivision (affine
invariance, planarity, linear reproduction, partition of unity), or a reduction to a textbook
routine (cubic B-spline curve subdivision along an infinitely sharp crease loop).
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests.crease_cases import GRID, grid_mesh as _grid_mesh, read_cases as _read_crease_cases

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _frac(s):
    return float(Fraction(s))


def _read_golden(name):
    counts, points, stencils = None, [], {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "counts":
            counts = tuple(int(t) for t in tok[1:])
        elif tok[0] == "point":
            points.append(tuple(_frac(t) for t in tok[1:4]))
        elif tok[0] in ("vertex", "face", "edge"):
            n, base = int(tok[1]), [_frac(t) for t in tok[2:5]]
            cls = set()
            for perm in itertools.permutations(base):
                for signs in itertools.product((1, -1), repeat=3):
                    cls.add(tuple(s * x for s, x in zip(signs, perm)))
            assert len(cls) == n, (name, line, len(cls))
            points.extend(sorted(cls))
        else:
            stencils[tok[0]] = sorted(_frac(t) for t in tok[1:])
    return counts, points, stencils


def _as_sorted(P):
    P = np.round(np.asarray(P, dtype=np.float64), 12) + 0.0
    return P[np.lexsort(P.T[::-1])]


@pytest.mark.parametrize("mesh_fn,scheme,gold", [
    (synth.cube, "cc", "cube_cc_level1.txt"),
    (synth.octahedron, "loop", "octahedron_loop_level1.txt"),
    (synth.octahedron, "sqrt3", "octahedron_sqrt3_level1.txt"),
    (synth.tetrahedron, "sqrt3", "tetrahedron_sqrt3_level1.txt"),
])
def test_level1_closed_forms(mesh_fn, scheme, gold):
    counts, pts, _ = _read_golden(gold)
    L = oracle.subdivide(mesh_fn(), 1, scheme)
    assert (L[1]["V"], L[1]["F"], L[1]["E"]) == counts
    np.testing.assert_allclose(_as_sorted(L[1]["P"]), _as_sorted(pts), atol=1e-14)


def _meshes():
    return [
        ("cc", synth.cube()),
        ("cc", synth.pillow(6)),
        ("cc", synth.prism(12)),
        ("cc", synth.torus_cc_mixed(12, 12, seed=11)),
        ("cc", synth.tube_cc(8, 5)),
        ("cc", synth.sheet_cc(5, 4)),
        ("cc", synth.holed_cc_mixed(12, 12, holes=3, seed=14)),
        ("loop", synth.octahedron()),
        ("loop", synth.torus_tri(10, 10, seed=12)),
        ("sqrt3", synth.tetrahedron()),
        ("sqrt3", synth.torus_tri(10, 10, seed=13, creases=False)),
        ("sqrt3", synth.triangulate(synth.sheet_cc(5, 4, seed=15))),
        ("sqrt3", synth.triangulate(synth.holed_cc_mixed(12, 12, holes=3, seed=16))),
        ("sqrt3", synth.torus_tri(10, 10, seed=17)),                  # infinitely sharp creases
        ("sqrt3", synth.polygon(3)),
    ]


def _boundary_edge_count(level):
    """Directed edges of a face table without the reverse edge (the boundary edges)."""
    off, fv = level["off"], level["fv"]
    d = set()
    for r in range(level["F"]):
        f = fv[off[r]:off[r + 1]]
        for j in range(len(f)):
            d.add((int(f[j]), int(f[(j + 1) % len(f)])))
    return sum(1 for a, b in d if (b, a) not in d)


@pytest.mark.parametrize("scheme,mesh", _meshes())
def test_counts_and_euler(scheme, mesh):
    """Per-level counts (Sec. 3.1 step 4, Appendix A/B) and the Euler characteristic."""
    levels = 3
    out = oracle.subdivide(mesh, levels, scheme)
    chi = out[0]["V"] - out[0]["E"] + out[0]["F"]
    for l in range(levels):
        a, b = out[l], out[l + 1]
        if scheme == "cc":
            exp = (a["V"] + a["F"] + a["E"], a["nnz"], 2 * a["E"] + a["nnz"])
            assert np.all(np.diff(b["off"]) == 4)
        elif scheme == "loop":
            exp = (a["V"] + a["E"], 4 * a["F"], 2 * a["E"] + 3 * a["F"])
        else:
            # sqrt(3) with feature edges (Kobbelt 2000): the second step of each pair adds two
            # points per boundary edge, one in the slot of the triangle beside it, one more
            B = _boundary_edge_count(a) if l % 2 == 1 else 0
            exp = (a["V"] + a["F"] + B, 3 * a["F"], a["E"] + 3 * a["F"] + B)
        assert (b["V"], b["F"], b["E"]) == exp
        assert b["V"] - b["E"] + b["F"] == chi


def _edge_endpoints_from_children(lvl0, lvl1, scheme):
    """Endpoints of each level-0 edge id, read off the level-1 face table (layout of Sec. 3.2)."""
    V, F = lvl0["V"], lvl0["F"]
    off, fv = lvl0["off"], lvl0["fv"]
    ends = {}
    for r in range(F):
        s, c = off[r], off[r + 1] - off[r]
        for j in range(c):
            a, b = fv[s + j], fv[s + (j + 1) % c]
            if scheme == "cc":
                e = lvl1["fv"][4 * (s + j) + 1] - V - F
            else:   # loop: child j of triangle r holds e_j at position 1
                e = lvl1["fv"][3 * (4 * r + j) + 1] - V
            ends[int(e)] = (int(min(a, b)), int(max(a, b)), r)
    return ends


def _rows(lvl):
    rows = {}
    for r, c, w in zip(lvl["R_rows"], lvl["R_cols"], lvl["R_w"]):
        rows.setdefault(int(r), {})[int(c)] = float(w)
    return rows


def test_regular_stencils_cc():
    """Regular quad grid: B-spline masks of the gold file (Sec. 3.1, Eqs. 1, 2, pos_update)."""
    _, _, st = _read_golden("regular_stencils.txt")
    N = M = 8
    m = synth.torus_cc_plain(N, M, jitter=0.0)
    out = oracle.subdivide(m, 1, "cc", operator=True)
    rows = _rows(out[0])
    V, F = m["V"], m["F"]
    for v in range(V):
        i, j = divmod(v, M)
        exp = {((i + di) % N) * M + (j + dj) % M: None for di in (-1, 0, 1) for dj in (-1, 0, 1)}
        assert set(rows[v]) == set(exp)
        assert sorted(rows[v].values()) == pytest.approx(st["cc_vertex"], abs=1e-15)
        assert rows[v][v] == pytest.approx(36 / 64, abs=1e-15)
        assert rows[v][((i + 1) % N) * M + j] == pytest.approx(6 / 64, abs=1e-15)
        assert rows[v][((i + 1) % N) * M + (j + 1) % M] == pytest.approx(1 / 64, abs=1e-15)
    for r in range(F):
        assert sorted(rows[V + r].values()) == pytest.approx(st["cc_face"], abs=1e-15)
        assert set(rows[V + r]) == set(m["fv"][4 * r:4 * r + 4].tolist())
    ends = _edge_endpoints_from_children(out[0], out[1], "cc")
    for e, (a, b, _) in ends.items():
        row = rows[V + F + e]
        assert sorted(row.values()) == pytest.approx(st["cc_edge"], abs=1e-15)
        assert row[a] == pytest.approx(3 / 8) and row[b] == pytest.approx(3 / 8)


def test_regular_stencils_loop_sqrt3():
    """Regular triangulation (valence 6): beta_6 = 1/16 and alpha_6 = 1/3 (Appendices A, B)."""
    _, _, st = _read_golden("regular_stencils.txt")
    m = synth.torus_tri(8, 8, flip_frac=0.0, creases=False, jitter=0.0)
    V, F = m["V"], m["F"]
    out = oracle.subdivide(m, 1, "loop", operator=True)
    rows = _rows(out[0])
    for v in range(V):
        assert sorted(rows[v].values()) == pytest.approx(st["loop_vertex"], abs=1e-15)
        assert rows[v][v] == pytest.approx(10 / 16, abs=1e-15)
    ends = _edge_endpoints_from_children(out[0], out[1], "loop")
    for e, (a, b, r) in ends.items():
        row = rows[V + e]
        assert sorted(row.values()) == pytest.approx(st["loop_edge"], abs=1e-15)
        assert row[a] == pytest.approx(3 / 8) and row[b] == pytest.approx(3 / 8)
        third = set(m["fv"][3 * r:3 * r + 3].tolist()) - {a, b}
        assert all(row[t] == pytest.approx(1 / 8) for t in third)
    out = oracle.subdivide(m, 1, "sqrt3", operator=True)
    rows = _rows(out[0])
    for v in range(V):
        assert sorted(rows[v].values()) == pytest.approx(st["sqrt3_vertex"], abs=1e-15)
    for r in range(F):
        assert sorted(rows[V + r].values()) == pytest.approx(st["sqrt3_face"], abs=1e-15)


@pytest.mark.parametrize("scheme,mesh", _meshes())
def test_partition_of_unity_and_positivity(scheme, mesh):
    """Every refined vertex is an affine (convex) combination: rows sum to 1, weights >= 0."""
    out = oracle.subdivide(mesh, 2, scheme, operator=True)
    for l in range(2):
        s = np.zeros(out[l + 1]["V"])
        np.add.at(s, out[l]["R_rows"], out[l]["R_w"])
        np.testing.assert_allclose(s, 1.0, atol=1e-13)
        assert out[l]["R_w"].min() >= 0.0


@pytest.mark.parametrize("scheme,mesh", _meshes())
def test_affine_invariance(scheme, mesh):
    rng = np.random.default_rng(5)
    A, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    A = A * 1.7
    b = np.array([0.3, -2.0, 5.0])
    P = mesh["P"].astype(np.float64)
    ref = oracle.subdivide(mesh, 2, scheme, P0=P)
    mov = oracle.subdivide(mesh, 2, scheme, P0=P @ A.T + b)
    np.testing.assert_allclose(mov[2]["P"], ref[2]["P"] @ A.T + b, atol=1e-12)


@pytest.mark.parametrize("scheme,mesh", _meshes())
def test_planarity_exact(scheme, mesh):
    P = mesh["P"].astype(np.float64).copy()
    P[:, 2] = 0.0
    out = oracle.subdivide(mesh, 2, scheme, P0=P)
    assert np.all(out[2]["P"][:, 2] == 0.0)


@pytest.mark.parametrize("scheme", ["cc", "loop", "sqrt3"])
def test_linear_reproduction_away_from_seam(scheme):
    """On a regular periodic grid, positions linear in the grid indices are reproduced
    wherever the stencil does not cross the seam."""
    N = M = 12
    if scheme == "cc":
        m = synth.torus_cc_plain(N, M, jitter=0.0)
    else:
        m = synth.torus_tri(N, M, flip_frac=0.0, creases=False, jitter=0.0)
    ij = np.array([divmod(v, M) for v in range(N * M)], dtype=np.float64)
    P = np.stack([ij[:, 0], ij[:, 1], 0.5 * ij[:, 0] - 0.25 * ij[:, 1]], axis=1)
    out = oracle.subdivide(m, 1, scheme, P0=P)
    inner = (ij[:, 0] >= 2) & (ij[:, 0] <= N - 3) & (ij[:, 1] >= 2) & (ij[:, 1] <= M - 3)
    np.testing.assert_allclose(out[1]["P"][:N * M][inner], P[inner], atol=1e-12)


def _loop_creases(N, M, sigma):
    """Tag the ring j = 0 of a quad torus: edges (i,0)-(i+1,0)."""
    cv = np.array([[i * M, ((i + 1) % N) * M] for i in range(N)], dtype=np.int32)
    return cv, np.full(N, sigma, dtype=np.float32)


def _bspline_curve(poly):
    """Closed uniform cubic B-spline curve subdivision: (1, 6, 1)/8 at vertices, midpoints."""
    n = len(poly)
    out = np.zeros((2 * n, 3))
    for i in range(n):
        out[2 * i] = (poly[i - 1] + 6 * poly[i] + poly[(i + 1) % n]) / 8.0
        out[2 * i + 1] = 0.5 * (poly[i] + poly[(i + 1) % n])
    return out


def _ordered_loop(level, start):
    adj = {}
    for a, b in level["crease_verts"]:
        adj.setdefault(int(a), []).append(int(b))
        adj.setdefault(int(b), []).append(int(a))
    seq, prev, cur = [start], None, start
    while True:
        nxt = [x for x in adj[cur] if x != prev]
        nxt = nxt[0] if prev is not None else min(adj[cur])
        if nxt == start:
            break
        seq.append(nxt)
        prev, cur = cur, nxt
    return seq


@pytest.mark.parametrize("scheme", ["cc", "loop"])
def test_sharp_crease_is_bspline_curve(scheme):
    """An infinitely sharp crease loop refines as a cubic B-spline curve, independent of the
    surface around it (Sec. 3.3 with the DeRose crease rules)."""
    N = M = 10
    if scheme == "cc":
        m = synth.torus_cc_plain(N, M, jitter=0.05, seed=99)
    else:
        m = synth.torus_tri(N, M, flip_frac=0.0, creases=False, jitter=0.05, seed=99)
    m["crease_verts"], m["crease_sharp"] = _loop_creases(N, M, np.inf)
    out = oracle.subdivide(m, 3, scheme)
    poly = m["P"][[i * M for i in range(N)]].astype(np.float64)
    for l in range(1, 4):
        poly = _bspline_curve(poly)
        seq = _ordered_loop(out[l], 0)
        got = out[l]["P"][seq]
        if not np.allclose(got[1], poly[1], atol=1e-12):
            got = got[[0] + list(range(len(seq) - 1, 0, -1))]
        assert len(seq) == N * 2 ** l
        np.testing.assert_allclose(got, poly, atol=1e-12)
        assert np.all(np.isinf(out[l]["crease_sharp"]))


def test_uniform_sharpness_decays_by_one():
    """A loop of equal sharpness sigma inherits sigma - 1 exactly (Chaikin rule, Sec. 3.3)."""
    N = M = 8
    m = synth.torus_cc_plain(N, M, jitter=0.0)
    m["crease_verts"], m["crease_sharp"] = _loop_creases(N, M, 3.0)
    out = oracle.subdivide(m, 4, "cc")
    for l, s in ((1, 2.0), (2, 1.0)):
        assert out[l]["K"] == N * 2 ** l
        assert np.all(out[l]["crease_sharp"] == np.float32(s))
    assert out[3]["K"] == 0 and out[4]["K"] == 0


def test_fractional_sharpness_is_affine_at_level1():
    """For sigma in [0, 1] the level-1 result blends the smooth and sharp results linearly."""
    N = M = 8
    base = synth.torus_cc_plain(N, M, jitter=0.03, seed=4)
    res = {}
    for s in (0.0, 0.3, 1.0):
        m = dict(base)
        m["crease_verts"], m["crease_sharp"] = _loop_creases(N, M, s)
        res[s] = oracle.subdivide(m, 1, "cc")[1]["P"]
    np.testing.assert_allclose(res[0.3], 0.7 * res[0.0] + 0.3 * res[1.0], atol=1e-14)
    m = dict(base)
    m["crease_verts"], m["crease_sharp"] = _loop_creases(N, M, np.inf)
    np.testing.assert_allclose(res[1.0], oracle.subdivide(m, 1, "cc")[1]["P"], atol=1e-15)


def test_corners_fixed():
    """k >= 3 infinitely sharp creases at a vertex keep it in place at every level."""
    m = synth.cube()
    e = set()
    for r in range(6):
        f = m["fv"][4 * r:4 * r + 4]
        for j in range(4):
            a, b = int(f[j]), int(f[(j + 1) % 4])
            e.add((min(a, b), max(a, b)))
    m["crease_verts"] = np.array(sorted(e), dtype=np.int32)
    m["crease_sharp"] = np.full(len(e), np.inf, dtype=np.float32)
    out = oracle.subdivide(m, 3, "cc")
    for l in range(1, 4):
        np.testing.assert_array_equal(out[l]["P"][:8], m["P"].astype(np.float64))


@pytest.mark.parametrize("scheme,mesh", [
    ("cc", synth.torus_cc_mixed(6, 6, seed=21)),
    ("cc", synth.pillow(5)),
    ("cc", synth.sheet_cc(3, 3, seed=24)),
    ("loop", synth.torus_tri(5, 5, seed=22)),
    ("loop", synth.triangulate(synth.sheet_cc(3, 3, seed=25))),
    ("sqrt3", synth.torus_tri(5, 5, seed=23, creases=False)),
    ("sqrt3", synth.triangulate(synth.sheet_cc(3, 3, seed=26))),
    ("sqrt3", synth.torus_tri(5, 5, seed=27, sharp_frac=0.1)),
])
def test_brute_force_operator(scheme, mesh):
    """Dense R_l from unit impulses equals the oracle's sparse operator, and the composed
    operator reproduces two levels of refinement."""
    import scipy.sparse as sp
    out = oracle.subdivide(mesh, 2, scheme, operator=True)
    V0, V1 = out[0]["V"], out[1]["V"]
    dense = np.zeros((V1, V0))
    for j in range(V0):
        P = np.zeros((V0, 3))
        P[j, 0] = 1.0
        dense[:, j] = oracle.subdivide(mesh, 1, scheme, P0=P)[1]["P"][:, 0]
    R0 = sp.csr_matrix((out[0]["R_w"], (out[0]["R_rows"], out[0]["R_cols"])), shape=(V1, V0))
    np.testing.assert_allclose(R0.toarray(), dense, atol=1e-14)
    R1 = sp.csr_matrix((out[1]["R_w"], (out[1]["R_rows"], out[1]["R_cols"])),
                       shape=(out[2]["V"], V1))
    P0 = mesh["P"].astype(np.float64)
    np.testing.assert_allclose((R1 @ R0) @ P0, out[2]["P"], atol=1e-13)


def test_rejects_invalid_meshes():
    m = synth.cube()
    o = synth.octahedron()
    open_tri = dict(o, F=7, off=o["off"][:8], fv=o["fv"][:21])
    oracle.subdivide(open_tri, 2, "sqrt3")          # sqrt(3) takes Kobbelt's boundary treatment
    oracle.subdivide(open_tri, 1, "loop")           # Loop takes the boundary rules of Eq. CC_boundary
    # an infinitely sharp sqrt(3) crease touching a boundary vertex
    t = synth.triangulate(dict(m, F=5, off=m["off"][:6], fv=m["fv"][:20]))
    f5 = m["fv"][20:24]
    with pytest.raises(oracle.OracleError) as ei:
        oracle.subdivide(dict(t, crease_verts=np.array([[f5[0], f5[1]]], np.int32),
                              crease_sharp=np.array([np.inf], np.float32)), 1, "sqrt3")
    assert ei.value.code == 3
    # two squares sharing only vertex 0: two fans at one vertex
    bow = dict(V=7, F=2, off=np.array([0, 4, 8], np.int32),
               fv=np.array([0, 1, 2, 3, 0, 4, 5, 6], np.int32), P=np.zeros((7, 3), np.float32),
               crease_verts=np.zeros((0, 2), np.int32), crease_sharp=np.zeros(0, np.float32))
    with pytest.raises(oracle.OracleError) as ei:
        oracle.subdivide(bow, 1, "cc")
    assert ei.value.code == 2
    # a crease touching a boundary vertex (open box: vertices of the missing face)
    box = dict(m, F=5, off=m["off"][:6], fv=m["fv"][:20])
    f5 = m["fv"][20:24]
    cre = dict(box, crease_verts=np.array([[f5[0], f5[1]]], np.int32), crease_sharp=np.array([2.0], np.float32))
    with pytest.raises(oracle.OracleError) as ei:
        oracle.subdivide(cre, 1, "cc")
    assert ei.value.code == 3
    dup = dict(m, F=7, off=np.append(m["off"], 28).astype(np.int32),
               fv=np.concatenate([m["fv"], m["fv"][:4]]))
    with pytest.raises(oracle.OracleError) as ei:
        oracle.subdivide(dup, 1, "cc")
    assert ei.value.code == 2
    bad = dict(m, crease_verts=np.array([[0, 7]], np.int32), crease_sharp=np.array([1.0], np.float32))
    with pytest.raises(oracle.OracleError) as ei:
        oracle.subdivide(bad, 1, "cc")
    assert ei.value.code == 5


def test_loop_beta_sqrt3_alpha_values():
    """beta_n and alpha_n special values quoted in the text (Appendices A, B)."""
    def beta(n):
        return (5 / 8 - (3 / 8 + 0.25 * math.cos(2 * math.pi / n)) ** 2) / n
    m = synth.torus_tri(6, 6, flip_frac=0.0, creases=False, jitter=0.0)
    out = oracle.subdivide(m, 1, "loop", operator=True)
    rows = _rows(out[0])
    assert max(rows[0].values()) == pytest.approx(1 - 6 * beta(6), abs=1e-15)
    assert beta(6) == pytest.approx(1 / 16, abs=1e-15)


# ---------------------------------------------------------------- boundaries (Catmull-Clark)

def _boundary_loops(level):
    """Directed boundary edges a -> b (no face holds b -> a), chained into closed loops."""
    off, fv = level["off"], level["fv"]
    directed = set()
    for r in range(level["F"]):
        f = fv[off[r]:off[r + 1]]
        for j in range(len(f)):
            directed.add((int(f[j]), int(f[(j + 1) % len(f)])))
    nxt = {a: b for a, b in directed if (b, a) not in directed}
    loops, seen = [], set()
    for a0 in sorted(nxt):
        if a0 in seen:
            continue
        loop, a = [], a0
        while a not in seen:
            seen.add(a)
            loop.append(a)
            a = nxt[a]
        loops.append(loop)
    return loops


def _cox_de_boor(t, i, k):
    """Uniform B-spline basis N_{i,k}(t) on the integer knots, order k (degree k - 1)."""
    if k == 1:
        return ((t >= i) & (t < i + 1)).astype(np.float64)
    return ((t - i) / (k - 1)) * _cox_de_boor(t, i, k - 1) + ((i + k - t) / (k - 1)) * _cox_de_boor(t, i + 1, k - 1)


def _cubic_two_scale_mask():
    """The coefficients c_k of N(t) = sum_k c_k N(2t - k) for the uniform cubic B-spline N,
    found by least squares on samples of the Cox-de Boor basis (not typed in)."""
    t = np.linspace(0.0, 4.0, 801)[:-1]
    A = np.stack([_cox_de_boor(2 * t - k, 0, 4) for k in range(5)], axis=1)
    c, *_ = np.linalg.lstsq(A, _cox_de_boor(t, 0, 4), rcond=None)
    return c


def _refine_closed_polygon(P, c):
    """Control polygon of the same closed cubic B-spline on the halved knot spacing:
    Q_m = sum_j c_{m - 2j} P_j (indices cyclic)."""
    n = len(P)
    Q = np.zeros((2 * n, 3))
    for m in range(2 * n):
        for j in range(n):
            k = (m - 2 * j) % (2 * n)
            if k < len(c):
                Q[m] += c[k] * P[j]
    return Q


@pytest.mark.parametrize("scheme,mesh", [
    ("cc", synth.tube_cc(10, 6, jitter=0.2, seed=31)), ("cc", synth.sheet_cc(6, 5, seed=32)),
    ("cc", synth.holed_cc_mixed(16, 14, holes=3, seed=33)),
    ("loop", synth.triangulate(synth.tube_cc(10, 6, jitter=0.2, seed=31))),
    ("loop", synth.triangulate(synth.sheet_cc(6, 5, seed=32))),
    ("loop", synth.triangulate(synth.holed_cc_mixed(16, 14, holes=3, seed=33)))],
    ids=["tube", "sheet", "holes", "loop_tube", "loop_sheet", "loop_holes"])
def test_boundary_is_cubic_bspline_curve(scheme, mesh):
    """Every boundary loop of the refined mesh is the control polygon of the cubic B-spline curve
    of the level-0 boundary loop, refined l times (Eq. CC_boundary with midpoint edge points;
    the mask comes from the Cox-de Boor basis), whatever the surface inside it."""
    c = _cubic_two_scale_mask()
    np.testing.assert_allclose(c * 8.0, [1, 4, 6, 4, 1], atol=1e-9)   # sanity of the derivation
    levels = 3
    out = oracle.subdivide(mesh, levels, scheme)
    loops0 = _boundary_loops(out[0])
    assert len(loops0) >= 1
    expected = []
    for loop in loops0:
        poly = out[0]["P"][loop].astype(np.float64)
        expected.append(poly)
    for l in range(1, levels + 1):
        expected = [_refine_closed_polygon(poly, c) for poly in expected]
        loops = _boundary_loops(out[l])
        assert sorted(len(x) for x in loops) == sorted(len(x) for x in expected)
        got = np.concatenate([out[l]["P"][x] for x in loops])
        np.testing.assert_allclose(_as_sorted(got), _as_sorted(np.concatenate(expected)), atol=1e-9)


@pytest.mark.parametrize("scheme", ["cc", "loop"])
def test_boundary_tube_height_is_linear(scheme):
    """Heights linear in the row index are reproduced exactly by every rule at every level
    (face, edge and vertex points are affine combinations symmetric across the rows, and the
    boundary rules act along rows; for Loop the tube is triangulated along one diagonal
    direction, whose edge and vertex stencils are symmetric across the rows too), so the refined
    tube has n 2^l vertices on each of the (M - 1) 2^l + 1 dyadic heights -- a boundary vertex
    taking the smooth rule would leave its row."""
    N, M, levels, h = 9, 6, 3, 0.25
    tube = synth.tube_cc(N, M, jitter=0.3, z_step=h, seed=34)
    out = oracle.subdivide(tube if scheme == "cc" else synth.triangulate(tube), levels, scheme)
    for l in range(1, levels + 1):
        z = out[l]["P"][:, 2] / (h / 2 ** l)
        k = np.round(z)
        np.testing.assert_array_equal(z, k)
        counts = np.bincount(k.astype(np.int64))
        assert len(counts) == (M - 1) * 2 ** l + 1
        assert np.all(counts == N * 2 ** l)


@pytest.mark.parametrize("scheme", ["cc", "loop"])
def test_boundary_leaves_far_interior_unchanged(scheme):
    """Cutting a ring of faces out of a closed torus changes nothing at the level-l vertices of
    faces at least three rings away from the cut: the boundary rules only reach about two
    level-0 rings inwards over any number of levels (the stencils halve in size every level).
    For Loop the torus is triangulated (two triangles per quad, in quad order)."""
    N, M, levels = 12, 8, 3
    closed = synth.torus_cc_plain(N, M, jitter=0.05, seed=35)
    F = closed["F"] - M                              # faces i = N - 1 are the last M
    cut = dict(closed, F=F, off=closed["off"][:F + 1], fv=closed["fv"][:4 * F])
    if scheme == "loop":
        closed, cut = synth.triangulate(closed), synth.triangulate(cut)
    a = oracle.subdivide(closed, levels, scheme)[levels]
    b = oracle.subdivide(cut, levels, scheme)[levels]
    k = 4 if scheme == "cc" else 3                  # corners of a refined face
    t = 1 if scheme == "cc" else 2                  # level-0 faces of one quad
    q = t * 4 ** levels                             # refined faces of one quad
    for i in range(3, N - 4):                       # face columns 3 .. N-5 touch vertex columns <= N-4
        for j in range(M):
            r = i * M + j
            ca = a["fv"][k * q * r:k * q * (r + 1)]
            cb = b["fv"][k * q * r:k * q * (r + 1)]
            np.testing.assert_array_equal(a["P"][ca], b["P"][cb])
    # and the cut does change the faces next to it
    assert not np.array_equal(a["P"][a["fv"][:k * q]], b["P"][b["fv"][:k * q]])


@pytest.mark.parametrize("scheme,mesh", [
    ("cc", synth.torus_cc_mixed(20, 18, crease_frac=0.1, seed=36)),
    ("loop", synth.torus_tri(16, 14, seed=37)),
    ("sqrt3", synth.torus_tri(14, 12, seed=38, creases=False)),
])
def test_patch_mode_matches_whole_mesh(scheme, mesh):
    """Patch mode (used for sampled checks of meshes too large for the oracle): the children of
    faces two rings inside a patch equal the whole mesh's children exactly, and points reaching
    beyond the cut are NaN."""
    from tests import patch
    whole = oracle.subdivide(mesh, 1, scheme)
    lvl0 = dict(whole[0], P=mesh["P"].astype(np.float64))
    faces = patch.sample_faces(mesh["F"], 12, seed=1)
    pm, local = patch.extract(lvl0, faces)
    assert pm["F"] < mesh["F"]
    part = oracle.subdivide(pm, 1, scheme, patch=True)
    for r, q in zip(faces, local):
        a = whole[1]["fv"][patch.child_corners(scheme, whole[0]["off"], int(r))]
        b = part[1]["fv"][patch.child_corners(scheme, pm["off"], int(q))]
        assert np.all(b >= 0)
        np.testing.assert_array_equal(whole[1]["P"][a], part[1]["P"][b])
    assert np.isnan(part[1]["P"]).any()          # the cut is there and marked


# ---------------------------------------------------------------- selective subdivision (Sec. 3.4)

def test_extraction_rings_closed_forms():
    """Around one vertex of a regular quad grid, r propagation rings keep the (2r)^2 faces and
    (2r+1)^2 vertices of the square block around it, a disk (Euler characteristic 1)."""
    m = synth.torus_cc_plain(12, 12, jitter=0.0)
    sel = np.zeros(m["V"], bool)
    sel[5 * 12 + 5] = True
    for r in (1, 2, 3):
        e = oracle.extract(m, sel, r)
        assert (e["F"], e["V"]) == ((2 * r) ** 2, (2 * r + 1) ** 2)
        sub = oracle.subdivide(e, 0, "cc")[0]
        assert sub["V"] - sub["E"] + sub["F"] == 1


def test_loop_extraction_rings_closed_forms():
    """Around one vertex of a regular triangle lattice (every valence 6), r propagation rings keep
    the hexagon of radius r: 6 r^2 triangles and 3 r (r + 1) + 1 vertices, a disk."""
    m = synth.torus_tri(16, 16, flip_frac=0.0, sharp_frac=0.0, jitter=0.0)
    assert set(np.bincount(m["fv"], minlength=m["V"]).tolist()) == {6}
    sel = np.zeros(m["V"], bool)
    sel[5 * 16 + 5] = True
    for r in (1, 2, 3):
        e = oracle.extract(m, sel, r, scheme="loop")
        assert (e["F"], e["V"]) == (6 * r * r, 3 * r * (r + 1) + 1)
        sub = oracle.subdivide(e, 0, "loop")[0]
        assert sub["V"] - sub["E"] + sub["F"] == 1


def test_extraction_interior_is_exact():
    """One level of the extracted region's refinement equals the whole mesh's refinement on the
    faces two rings inside the cut (the region's own cut is refined by the boundary rules)."""
    m = synth.torus_cc_mixed(16, 14, merge_frac=0.02, split_frac=0.01, crease_frac=0.0, seed=39)
    whole = oracle.subdivide(m, 1, "cc")
    sel = np.zeros(m["V"], bool)
    sel[[40, 100, 150]] = True
    e = oracle.extract(m, sel, 3)
    part = oracle.subdivide(e, 1, "cc")
    inner = oracle.extract(m, sel, 1)["fmap"]          # faces touching the selected vertices
    local = np.searchsorted(e["fmap"], inner)
    assert np.array_equal(e["fmap"][local], inner)
    for r, q in zip(inner, local):
        a = whole[1]["fv"][4 * whole[0]["off"][r]:4 * whole[0]["off"][r + 1]]
        b = part[1]["fv"][4 * e["off"][q]:4 * e["off"][q + 1]]
        np.testing.assert_array_equal(whole[1]["P"][a], part[1]["P"][b])


def test_adaptive_refinement_tracks_extraordinary_vertices_exactly():
    """Feature-adaptive refinement (extract two rings around the extraordinary vertices, refine one
    level, repeat) puts every extraordinary vertex exactly where uniform refinement puts it."""
    m = synth.torus_cc_mixed(14, 12, merge_frac=0.03, split_frac=0.02, crease_frac=0.0, seed=40)
    levels = 3
    uni = oracle.subdivide(m, levels, "cc", keep_all=False)[levels]
    valence = np.bincount(m["fv"], minlength=m["V"])
    evs = np.flatnonzero(valence != 4)
    assert evs.size > 0
    cur, ids = dict(m, P=m["P"].astype(np.float64)), evs.copy()
    for _ in range(levels):
        e = oracle.extract(cur, None, 2)
        pos = np.searchsorted(e["vmap"], ids)
        assert np.array_equal(e["vmap"][pos], ids)    # every extraordinary vertex is kept
        nxt = oracle.subdivide(e, 1, "cc")[1]
        cur, ids = nxt, pos                          # old vertices keep their ids when refined
    np.testing.assert_array_equal(cur["P"][ids], uni["P"][evs])


def test_loop_extraction_interior_is_exact():
    """Loop: one level of an extracted region (its cut refined by the Loop boundary rules) equals
    the whole mesh's refinement on the triangles around the selected vertices (their children read
    one ring, well inside the three extracted rings)."""
    m = synth.torus_tri(24, 20, flip_frac=0.02, sharp_frac=0.0, seed=41)
    whole = oracle.subdivide(m, 1, "loop")
    sel = np.zeros(m["V"], bool)
    sel[[40, 200, 333]] = True
    e = oracle.extract(m, sel, 3, scheme="loop")
    assert e["F"] < m["F"]
    part = oracle.subdivide(e, 1, "loop")
    inner = oracle.extract(m, sel, 1, scheme="loop")["fmap"]
    local = np.searchsorted(e["fmap"], inner)
    assert np.array_equal(e["fmap"][local], inner)
    for r, q in zip(inner, local):
        a = whole[1]["fv"][12 * r:12 * (r + 1)]
        b = part[1]["fv"][12 * q:12 * (q + 1)]
        np.testing.assert_array_equal(whole[1]["P"][a], part[1]["P"][b])


def test_loop_adaptive_refinement_tracks_extraordinary_vertices_exactly():
    """Loop feature-adaptive refinement (two rings around the valence != 6 vertices, one level,
    repeat) puts every extraordinary vertex exactly where uniform refinement puts it."""
    m = synth.torus_tri(20, 16, flip_frac=0.02, sharp_frac=0.0, seed=42)
    levels = 3
    uni = oracle.subdivide(m, levels, "loop", keep_all=False)[levels]
    valence = np.bincount(m["fv"], minlength=m["V"])
    evs = np.flatnonzero(valence != 6)
    assert evs.size > 0
    cur, ids = dict(m, P=m["P"].astype(np.float64)), evs.copy()
    for _ in range(levels):
        e = oracle.extract(cur, None, 2, scheme="loop")
        pos = np.searchsorted(e["vmap"], ids)
        assert np.array_equal(e["vmap"][pos], ids)
        assert e["F"] < cur["F"]
        cur, ids = oracle.subdivide(e, 1, "loop")[1], pos
    np.testing.assert_array_equal(cur["P"][ids], uni["P"][evs])


@pytest.mark.parametrize("scheme,mesh", [
    ("cc", synth.torus_cc_mixed(10, 8, merge_frac=0.03, split_frac=0.02, crease_frac=0.0, seed=44)),
    ("cc", synth.torus_cc_mixed(12, 10, merge_frac=0.03, split_frac=0.02, crease_frac=0.06, seed=45)),
    ("loop", synth.torus_tri(10, 8, flip_frac=0.03, sharp_frac=0.0, seed=46)),
])
def test_adaptive_operator_columns_are_the_chain_of_unit_vectors(scheme, mesh):
    """Brute force: column j of the stacked adaptive operator is what the chain of (extract two
    rings, refine one level) makes of the unit vector e_j through the eval rules (the positions of
    the refined levels, not the operator rows), the control mesh's block first; and every row sums
    to 1 (each rule is affine, an extraction selects)."""
    rounds = 2
    A = oracle.adaptive_operator(mesh, rounds, 2, scheme, stacked=True).toarray()
    V0 = int(mesh["V"])
    cols = np.zeros((A.shape[0], V0))
    for j0 in range(0, V0, 3):                 # three unit vectors at once, one per coordinate
        P = np.zeros((V0, 3))
        js = [j for j in range(j0, min(j0 + 3, V0))]
        for c, j in enumerate(js):
            P[j, c] = 1.0
        cur, out = dict(mesh, P=P), [P]
        for _ in range(rounds):
            e = oracle.extract(cur, None, 2, scheme=scheme)
            cur = oracle.subdivide(e, 1, scheme)[1]
            out.append(cur["P"])
        S = np.vstack(out)
        for c, j in enumerate(js):
            cols[:, j] = S[:, c]
    assert A.shape == cols.shape
    np.testing.assert_allclose(A, cols, rtol=0, atol=1e-12)
    np.testing.assert_allclose(A.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    last = oracle.adaptive_operator(mesh, rounds, 2, scheme).toarray()
    np.testing.assert_array_equal(last, A[A.shape[0] - last.shape[0]:])


# ---------------------------------------------------------------- hierarchical edits (Sec. 3.5)

@pytest.mark.parametrize("scheme,mesh", [
    ("cc", synth.torus_cc_mixed(10, 9, crease_frac=0.1, seed=41)),
    ("cc", synth.sheet_cc(5, 4, seed=42)),
    ("loop", synth.torus_tri(8, 7, seed=43)),
])
def test_edits_are_refined_by_the_remaining_operators(scheme, mesh):
    """Refinement is linear in the positions, so an edit added on level l reaches level L as
    R_{L-1} ... R_l applied to it (the operator rows, pinned separately by brute force), and no
    edit gives plain refinement bit for bit."""
    import scipy.sparse as sp
    L = 3
    plain = oracle.subdivide(mesh, L, scheme, operator=True)
    none = oracle.subdivide_edits(mesh, L, scheme, {})
    np.testing.assert_array_equal(none[L]["P"], plain[L]["P"])
    rng = np.random.default_rng(8)
    edits = {}
    for l in (1, 2):
        vid = rng.choice(plain[l]["V"], 5, replace=False)
        edits[l] = (vid, rng.standard_normal((5, 3)))
    got = oracle.subdivide_edits(mesh, L, scheme, edits)
    R = [sp.csr_matrix((plain[l]["R_w"], (plain[l]["R_rows"], plain[l]["R_cols"])),
                       shape=(plain[l + 1]["V"], plain[l]["V"])) for l in range(L)]
    want = plain[L]["P"].copy()
    for l, (vid, off) in edits.items():
        d = np.zeros((plain[l]["V"], 3))
        d[vid] = off
        for k in range(l, L):
            d = R[k] @ d
        want += d
    np.testing.assert_allclose(got[L]["P"], want, atol=1e-12)


# ---------------------------------------------------------------- regular patches (Sec. 3.4)

def test_regular_patch_is_the_limit_of_subdivision():
    """On regular faces Catmull-Clark converges to the bicubic B-spline patch: the positions of a
    face's face point and corner vertex after l levels approach the patch at (1/2, 1/2) and (0, 0),
    the error shrinking by 4 per level (the patch from the Cox-de Boor basis, the subdivision from
    the classical rules)."""
    m = synth.torus_cc_plain(8, 8, jitter=0.05, seed=3)
    lvl = dict(m, P=m["P"].astype(np.float64))
    flags, g = oracle.regular_patches(lvl, 5)
    assert flags.all()
    V = m["V"]
    corner_face = {int(m["fv"][4 * r]): r for r in range(m["F"])}
    prev = None
    for L in (2, 3, 4, 5):
        P = oracle.subdivide(m, L, "cc", keep_all=False)[L]["P"]
        ef = max(np.abs(P[V + f] - g[f][2, 2]).max() for f in range(m["F"]))
        ev = max(np.abs(P[v] - g[r][0, 0]).max() for v, r in corner_face.items())
        if prev is not None:
            assert 3.5 < prev[0] / ef < 4.5 and 3.5 < prev[1] / ev < 4.5
        prev = (ef, ev)
    assert prev[0] < 2e-4


def test_regular_patch_reproduces_linear_functions_and_detects_irregularity():
    """A control net linear in the grid indices gives the bilinear image of the parameter square;
    faces next to an extraordinary vertex or a crease are not regular."""
    N = M = 10
    m = synth.torus_cc_plain(N, M, jitter=0.0)
    ij = np.array([divmod(v, M) for v in range(N * M)], dtype=np.float64)
    P = np.stack([ij[:, 0], ij[:, 1], 0.5 * ij[:, 0] - 0.25 * ij[:, 1]], axis=1)
    flags, g = oracle.regular_patches(dict(m, P=P), 3)
    u = np.array([0.0, 0.5, 1.0 - 1e-12])
    for r in range(m["F"]):
        i0, j0 = divmod(int(m["fv"][4 * r]), M)
        if not (1 <= i0 <= N - 3 and 1 <= j0 <= M - 3):
            continue                                   # the control net crosses the seam
        want = np.stack(np.meshgrid(i0 + u, j0 + u), axis=-1)      # [b, a] -> (x = i0 + u_a, y = j0 + u_b)
        np.testing.assert_allclose(g[r][..., 0], want[..., 0], atol=1e-9)
        np.testing.assert_allclose(g[r][..., 1], want[..., 1], atol=1e-9)
    mm = dict(m, P=P, crease_verts=np.array([[0, 1]], np.int32), crease_sharp=np.array([2.0], np.float32))
    fl2, _ = oracle.regular_patches(mm, 3)
    assert fl2.sum() < flags.sum()


# ---------------------------------------------------------------- mesh reordering (Sec. 4.5)

def test_cuthill_mckee_matches_scipy_when_the_start_is_unique():
    """With one connected component whose least-degree vertex is unique, the reverse Cuthill-McKee
    order is scipy's (its siblings are visited by degree, ties in index order)."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(120):
        n = int(rng.integers(6, 60))
        A = rng.random((n, n)) < rng.uniform(0.06, 0.3)
        A = np.triu(A, 1)
        A = A | A.T
        for i in range(n):                       # every vertex of degree >= 2 ...
            if A[i].sum() < 2:
                for j in ((i + 1) % n, (i + 2) % n):
                    A[i, j] = A[j, i] = True
        B = np.zeros((n + 1, n + 1), dtype=bool)  # ... and one pendant vertex: the unique start
        B[:n, :n] = A
        p = int(rng.integers(0, n))
        B[n, p] = B[p, n] = True
        G = sp.csr_matrix(B.astype(np.int32))
        if csgraph.connected_components(G)[0] != 1:
            continue
        adj = [np.flatnonzero(B[i]).tolist() for i in range(n + 1)]
        rcm = oracle.cuthill_mckee(adj)[::-1]
        np.testing.assert_array_equal(rcm, csgraph.reverse_cuthill_mckee(G, symmetric_mode=True))
        checked += 1
    assert checked > 100


def _ladder(n):
    """A strip of n quads: bottom row 0 .. n, top row n+1 .. 2n+1."""
    fv = []
    for i in range(n):
        fv += [i, i + 1, n + 2 + i, n + 1 + i]
    return dict(V=2 * (n + 1), F=n, off=np.arange(n + 1, dtype=np.int32) * 4, fv=np.asarray(fv, np.int32))


@pytest.mark.parametrize("n", [2, 3, 7])
def test_cuthill_mckee_of_a_ladder_alternates_the_rows(n):
    """Closed form: the start is corner 0 (degree 2, least index); its neighbours are top vertex
    n+1 (degree 2) and bottom vertex 1 (degree 3), so the top one comes first, and from there every
    rung follows: bottom vertex i at position 2i, top vertex n+1+i at 2i+1. RCM bandwidth 2, against
    n+1 for the row-by-row numbering. (A single quad, n = 1, is a 4-cycle: 0, 1, 2, 3.)"""
    m = _ladder(n)
    order = oracle.cuthill_mckee(oracle.vertex_graph(m))
    expect = np.empty(2 * (n + 1), dtype=np.int64)
    expect[0::2] = np.arange(n + 1)
    expect[1::2] = np.arange(n + 1, 2 * n + 2)
    np.testing.assert_array_equal(order, expect)
    r = oracle.rcm_reorder(m)
    assert oracle.bandwidth(oracle.vertex_graph(r)) == 2
    assert oracle.bandwidth(oracle.vertex_graph(m)) == n + 1
    np.testing.assert_array_equal(oracle.cuthill_mckee(oracle.vertex_graph(_ladder(1))), [0, 1, 2, 3])


def _shuffled(m, seed):
    rng = np.random.default_rng(seed)
    pv = rng.permutation(m["V"])
    order = rng.permutation(m["F"])
    off, fv = np.asarray(m["off"]), np.asarray(m["fv"])
    faces = [pv[fv[off[r]:off[r + 1]]] for r in order]
    noff = np.zeros(m["F"] + 1, np.int32)
    noff[1:] = np.cumsum([len(f) for f in faces])
    out = dict(m, off=noff, fv=np.concatenate(faces).astype(np.int32), P=np.asarray(m["P"])[np.argsort(pv)])
    if "crease_verts" in m:
        out["crease_verts"] = pv[np.asarray(m["crease_verts"])].astype(np.int32).reshape(-1, 2)
    return out


@pytest.mark.parametrize("scheme,mesh", [
    ("cc", lambda: synth.torus_cc_mixed(10, 8, merge_frac=0.05, split_frac=0.05, crease_frac=0.08, seed=41)),
    ("cc", lambda: synth.holed_cc_mixed(12, 10, holes=3, seed=42)),
    ("loop", lambda: synth.torus_tri(8, 6, seed=43)),
])
def test_reordering_keeps_the_surface(scheme, mesh):
    """Renumbering changes no point of the refined surface: two levels of the reordered mesh give
    the same set of points as two levels of the input (creases and boundaries included), while the
    reordered faces are sorted by their least vertex and keep their corners' cyclic order."""
    m = _shuffled(mesh(), 44)
    r = oracle.rcm_reorder(m)
    assert sorted(r["vmap"].tolist()) == list(range(m["V"]))
    assert sorted(r["fmap"].tolist()) == list(range(m["F"]))
    off, noff = np.asarray(m["off"]), r["off"]
    new_id = np.empty(m["V"], np.int64)
    new_id[r["vmap"]] = np.arange(m["V"])
    least = [r["fv"][noff[f]:noff[f + 1]].min() for f in range(r["F"])]
    assert all(a <= b for a, b in zip(least, least[1:]))
    ties = [f for f in range(1, r["F"]) if least[f] == least[f - 1]]
    assert ties and all(r["fmap"][f - 1] < r["fmap"][f] for f in ties)   # stable: input order
    for f, g in enumerate(r["fmap"]):
        np.testing.assert_array_equal(r["fv"][noff[f]:noff[f + 1]], new_id[m["fv"][off[g]:off[g + 1]]])
    a = oracle.subdivide(m, 2, scheme, keep_all=False)[2]["P"]
    b = oracle.subdivide(r, 2, scheme, keep_all=False)[2]["P"]
    assert a.shape == b.shape
    a = a[np.lexsort(a.T[::-1])]
    b = b[np.lexsort(b.T[::-1])]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_reordering_restores_a_small_bandwidth():
    """A shuffled 24 x 20 torus: its bandwidth is of the order of V; after RCM it is below twice
    the widest breadth-first level of a torus grid (the diagonal of its 24 x 20 cross-section)."""
    m = _shuffled(synth.torus_cc_plain(24, 20), 45)
    g = oracle.vertex_graph(m)
    r = oracle.rcm_reorder(m)
    assert oracle.bandwidth(g) > m["V"] // 2
    assert oracle.bandwidth(oracle.vertex_graph(r)) <= 2 * (24 + 20)


# ---- crease inheritance and vertex sharpness with unequal neighbours (Sec. 3.3) --------------

def _neighbours(lvl):
    """Vertex -> set of vertices sharing a face edge, from a level's face table."""
    nb = {}
    off, fv = lvl["off"], lvl["fv"]
    for r in range(len(off) - 1):
        f = fv[off[r]:off[r + 1]]
        for j in range(len(f)):
            a, b = int(f[j]), int(f[(j + 1) % len(f)])
            nb.setdefault(a, set()).add(b)
            nb.setdefault(b, set()).add(a)
    return nb


@pytest.mark.parametrize("scheme", ["cc", "loop"])
@pytest.mark.parametrize("case", _read_crease_cases("crease_inheritance.txt"), ids=lambda c: c["name"])
def test_chaikin_inheritance_with_unequal_neighbours(scheme, case):
    """Level-1 sharpness of every child half equals the paper's two Chaikin equations, hand-derived
    per half (tests/golden/crease_inheritance.txt); no other crease survives."""
    m, vid = _grid_mesh(scheme, case)
    out = oracle.subdivide(m, 1, scheme)
    nb = _neighbours(out[1])
    got = {}
    for (a, b), s in zip(out[1]["crease_verts"], out[1]["crease_sharp"]):
        got[(min(a, b), max(a, b))] = s
    expected_live = 0
    for (i0, j0, i1, j1), end, want in case["halves"]:
        a, b = vid(i0, j0), vid(i1, j1)
        x = nb[a] & nb[b]                      # the edge point of (a, b) on level 1
        assert len(x) == 1
        x = x.pop()
        v = a if end == 0 else b
        key = (min(v, x), max(v, x))
        if want == 0:
            assert key not in got, f"half at {v} of ({a},{b}) should have been dropped"
        else:
            expected_live += 1
            assert key in got, f"half at {v} of ({a},{b}) missing"
            assert got[key] == np.float32(want), (key, got[key], want)
    assert len(got) == expected_live


def _smooth_point(scheme, P, v, nb0):
    """The smooth level-1 point of a regular vertex from its fixed stencil (regular_stencils.txt)."""
    p = P[v]
    if scheme == "cc":
        # valence 4 on the quad grid: the edge neighbours share an edge; the diagonal ones share a face
        i, j = divmod(v, GRID)
        e = [((i + di) % GRID) * GRID + (j + dj) % GRID for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1))]
        d = [((i + di) % GRID) * GRID + (j + dj) % GRID for di, dj in ((1, 1), (1, -1), (-1, 1), (-1, -1))]
        assert set(e) == nb0[v]
        return (36.0 * p + 6.0 * P[e].sum(axis=0) + P[d].sum(axis=0)) / 64.0
    ring = sorted(nb0[v])
    assert len(ring) == 6
    return (10.0 * p + P[ring].sum(axis=0)) / 16.0


@pytest.mark.parametrize("scheme", ["cc", "loop"])
@pytest.mark.parametrize("case", _read_crease_cases("crease_vertex_sharpness.txt"), ids=lambda c: c["name"])
def test_vertex_sharpness_is_the_mean_of_unequal_creases(scheme, case):
    """Crease vertices with unequal incident sharpness (k = 2, k >= 3) and darts (k = 1) at level
    1 against hand-derived blend weights (tests/golden/crease_vertex_sharpness.txt)."""
    m, vid = _grid_mesh(scheme, case)
    out = oracle.subdivide(m, 1, scheme)
    P = m["P"].astype(np.float64)
    nb0 = _neighbours(dict(off=m["off"], fv=m["fv"]))
    creased = {}
    for (i0, j0, i1, j1), _ in case["creases"]:
        a, b = vid(i0, j0), vid(i1, j1)
        creased.setdefault(a, []).append(b)
        creased.setdefault(b, []).append(a)
    for (i, j), rule, w in case["vertices"]:
        v = vid(i, j)
        smooth = _smooth_point(scheme, P, v, nb0)
        if rule == "smooth":
            want = smooth
        elif rule == "k2":
            a, b = creased[v]
            want = w * (P[a] + 6.0 * P[v] + P[b]) / 8.0 + (1.0 - w) * smooth
        else:
            want = w * P[v] + (1.0 - w) * smooth
        np.testing.assert_allclose(out[1]["P"][v], want, rtol=0, atol=1e-15)


# ---- sqrt(3) feature edges: boundaries and infinitely sharp creases (Kobbelt 2000) ---------------

def _ternary_cubic_mask():
    """The coefficients c_k of N(t) = sum_k c_k N(3t - k) for the uniform cubic B-spline N,
    found by least squares on samples of the Cox-de Boor basis (not typed in)."""
    t = np.linspace(0.0, 4.0, 1201)[:-1]
    A = np.stack([_cox_de_boor(3 * t - k, 0, 4) for k in range(10)], axis=1)
    c, *_ = np.linalg.lstsq(A, _cox_de_boor(t, 0, 4), rcond=None)
    return c


def _refine_closed_polygon_3(P, c):
    """Control polygon of the same closed cubic B-spline on a third of the knot spacing:
    Q_m = sum_j c_{m - 3j} P_j (indices cyclic), rolled so that entry 3i is the point at P_i (the
    mask's centre is c_4, so Q_{3i+4} sits at P_i)."""
    n = len(P)
    Q = np.zeros((3 * n, 3))
    for m in range(3 * n):
        for j in range(n):
            k = (m - 3 * j) % (3 * n)
            if k < len(c):
                Q[m] += c[k] * P[j]
    return np.roll(Q, -4, axis=0)


@pytest.mark.parametrize("mesh", [synth.triangulate(synth.tube_cc(10, 6, jitter=0.2, seed=41)),
                                  synth.triangulate(synth.sheet_cc(6, 5, seed=42)),
                                  synth.triangulate(synth.holed_cc_mixed(16, 14, holes=3, seed=43)),
                                  synth.polygon(3)],
                         ids=["tube", "sheet", "holes", "triangle"])
def test_sqrt3_boundary_is_ternary_cubic_bspline_curve(mesh):
    """sqrt(3) boundaries: every second step refines each boundary loop as the cubic B-spline
    curve of the level-0 loop on a third of the knot spacing (the mask comes from the Cox-de Boor
    basis), and every first step leaves the boundary points where they are."""
    c = _ternary_cubic_mask()
    np.testing.assert_allclose(c * 27.0, [1, 4, 10, 16, 19, 16, 10, 4, 1, 0], atol=1e-9)
    out = oracle.subdivide(mesh, 4, "sqrt3")
    expected = [out[0]["P"][loop].astype(np.float64) for loop in _boundary_loops(out[0])]
    for l in range(1, 5):
        if l % 2 == 0:
            expected = [_refine_closed_polygon_3(poly, c) for poly in expected]
        loops = _boundary_loops(out[l])
        assert sorted(len(x) for x in loops) == sorted(len(x) for x in expected)
        got = np.concatenate([out[l]["P"][x] for x in loops])
        np.testing.assert_allclose(_as_sorted(got), _as_sorted(np.concatenate(expected)), atol=1e-12)


def test_sqrt3_sharp_crease_is_ternary_cubic_bspline_curve():
    """An infinitely sharp crease loop on a sqrt(3) torus refines as the ternary cubic B-spline
    curve of its polygon, whatever the surface on either side, and keeps still on first steps."""
    N = M = 9
    m = synth.torus_tri(N, M, flip_frac=0.0, creases=False, jitter=0.05, seed=44)
    m["crease_verts"], m["crease_sharp"] = _loop_creases(N, M, np.inf)
    c = _ternary_cubic_mask()
    out = oracle.subdivide(m, 4, "sqrt3")
    poly = m["P"][[i * M for i in range(N)]].astype(np.float64)
    for l in range(1, 5):
        if l % 2 == 0:
            poly = _refine_closed_polygon_3(poly, c)
        seq = _ordered_loop(out[l], 0)
        got = out[l]["P"][seq]
        if not np.allclose(got[1], poly[1], atol=1e-12):
            got = got[[0] + list(range(len(seq) - 1, 0, -1))]
        assert len(seq) == len(poly)
        np.testing.assert_allclose(got, poly, atol=1e-12)
        assert np.all(np.isinf(out[l]["crease_sharp"]))


def test_sqrt3_finite_sharpness_is_ignored_and_corners_fixed():
    """Finite sharpness has no sqrt(3) form (the paper and Kobbelt 2000 give none): it changes
    nothing. Three infinitely sharp creases meeting at a vertex (a corner) keep it fixed."""
    N = M = 8
    base = synth.torus_tri(N, M, flip_frac=0.0, creases=False, jitter=0.04, seed=45)
    plain = oracle.subdivide(base, 3, "sqrt3")
    fin = dict(base, crease_verts=np.array([[0, M], [M, 2 * M]], np.int32),
               crease_sharp=np.array([2.5, 0.5], np.float32))
    out = oracle.subdivide(fin, 3, "sqrt3")
    for l in range(4):
        np.testing.assert_array_equal(out[l]["fv"], plain[l]["fv"])
        np.testing.assert_array_equal(out[l]["P"], plain[l]["P"])
    v = 3 * M + 3
    corner = dict(base, crease_verts=np.array([[v, v + M], [v, v + 1], [v, v - M]], np.int32),
                  crease_sharp=np.full(3, np.inf, np.float32))
    out = oracle.subdivide(corner, 4, "sqrt3")
    for l in range(1, 5):
        np.testing.assert_array_equal(out[l]["P"][v], base["P"][v].astype(np.float64))


def test_sqrt3_boundary_leaves_far_interior_unchanged():
    """Cutting a ring of quads (two triangles each) out of a sqrt(3) torus leaves the level-2 and
    level-4 children of triangles far from the cut exactly as on the closed torus."""
    N, M = 14, 8
    closed = synth.torus_cc_plain(N, M, jitter=0.05, seed=46)
    F = closed["F"] - M
    cut = dict(closed, F=F, off=closed["off"][:F + 1], fv=closed["fv"][:4 * F])
    closed, cut = synth.triangulate(closed), synth.triangulate(cut)
    for levels in (2, 4):
        a = oracle.subdivide(closed, levels, "sqrt3")[levels]
        b = oracle.subdivide(cut, levels, "sqrt3")[levels]
        q = 2 * 3 ** levels                          # refined triangles of one quad
        for i in range(4, N - 5):
            for j in range(M):
                r = i * M + j
                ca = a["fv"][3 * q * r:3 * q * (r + 1)]
                cb = b["fv"][3 * q * r:3 * q * (r + 1)]
                np.testing.assert_array_equal(a["P"][ca], b["P"][cb])
        assert not np.array_equal(a["P"][a["fv"][:3 * q]], b["P"][b["fv"][:3 * q]])
