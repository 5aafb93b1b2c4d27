"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Topology: bit-exact after canonical relabelling of the edge numbering; crease lists: bit-exact
(FP32 sharpness); positions: max abs error <= 2e-6 x bounding-box diagonal at every level.
"""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import crease_cases, gpu_util

pytestmark = pytest.mark.gpu


def _check(mesh, scheme, levels, mode="static"):
    ref = oracle.subdivide(mesh, levels, scheme, keep_all=True)
    gpu = gpu_util.gpu_run(mesh, scheme, levels, mode=mode)
    return gpu_util.compare(scheme, gpu, ref)


@pytest.mark.parametrize("mode", ["static", "dynamic"])
def test_cc_torus16_L3(mode):
    """Plain Catmull-Clark, 3 levels of a 16 x 16 quad torus -> 16384 quads."""
    m = synth.workload("cc_torus16_L3")
    errs = _check(m, "cc", 3, mode)
    assert max(errs) < 2e-6


@pytest.mark.parametrize("mode", ["static", "dynamic"])
def test_cc_creased_torus96_L5(mode):
    """Mixed polygons (hexagons, quads, triangles), valences 3..6, semi-sharp creases: every
    level up to 5 (the creases have all decayed by level 4; the last level derives its edge ids
    and twins from level 3)."""
    m = synth.workload("cc_creased_torus96_L6")
    _check(m, "cc", 5, mode)


@pytest.mark.parametrize("mode", ["static", "dynamic"])
def test_loop_tri_torus128_L4(mode):
    """Loop with 2% infinitely sharp edges on a flipped triangulated torus (valence 4..8)."""
    m = synth.workload("loop_tri_torus128_L6")
    _check(m, "loop", 4, mode)


@pytest.mark.parametrize("mode", ["static", "dynamic"])
def test_sqrt3_tri_torus128_L5(mode):
    m = synth.workload("sqrt3_tri_torus128_L8")
    _check(m, "sqrt3", 5, mode)


SMALL = [
    ("cc", synth.cube, 4),
    ("cc", lambda: synth.pillow(6), 3),
    ("cc", lambda: synth.pillow(11), 3),
    ("cc", lambda: synth.prism(12), 4),
    ("cc", lambda: synth.torus_cc_mixed(7, 9, seed=41), 3),
    ("loop", synth.octahedron, 4),
    ("loop", synth.tetrahedron, 4),
    ("loop", lambda: synth.torus_tri(7, 5, seed=42), 3),
    ("sqrt3", synth.tetrahedron, 5),
    ("sqrt3", synth.octahedron, 4),
    ("sqrt3", lambda: synth.torus_tri(6, 9, seed=43, creases=False), 4),
]


@pytest.mark.parametrize("scheme,fn,levels", SMALL)
@pytest.mark.parametrize("mode", ["static", "dynamic"])
def test_small_and_degenerate(scheme, fn, levels, mode):
    """Valence 2 (pillow) and 3 (cube, tetrahedron), n-gons, tiny grids with ragged tails."""
    _check(fn(), scheme, levels, mode)


def _ring_creases(N, M, sigma):
    cv = np.array([[i * M, ((i + 1) % N) * M] for i in range(N)], dtype=np.int32)
    return cv, np.full(N, sigma, dtype=np.float32)


@pytest.mark.parametrize("sigma", [np.inf, 3.0, 1.0, 0.4])
@pytest.mark.parametrize("scheme", ["cc", "loop"])
def test_crease_loop_rules(scheme, sigma):
    """A ring of equal sharpness: infinitely sharp, decaying, one-step and fractional."""
    N, M = 8, 6
    m = synth.torus_cc_plain(N, M, jitter=0.02) if scheme == "cc" else \
        synth.torus_tri(N, M, flip_frac=0.0, creases=False, jitter=0.02)
    m["crease_verts"], m["crease_sharp"] = _ring_creases(N, M, sigma)
    _check(m, scheme, 4)


def test_corner_creases_cube():
    """All 12 cube edges infinitely sharp: k = 3 corners stay fixed, edges follow B-splines."""
    m = synth.cube()
    e = set()
    for r in range(6):
        f = m["fv"][4 * r:4 * r + 4]
        for j in range(4):
            a, b = int(f[j]), int(f[(j + 1) % 4])
            e.add((min(a, b), max(a, b)))
    m["crease_verts"] = np.array(sorted(e), dtype=np.int32)
    m["crease_sharp"] = np.full(len(e), np.inf, dtype=np.float32)
    _check(m, "cc", 4)


def test_mixed_sharpness_darts_and_corners():
    """Random sharpness on a mixed mesh: darts (k = 1), creases (k = 2) and corners (k >= 3)."""
    m = synth.torus_cc_mixed(12, 12, crease_frac=0.3, seed=44)
    _check(m, "cc", 4)


def test_levels_zero_and_one():
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_mixed(6, 6, seed=45)
    M = alsub.Mesh.from_dict(m, "cc")
    T0 = alsub.Topology(M, 0)
    P0 = torch.from_numpy(m["P"]).cuda()
    assert torch.equal(T0.refine_vertices(P0), P0)
    _check(m, "cc", 1)


def test_dynamic_equals_static_bitwise():
    """alsub_subdivide (fused build + eval) and alsub_refine_topology + alsub_refine_vertices
    give identical bits, and two runs give identical bits."""
    import torch
    from paper_1809_06047_gb300 import alsub
    for name in ("cc_creased_torus96_L6", "loop_tri_torus128_L6"):
        m = synth.workload(name)
        lv = 5 if m["scheme"] == "cc" else 4
        M = alsub.Mesh.from_dict(m)
        P0 = torch.from_numpy(m["P"]).cuda()
        Ts = alsub.Topology(M, lv, build=True)
        Td = alsub.Topology(M, lv, build=False)
        a = Ts.refine_vertices(P0)
        b = Td.subdivide(P0)
        c = Td.subdivide(P0)
        torch.cuda.synchronize()
        Ts.status(); Td.status()
        assert torch.equal(a, b) and torch.equal(b, c)
        for l in range(lv + 1):
            assert np.array_equal(Ts.faces(l), Td.faces(l))


def test_device_errors_are_latched():
    """Non-manifold and crease-not-an-edge inputs are reported, not trapped."""
    from paper_1809_06047_gb300 import alsub
    c = synth.cube()
    # two faces sharing a directed edge twice: glue a duplicate of face 0 with a seventh vertex
    fv = np.concatenate([c["fv"], c["fv"][:4], c["fv"][:4][::-1]]).astype(np.int32)
    off = np.arange(0, 4 * 8 + 1, 4, dtype=np.int32)
    M = alsub.Mesh("cc", 8, 8, fv, off)
    T = alsub.Topology(M, 1)
    with pytest.raises(alsub.AlsubError) as e:
        T.status()
    assert e.value.status == 2
    M2 = alsub.Mesh("cc", 8, 6, c["fv"], c["off"], np.array([[0, 7]]), np.array([1.0]))
    T2 = alsub.Topology(M2, 1)
    with pytest.raises(alsub.AlsubError) as e:
        T2.status()
    assert e.value.status == 1


CREASE_CASES = [(f, c) for f in ("crease_inheritance.txt", "crease_vertex_sharpness.txt")
                for c in crease_cases.read_cases(f)]


@pytest.mark.parametrize("scheme", ["cc", "loop"])
@pytest.mark.parametrize("case", [c for _, c in CREASE_CASES], ids=[c["name"] for _, c in CREASE_CASES])
def test_unequal_crease_sharpness(scheme, case):
    """The meshes that pin the oracle's Chaikin inheritance and mean vertex sharpness to Sec. 3.3
    (unequal neighbours, darts, corners, infinite next to finite): crease lists bit-exact and
    positions within tolerance over four levels, static and dynamic."""
    m, _ = crease_cases.grid_mesh(scheme, case)
    for mode in ("static", "dynamic"):
        _check(m, scheme, 4, mode)
