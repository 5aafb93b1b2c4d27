"""C-ABI checks that need no GPU: the library builds, loads and exports every symbol that
include/*.h declares; host-side planning and validation reject bad input before any CUDA call."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import _lib, alsub, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(alsub_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    declared = _declared()
    assert len(declared) >= 15
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding declares the same set, no more, no fewer
    assert set(_lib.SIGNATURES) == set(declared)


def test_status_strings():
    lib = _lib.load()
    assert lib.alsub_status_string(0) == b"ALSUB_OK"
    assert lib.alsub_status_string(2) == b"ALSUB_ERR_NONMANIFOLD"


@pytest.mark.parametrize("name", ["cc_torus16_L3", "cc_creased_torus96_L6", "loop_tri_torus128_L6",
                                  "sqrt3_tri_torus128_L8"])
def test_plan_closed_forms(name):
    m = synth.workload(name)
    levels = m["levels"]
    counts = alsub.plan(m["scheme"], m["V"], m["F"], len(m["fv"]), levels)
    # against the oracle's own counts on the first levels
    ref = oracle.subdivide(m, min(levels, 2), m["scheme"], keep_all=True)
    for l, d in enumerate(ref):
        assert tuple(counts[l]) == (d["V"], d["F"], d["nnz"], d["E"])
    if name == "cc_creased_torus96_L6":
        assert counts[6][1] == 37_750_784
    if name == "loop_tri_torus128_L6":
        assert counts[6][1] == 134_217_728 and counts[6][0] == 67_108_864
    if name == "sqrt3_tri_torus128_L8":
        assert counts[8][1] == 214_990_848 and counts[8][0] == 107_495_424


def test_plan_rejects():
    with pytest.raises(alsub.AlsubError) as e:
        alsub.plan("cc", 8, 6, 23, 1)              # odd corner count: open mesh
    assert e.value.status == 3
    with pytest.raises(alsub.AlsubError) as e:
        alsub.plan("loop", 8, 6, 24, 1)            # not triangles
    assert e.value.status == 1
    with pytest.raises(alsub.AlsubError) as e:
        alsub.plan("cc", 1 << 20, 1 << 20, 1 << 22, 12)   # beyond int32
    assert e.value.status == 3


@pytest.mark.parametrize("scheme,mesh", [
    ("cc", lambda: synth.holed_cc_mixed(12, 10, holes=3, seed=71)),
    ("loop", lambda: synth.triangulate(synth.holed_cc_mixed(12, 10, holes=3, seed=72))),
    ("loop", lambda: synth.triangulate(synth.open_box())),
])
def test_plan_open_against_the_oracle(scheme, mesh):
    """Level counts of open meshes (E0 = (nnz + B) / 2, each boundary edge splitting in two)
    against the oracle's own counts, for sqrt(3) too (two kinds of step, Kobbelt 2000)."""
    m = mesh()
    off, fv = np.asarray(m["off"]), np.asarray(m["fv"])
    d = set()
    for r in range(m["F"]):
        f = fv[off[r]:off[r + 1]].tolist()
        d.update((f[j], f[(j + 1) % len(f)]) for j in range(len(f)))
    B = sum((b, a) not in d for a, b in d)
    assert B > 0
    counts = alsub.plan(scheme, m["V"], m["F"], len(fv), 3, boundary=B)
    ref = oracle.subdivide(m, 3, scheme, keep_all=True)
    for l, r in enumerate(ref):
        assert tuple(counts[l]) == (r["V"], r["F"], r["nnz"], r["E"])
    if scheme == "loop":
        # sqrt(3) (Kobbelt's boundary treatment): its own counts against the oracle's, over two
        # pairs of steps
        counts = alsub.plan("sqrt3", m["V"], m["F"], len(fv), 4, boundary=B)
        ref = oracle.subdivide(m, 4, "sqrt3", keep_all=True)
        for l, r in enumerate(ref):
            assert tuple(counts[l]) == (r["V"], r["F"], r["nnz"], r["E"])


def _create(scheme, V, F, fv, off=None, cv=None, cs=None):
    return alsub.Mesh(scheme, V, F, fv, off, cv, cs, stream=0)


def test_mesh_validation_on_host():
    c = synth.cube()
    with pytest.raises(alsub.AlsubError) as e:           # vertex id out of range
        _create("cc", 8, 6, np.where(c["fv"] == 7, 8, c["fv"]), c["off"])
    assert e.value.status == 1
    fv = c["fv"].copy()
    fv[1] = fv[0]                                        # repeated vertex in a face
    with pytest.raises(alsub.AlsubError) as e:
        _create("cc", 8, 6, fv, c["off"])
    assert e.value.status == 1
    with pytest.raises(alsub.AlsubError) as e:           # unused vertex
        _create("cc", 9, 6, c["fv"], c["off"])
    assert e.value.status == 1
    with pytest.raises(alsub.AlsubError) as e:           # Loop needs triangles
        _create("loop", 8, 6, c["fv"], c["off"])
    assert e.value.status == 1
    with pytest.raises(alsub.AlsubError) as e:           # negative sharpness
        _create("cc", 8, 6, c["fv"], c["off"], np.array([[0, 1]]), np.array([-1.0]))
    assert e.value.status == 1
    with pytest.raises(alsub.AlsubError) as e:           # NaN sharpness
        _create("cc", 8, 6, c["fv"], c["off"], np.array([[0, 1]]), np.array([np.nan]))
    assert e.value.status == 1
    with pytest.raises(alsub.AlsubError) as e:           # a sqrt(3) face that is not a triangle
        _create("sqrt3", 8, 6, c["fv"], c["off"])
    assert e.value.status == 1


def test_last_error_message():
    lib = _lib.load()
    out = np.zeros(8, np.int64)
    st = lib.alsub_plan(7, 1, 1, 3, 0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    assert st == 1 and b"scheme" in lib.alsub_last_error()


def test_plan_bytes_host_only():
    """Closed-form device sizes the serving admission uses: host only, no CUDA call."""
    m = synth.torus_cc_mixed(20, 20, seed=5)
    nnz = len(m["fv"])
    sizes = [alsub.plan_bytes("cc", m["V"], m["F"], nnz, L) for L in range(7)]
    assert all(b > a for a, b in zip(sizes, sizes[1:]))
    # the per-level arrays grow by 4x per level, so the total does too, asymptotically
    assert 3.5 < sizes[6] / sizes[5] < 4.5
    K = len(m["crease_sharp"])
    with_creases = alsub.plan_bytes("cc", m["V"], m["F"], nnz, 3, K, float(m["crease_sharp"].max()))
    assert with_creases > sizes[3]
    # sqrt(3) keeps infinitely sharp creases only (the feature path stores every level): finite
    # sharpness costs nothing, infinite sharpness takes the feature path's arrays
    t = synth.torus_tri(10, 10, seed=6)
    plain = alsub.plan_bytes("sqrt3", t["V"], t["F"], len(t["fv"]), 3)
    assert alsub.plan_bytes("sqrt3", t["V"], t["F"], len(t["fv"]), 3, 50, 3.5) == plain
    assert alsub.plan_bytes("sqrt3", t["V"], t["F"], len(t["fv"]), 3, 50, float("inf")) > plain
    for bad in [dict(nnz=nnz + 1), dict(levels=-1)]:
        with pytest.raises(alsub.AlsubError):
            alsub.plan_bytes("cc", m["V"], m["F"], bad.get("nnz", nnz), bad.get("levels", 2))
    with pytest.raises(alsub.AlsubError):
        alsub.plan_bytes("cc", m["V"], m["F"], nnz, 2, 3, -1.0)


def test_allocator_needs_both_callbacks():
    """alsub_mesh_create_ex refuses an allocator without a free callback before any device work."""
    lib = _lib.load()
    c = synth.cube()
    fv = np.ascontiguousarray(c["fv"], dtype=np.int32)
    a = _lib.Allocator(_lib.ALLOC_FN(lambda n, ctx, s: None), _lib.FREE_FN(), None)
    h = ctypes.c_void_p()
    st = lib.alsub_mesh_create_ex(0, 8, 6, None, fv.ctypes.data_as(ctypes.c_void_p), 0, None, None,
                                  ctypes.byref(a), None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"alloc and free" in lib.alsub_last_error()


def test_adaptive_operator_argument_checks_on_host():
    """alsub_build_adaptive_operator refuses a NULL chain, an empty one and flags other than
    TRANSPOSE and STACKED before it reads a handle or calls CUDA."""
    lib = _lib.load()
    out = ctypes.c_void_p()
    assert lib.alsub_build_adaptive_operator(None, 1, 0, None, ctypes.byref(out)) == 1
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.alsub_build_adaptive_operator(arr, 0, 0, None, ctypes.byref(out)) == 1
    assert lib.alsub_build_adaptive_operator(arr, 1, alsub.Operator.COMPOSE, None, ctypes.byref(out)) == 1
    assert lib.alsub_build_adaptive_operator(arr, 1, 0, None, None) == 1
    # a NULL entry in the chain
    assert lib.alsub_build_adaptive_operator(arr, 1, alsub.Operator.STACKED, None, ctypes.byref(out)) == 1
    assert b"NULL topology" in lib.alsub_last_error()
    assert out.value is None
