"""Serving loop: every request served in a mix (overlapping slots, cached topologies and operators,
fresh meshes) equals the same request run alone through the plain calls; the closed-form sizes the
admission uses equal what the handles allocate; timeouts, budget refusals and device-detected
mesh errors come back as statuses while the server keeps serving."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu

TOL = 2e-6


def _close(got, want):
    diag = float(np.linalg.norm(want.max(0) - want.min(0)))
    assert got.shape == want.shape
    assert float(np.abs(got - want).max()) <= TOL * max(diag, 1e-3)


def _alone(m, scheme, levels, P0):
    """The plain path: fresh mesh, topology build and vertex refinement, nothing cached."""
    import torch
    from paper_1809_06047_gb300 import alsub
    M = alsub.Mesh.from_dict(m, scheme)
    T = alsub.Topology(M, levels)
    out = T.refine_vertices(torch.from_numpy(np.ascontiguousarray(P0, np.float32)).cuda())
    torch.cuda.synchronize()
    T.status()
    return out.cpu().numpy()


def _vs_oracle(m, scheme, levels, P0, got, topo_cache=None):
    """The served result against the oracle: positions relabelled through the face tables of a
    CUDA run of the same mesh (the library numbers edges its own way)."""
    mm = dict(m, P=np.ascontiguousarray(P0, np.float32))
    key = id(m)
    if topo_cache is not None and key in topo_cache:
        gpu = topo_cache[key]
    else:
        gpu = gpu_util.gpu_run(mm, scheme, levels, per_level=False)
        if topo_cache is not None:
            topo_cache[key] = gpu
    gpu = [dict(g) for g in gpu]
    gpu[0]["P"] = mm["P"]
    gpu[-1]["P"] = got
    ref = oracle.subdivide(mm, levels, scheme, keep_all=True)
    gpu_util.compare(scheme, gpu, ref, pos_levels={levels})


def test_plan_bytes_match_allocation():
    from paper_1809_06047_gb300 import alsub
    cases = [("cc", synth.torus_cc_mixed(14, 10, seed=91), 3), ("cc", synth.torus_cc_plain(8, 6, seed=92), 4),
             ("loop", synth.torus_tri(9, 7, seed=93), 3), ("sqrt3", synth.torus_tri(8, 8, seed=94, creases=False), 4),
             ("cc", synth.cube(), 0)]
    for scheme, m, lv in cases:
        cs = m.get("crease_sharp")
        K = 0 if cs is None else int(np.count_nonzero(cs))
        smax = 0.0 if cs is None or len(cs) == 0 else float(np.max(cs))
        want = alsub.plan_bytes(scheme, m["V"], m["F"], len(m["fv"]), lv, K, smax)
        M = alsub.Mesh.from_dict(m, scheme)
        T = alsub.Topology(M, lv, build=False)
        assert T.bytes() == want, (scheme, lv)
        T2 = alsub.Topology(M, lv)
        assert T2.bytes() == want


def test_mix_equals_alone():
    from paper_1809_06047_gb300 import alsub
    w = synth.serving_requests(n_requests=40, n_resident=4, fmin=200, fmax=3000, rate_hz=1e5, seed=777)
    S = alsub.Server(budget_bytes=8 << 30, max_slots=6)
    try:
        rids = [S.register(m, m["scheme"], m["levels"],
                           frames=("operator", "eval", "fastest", "operator_mf")[i % 4])
                for i, m in enumerate(w["resident"])]
        tickets = []
        for q in w["requests"]:
            if q["kind"] == "frame":
                tickets.append(S.submit_frame(rids[q["resident"]], q["P"]))
            else:
                m = q["mesh"]
                tickets.append(S.submit_mesh(m, m["scheme"], m["levels"]))
        results = [S.poll(t, timeout_us=60_000_000) for t in tickets]
        st = S.stats()
    finally:
        S.close()
    cache = {}
    for q, r in zip(w["requests"], results):
        assert r is not None and r["status"] == 0
        if q["kind"] == "frame":
            m = w["resident"][q["resident"]]
            P0 = q["P"]
        else:
            m = q["mesh"]
            P0 = m["P"]
        _close(r["P"], _alone(m, m["scheme"], m["levels"], P0))
        _vs_oracle(m, m["scheme"], m["levels"], P0, r["P"], cache)
        assert r["done_s"] >= r["start_s"] >= r["submit_s"]
    assert st["completed"] == len(tickets) and st["failed"] == 0
    # requests were admitted side by side and their kernels overlapped on the device
    assert st["peak_in_flight"] > 1, st
    assert st["device_overlap_peak"] > 1, st
    assert st["frames_operator"] + st["frames_eval"] + st["meshes"] == len(tickets)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["hbm_peak"] <= st["hbm_budget"]


def test_frame_against_oracle_and_pinned_output():
    """A frame served by the cached composite operator, written by DMA into page-locked memory,
    against the oracle."""
    import torch
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_mixed(10, 12, seed=95)
    S = alsub.Server(budget_bytes=1 << 30, max_slots=2)
    try:
        rid = S.register(m, "cc", 3, frames="operator")
        P = (m["P"] * 1.25 + 0.5).astype(np.float32)
        VL = int(alsub.plan("cc", m["V"], m["F"], len(m["fv"]), 3)[3][0])
        out = torch.empty((VL, 3), dtype=torch.float32, pin_memory=True).numpy()
        r = S.poll(S.submit_frame(rid, P, out=out), timeout_us=30_000_000)
        r2 = S.poll(S.submit_frame(rid, P), timeout_us=30_000_000)
        assert S.stats()["frames_operator"] == 2
    finally:
        S.close()
    assert r["status"] == 0 and r["P"] is not None
    assert np.shares_memory(r["P"], out)
    mm = dict(m, P=P)
    ref = oracle.subdivide(mm, 3, "cc", keep_all=True)
    # the library numbers edges its own way: relabel through the face tables of the alone run
    gpu = gpu_util.gpu_run(mm, "cc", 3, per_level=False)
    _close(gpu[-1]["P"], _alone(m, "cc", 3, P))
    gpu[-1]["P"] = out
    gpu_util.compare("cc", gpu, ref, pos_levels={3})
    assert np.array_equal(r2["P"], out)      # same path, same bits


@pytest.mark.parametrize("frames", ["operator_mf", "eval"])
def test_frames_of_one_resident_in_flight_together(frames):
    """Many frames of one resident admitted side by side (six slots, three workers): each result is
    bit for bit the plain eval call's on its own input. Matrix-free operator frames share the
    operator's scratch and run one after another on the device; eval frames use their own."""
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_mixed(30, 24, crease_frac=0.1, seed=88)
    rng = np.random.default_rng(89)
    Ps = [(m["P"] + 0.05 * rng.standard_normal(m["P"].shape)).astype(np.float32) for _ in range(24)]
    S = alsub.Server(budget_bytes=4 << 30, max_slots=6)
    try:
        rid = S.register(m, "cc", 4, frames=frames)
        tickets = [S.submit_frame(rid, P) for P in Ps]
        results = [S.poll(t, timeout_us=60_000_000) for t in tickets]
        st = S.stats()
    finally:
        S.close()
    assert st["completed"] == len(Ps) and st["failed"] == 0
    assert st["frames_operator" if frames == "operator_mf" else "frames_eval"] == len(Ps)
    assert st["peak_in_flight"] > 1, st
    for P, r in zip(Ps, results):
        assert r["status"] == 0
        assert np.array_equal(r["P"], _alone(m, "cc", 4, P))
    _vs_oracle(m, "cc", 4, Ps[-1], results[-1]["P"])


def test_timeout_pause_and_resume():
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_plain(8, 8, seed=96)
    S = alsub.Server(budget_bytes=1 << 30, max_slots=2)
    try:
        S.pause(True)
        t = S.submit_mesh(m, "cc", 2)
        assert S.poll(t, timeout_us=0) is None          # NOT_READY
        assert S.poll(t, timeout_us=20_000) is None     # TIMEOUT after 20 ms: nothing is admitted
        assert S.stats()["queued"] == 1
        S.pause(False)
        r = S.poll(t, timeout_us=30_000_000)
        assert r is not None and r["status"] == 0
        _close(r["P"], _alone(m, "cc", 2, m["P"]))
        with pytest.raises(alsub.AlsubError) as e:
            S.poll(t, timeout_us=0)                     # released after the first successful poll
        assert e.value.status == 1
    finally:
        S.close()


def test_budget_refusals():
    from paper_1809_06047_gb300 import alsub
    m = synth.torus_cc_plain(16, 16, seed=97)
    need = alsub.plan_bytes("cc", m["V"], m["F"], len(m["fv"]), 4)
    # a budget smaller than one request: refused at submit, and a resident cannot be made
    S = alsub.Server(budget_bytes=need // 2, max_slots=2)
    try:
        with pytest.raises(alsub.AlsubError) as e:
            S.submit_mesh(m, "cc", 4)
        assert e.value.status == 4
        with pytest.raises(alsub.AlsubError) as e:
            S.register(m, "cc", 4)
        assert e.value.status == 4
        small = synth.cube()
        r = S.poll(S.submit_mesh(small, "cc", 1), timeout_us=30_000_000)
        assert r["status"] == 0                         # the server still serves what fits
    finally:
        S.close()
    # a queued request that a later resident pushes over the budget finishes with status OOM
    S = alsub.Server(budget_bytes=int(need * 1.6), max_slots=2)
    try:
        S.pause(True)
        t = S.submit_mesh(m, "cc", 4)
        S.register(m, "cc", 4, frames="eval")          # takes about `need` of the budget
        S.pause(False)
        r = S.poll(t, timeout_us=30_000_000)
        assert r["status"] == 4 and r["P"] is None
        assert S.stats()["failed"] == 1
    finally:
        S.close()


def test_bad_mesh_fails_only_its_request():
    from paper_1809_06047_gb300 import alsub
    c = synth.cube()
    fv = np.concatenate([c["fv"], c["fv"][:4], c["fv"][:4][::-1]]).astype(np.int32)
    bad = dict(V=8, F=8, fv=fv, off=np.arange(0, 33, 4, dtype=np.int32), P=c["P"])
    good = synth.torus_cc_plain(6, 6, seed=98)
    S = alsub.Server(budget_bytes=1 << 30, max_slots=2)
    try:
        t_bad = S.submit_mesh(bad, "cc", 2)
        t_inv = S.submit_mesh(dict(bad, fv=np.where(fv == 3, 99, fv)), "cc", 1)   # vertex id out of range
        t_good = S.submit_mesh(good, "cc", 3)
        r_bad, r_inv, r_good = (S.poll(t, timeout_us=30_000_000) for t in (t_bad, t_inv, t_good))
        st = S.stats()
    finally:
        S.close()
    assert r_bad["status"] == 2 and r_bad["P"] is None     # non-manifold, found on the device
    assert r_inv["status"] == 1                              # refused by host validation
    assert r_good["status"] == 0
    _close(r_good["P"], _alone(good, "cc", 3, good["P"]))
    assert st["failed"] == 2 and st["completed"] == 1
