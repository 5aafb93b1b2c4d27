"""Regular-patch evaluation (Sec. 3.4) on the CUDA path against the oracle: the regular faces of a
level bit for bit, and every sample of their bicubic B-spline patches within 2e-6 x the
bounding-box diagonal (FP32 basis against the oracle's Cox-de Boor in FP64)."""
import numpy as np
import pytest

import oracle
from paper_1809_06047_gb300 import synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,mesh", [
    ("mixed_creases", lambda: synth.torus_cc_mixed(16, 14, merge_frac=0.03, split_frac=0.02, crease_frac=0.05,
                                                   seed=111)),
    ("holes", lambda: synth.holed_cc_mixed(14, 12, holes=3, seed=112)),
    ("regular", lambda: synth.torus_cc_plain(10, 9, jitter=0.05, seed=113)),
])
@pytest.mark.parametrize("level", [0, 1, 2])
def test_regular_patches_match_oracle(name, mesh, level):
    import torch
    from paper_1809_06047_gb300 import alsub
    m = mesh()
    samples = 5
    ref = oracle.subdivide(m, level, "cc", keep_all=False)[level]
    flags_ref, grids = oracle.regular_patches(ref, samples)
    M = alsub.Mesh.from_dict(m, "cc")
    T = alsub.Topology(M, level + 1, build=True)
    P0 = torch.from_numpy(np.ascontiguousarray(m["P"])).cuda()
    P = P0 if level == 0 else alsub.Topology(M, level, build=True).refine_vertices(P0)
    flags = T.regular_faces(level).cpu().numpy().astype(bool)
    np.testing.assert_array_equal(flags, flags_ref)
    faces = np.arange(ref["F"], dtype=np.int32)
    out = T.eval_patches(level, torch.from_numpy(faces).cuda(), P, samples).cpu().numpy()
    T.status()
    assert np.isnan(out[~flags]).all()
    if flags.any():
        got = out[flags]
        want = np.stack([grids[r] for r in np.flatnonzero(flags)])
        diag = float(np.linalg.norm(ref["P"].max(0) - ref["P"].min(0)))
        assert float(np.abs(got - want).max()) <= gpu_util.POS_TOL * diag
