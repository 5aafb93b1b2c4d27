"""Crease cases of tests/golden/crease_inheritance.txt and crease_vertex_sharpness.txt (Sec. 3.3):
creases tagged on a 10 x 10 grid torus, shared by the oracle pins and the GPU parity tests."""
import os
from fractions import Fraction

import numpy as np

from paper_1809_06047_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def read_cases(name):
    """Cases of tests/golden/crease_*.txt: creases, expected child halves, expected vertices."""
    def sig(t):
        return np.inf if t == "inf" else float(Fraction(t))
    cases, cur = [], None
    for line in open(os.path.join(GOLD, name)):
        tok = line.split("#")[0].split()
        if not tok:
            continue
        if tok[0] == "case":
            cur = dict(name=tok[1], creases=[], halves=[], vertices=[])
            cases.append(cur)
        elif tok[0] == "crease":
            cur["creases"].append((tuple(int(t) for t in tok[1:5]), sig(tok[5])))
        elif tok[0] == "half":
            cur["halves"].append((tuple(int(t) for t in tok[1:5]), int(tok[5]), sig(tok[6])))
        elif tok[0] == "vertex":
            cur["vertices"].append(((int(tok[1]), int(tok[2])), tok[3], float(Fraction(tok[4]))))
    return cases


GRID = 10


def grid_mesh(scheme, case):
    """10 x 10 grid torus (quads, or split into triangles without flips) with the case's creases."""
    if scheme == "cc":
        m = synth.torus_cc_plain(GRID, GRID, jitter=0.03, seed=31)
    else:
        m = synth.torus_tri(GRID, GRID, flip_frac=0.0, creases=False, jitter=0.03, seed=32)
    vid = lambda i, j: (i % GRID) * GRID + (j % GRID)   # noqa: E731
    m["crease_verts"] = np.array([[vid(c[0], c[1]), vid(c[2], c[3])] for c, _ in case["creases"]],
                                 dtype=np.int32).reshape(-1, 2)
    m["crease_sharp"] = np.array([s for _, s in case["creases"]], dtype=np.float32)
    return m, vid
