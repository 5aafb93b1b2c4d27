"""GB300-native uniform subdivision (Catmull-Clark, Loop, sqrt(3)) as sparse linear algebra on
the mesh matrix, after AlSub (Mlakar et al., arXiv 1809.06047).

The compute path is libalsub.so (hand-written CUDA for sm_103a behind a C ABI, include/alsub.h);
``paper_1809_06047_gb300.alsub`` is its Python binding. Importing this package does not load
the library; the first call into the binding does, and raises if it cannot.
"""

__all__ = ["alsub", "synth", "build"]
