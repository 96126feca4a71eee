"""GB300-native constrained Delaunay refinement (gDP2d hot path).

The compute path is the CUDA library ``libgdp.so`` (``csrc/``), reached
through the thin ctypes binding in ``gdp.py``.
"""
