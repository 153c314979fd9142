"""GB300-native conservative spectral Boltzmann collision operator (arXiv:1211.0540).

The compute path lives in the CUDA library ``libbte`` (``csrc/``), reached
through the C ABI declared in ``include/bte.h``. ``paper_1211_0540_gb300.bte``
is the thin ctypes binding; importing the package itself loads nothing.
"""
