"""GB300-native MG-MLMC++ estimation of tr(D^{-1}) for the 2D Schwinger
Wilson-Dirac operator (Frommer & Nasr Khalil, Lattice 2022).

The computation lives in libmgmlmc.so (hand-written sm_103a CUDA behind the C
ABI of include/mgmlmc.h); `paper_2303_11512_gb300.api` binds it with ctypes
and torch CUDA tensors, `paper_2303_11512_gb300.estimator` is the user-facing
driver.  Build the library with `python -m paper_2303_11512_gb300.build`.
"""

__all__ = ["api", "estimator", "build"]
