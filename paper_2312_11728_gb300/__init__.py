"""GB300-native batched Kalman track building and fitting (arXiv:2312.11728 hot path).

The compute path is the C-ABI library ``libmkgb.so`` (hand-written CUDA for sm_103a),
reached through :mod:`paper_2312_11728_gb300.mkgb`.  Importing this package loads
nothing; the binding raises if the library has not been built.
"""
__all__ = ["mkgb", "synth"]
