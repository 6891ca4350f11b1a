"""GB300-native matrix-free S_N radiative-transfer operator A = Id - Lambda Sigma
and its Krylov solve (hand-written CUDA for sm_103a behind a C ABI).

The CUDA library is loaded lazily by :mod:`paper_2602_21958_gb300.rt`; importing
this package alone loads nothing native.
"""
__all__ = ["workloads", "rt"]
