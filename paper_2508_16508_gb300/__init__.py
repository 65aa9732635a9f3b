"""GB300-native engine for the selective-update hot path of ABMax (arXiv 2508.16508).

The product is ``libabm.so`` (C ABI, include/abm.h) built from ``csrc/`` for
sm_103a; :mod:`.abm` is its ctypes binding and :mod:`.engine` a thin object
layer over it for torch users. Nothing in this package computes on the CPU.
"""
from . import abm  # noqa: F401

__all__ = ["abm"]
