"""GB300-native multigrid-preconditioned CG solver for SIMP topology optimisation.

The compute path is the CUDA library built from ``csrc/`` (``build.build()``) and reached
through its C ABI (``include/tomg.h``); :mod:`.tomg` is the ctypes binding.
"""
__all__ = ["build", "tomg"]
