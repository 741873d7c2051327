"""GB300-native (sm_103a) SlingBAG Pro hot path: differentiable N-wave
radiator, its adjoint, zero-gradient filtering and adaptive growth, behind
the C ABI of include/slingbag.h.

Importing the package loads nothing; `paper_2601_00551_gb300.slingbag`
loads the CUDA library on first use and raises if it is missing.
"""

__all__ = ["slingbag", "build"]
