"""B300-native matrix-free LDG hot path: residual, exact J.v and Newton-GMRES
(CUDA kernels for sm_103a behind the C-ABI of include/ldg.h)."""
from . import synth  # noqa: F401

__all__ = ["synth", "ldg", "build"]
