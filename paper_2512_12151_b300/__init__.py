"""B300 (sm_103a) implementation of the inner Newton step, active-set update
and CCD of the barrier-free augmented-Lagrangian contact method
(arXiv 2512.12151), exposed through the C ABI in include/bf.h."""
from . import scenes  # noqa: F401

__all__ = ["scenes", "binding", "build"]
