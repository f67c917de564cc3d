"""GB300-native adaptive particle-mesh (APM) gravity level solve.

Implements the method of Passy & Bryan, "An adaptive particle-mesh gravity
solver for ENZO" (arXiv:1410.0010) as hand-written sm_103a CUDA kernels behind
the C ABI in include/apm.h (libapm.so).  This package holds the kernels
(csrc/), their build script (buildlib.py) and a thin Python binding
(_lib.py, solver.py); importing it does not load the library.
"""
from ._lib import ApmError  # noqa: F401

__all__ = ["ApmError", "Solver", "Particles", "build"]


def __getattr__(name):
    if name in ("Solver", "Particles"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)


def build(force=False, verbose=False):
    from . import buildlib
    return buildlib.build(force=force, verbose=verbose)
