"""Exhaustive QUBO minimisation by Gray-code walk on one GB300 (arXiv 2310.19373).

The compute path is the CUDA library ``libqubobf`` (declared in include/qbf.h);
this package only builds it and marshals arguments to it.
"""
from . import inputs  # noqa: F401  (seeded generators, no CUDA)

__all__ = ["inputs", "solve", "walk_trace", "QbfError"]


def __getattr__(name):
    if name in ("solve", "walk_trace", "QbfError", "Solution", "make_options"):
        from . import _binding

        return getattr(_binding, name)
    raise AttributeError(name)
