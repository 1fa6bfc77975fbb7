"""B300-native GP-BO hot path for the tuning methodology of arXiv 2403.08131.

Importing the package is cheap: the CUDA library (``libgpbo.so``) is loaded only
when :mod:`paper_2403_08131_b300.gpbo` is imported, and that import fails loudly
when the library has not been built.  The seeded input generators live in
:mod:`paper_2403_08131_b300.workloads` and need only numpy.
"""

__all__ = ["gpbo", "workloads"]
