"""GB300-native enlarged Conjugate Gradient solvers (arXiv 2305.19013).

The solver itself lives in the CUDA library ``libecg.so`` built from
``csrc/``; ``ecg`` is its thin ctypes binding and ``workloads`` builds seeded
synthetic problems.  Importing the package loads nothing: submodules are
imported on demand.
"""
__all__ = ["ecg", "workloads", "build"]
