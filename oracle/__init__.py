"""Plain FP64 CPU oracle for the enlarged CG methods (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package; the CUDA solver never imports it.  The arithmetic lives in
``ecg_oracle.c``; ``ecg_oracle.py`` loads it through ctypes.
"""
from .ecg_oracle import *  # noqa: F401,F403
