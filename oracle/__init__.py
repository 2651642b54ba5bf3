"""FP64 CPU oracle of the windowed LBM-LES and its discrete adjoint.

Test infrastructure only: imported by tests, the smoke check and the CPU
baseline of the benchmark, never by the library.  See ``oracle.lbm``.
"""
from .lbm import *  # noqa: F401,F403
