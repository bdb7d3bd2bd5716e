"""GB300-native HDG linearize + condense (compressible Navier-Stokes).

The compute path is ``libhdg.so`` (hand-written CUDA for sm_103a behind the C-ABI
of ``include/hdg.h``); ``hdg`` is its ctypes binding and ``build`` compiles it.
"""
from . import hdg  # noqa: F401
