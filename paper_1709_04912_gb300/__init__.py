"""GB300-native TV-superiorized conjugate gradient for parallel-beam CT.

The compute path is ``libscg.so`` (hand-written CUDA for sm_103a behind a C
ABI, declared in ``include/scg.h``); :mod:`.scg` is a thin ctypes binding
with the same entry-point names.  :mod:`.inputs` draws the seeded synthetic
workloads.  Nothing here falls back to the CPU: if the CUDA library is
missing, every call raises.
"""
from . import inputs  # noqa: F401
