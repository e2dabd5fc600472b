"""GB300-native improved random batch Ewald (RBL + RBE) force step.

``systems`` generates seeded synthetic inputs; ``rbe`` is the thin ctypes
binding of the C-ABI library ``librbe.so`` (CUDA kernels for sm_103a).
"""
from . import systems  # noqa: F401
