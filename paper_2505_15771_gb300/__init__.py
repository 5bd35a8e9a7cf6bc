"""GB300-native ERK stage operator of the HHO elasto-acoustic scheme.

``hho`` is the ctypes binding of the C ABI in include/hho.h; ``solver`` is a
small convenience layer that keeps device buffers in torch tensors.
"""
from . import hho  # noqa: F401
