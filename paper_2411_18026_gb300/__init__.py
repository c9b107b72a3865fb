"""GB300-native fast direct solver for 2D elastic wave scattering by a cavity
(proxy-surface compression + LU-based Martinsson–Rokhlin variant, arXiv 2411.18026).

``fds`` holds the ctypes binding of the CUDA library ``libfds.so`` (C ABI in
``include/fds.h``); ``build`` compiles it for sm_103a.
"""
from . import build  # noqa: F401
