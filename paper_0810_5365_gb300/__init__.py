"""GB300-native Wilson-Dirac hopping operator and even-odd CG solver.

The compute lives in libwd (``csrc/``, CUDA for sm_103a, C ABI in
``include/wd.h``); ``wd`` is its ctypes binding (plus two helpers that
allocate packed buffers as torch byte tensors).  Building: ``python -m paper_0810_5365_gb300.build``.
"""
from . import wd  # noqa: F401
from .wd import *  # noqa: F401,F403
