"""GB300 (sm_103a) phase-field WMRT lattice Boltzmann library.

The CUDA kernels live in ``csrc/`` and are built in-tree into
``_build/liblbm.so`` (``build.build()``); ``lbm`` is the ctypes binding of the
C ABI declared in ``include/lbm.h``.
"""
from . import build  # noqa: F401
