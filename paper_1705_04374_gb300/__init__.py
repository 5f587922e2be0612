"""GB300 (sm_103a) implementation of the hot path of optimal-fidelity MLMC for
cloud cavitation collapse (Sukys et al. 2017).

The compute path lives in ``libofmlmc.so`` (CUDA kernels + C ABI, declared in
include/ofmlmc.h).  ``native`` is the ctypes binding with the header's names,
``api`` a thin Python front end.  Importing ``native`` functions raises if the
library has not been built: there is no CPU fallback.
"""
from . import native  # noqa: F401

__all__ = ["native", "api"]
