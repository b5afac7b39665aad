"""GB300 (sm_103a) implementation of the D2Q9 T2S2-FDLBM time step of
arXiv 1911.12913: CUDA kernels behind the C ABI of ``include/fdlbm.h``, with a
thin Python binding.

``FDLBM`` (in ``solver``) needs PyTorch with CUDA for device memory and streams;
``binding`` alone loads the C library with ctypes.
"""
from .binding import FdlbmError, load  # noqa: F401


def __getattr__(name):
    if name in ("FDLBM", "FDLBMBatch"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
