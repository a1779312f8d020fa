"""GB300 (sm_103a) dual messenger Wiener filter for joint T/Q/U CMB maps on the
HEALPix sphere (Kodi Ramanah, Lavaux & Wandelt, arXiv:1801.05358).

The compute path is the CUDA library libdmwf (csrc/, C ABI in include/dmwf.h);
``dmwf`` is its ctypes binding."""
from . import dmwf  # noqa: F401
from .dmwf import DM_FP64, DM_MIXED_FP32, DmError, Plan  # noqa: F401
