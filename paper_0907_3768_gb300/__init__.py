"""libdust: GB300-native dust-grain equilibrium temperatures and IR emission.

The compute path lives in the CUDA library built from csrc/ (C ABI in
include/dust.h); this package is its thin Python binding.
"""
from ._lib import (  # noqa: F401
    DUST_FLAG_HIGH,
    DUST_FLAG_INVALID,
    DUST_FLAG_LOW,
    DUST_FLAG_OK,
    DUST_PREC_BF16X3,
    DUST_PREC_FP16X3,
    DUST_PREC_FP32,
    DustError,
    PRECISIONS,
    header_functions,
    lib,
)


def __getattr__(name):
    # the torch-facing front end is imported lazily so that the ctypes layer
    # stays usable without touching CUDA
    if name in ("Context", "Server", "padded_rows"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
