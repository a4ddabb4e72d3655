"""ctypes binding of the measurement library libdpcs_probe.so (roof probes:
L2 load bandwidth and scattered float4 atomic throughput), used by the
benchmark and its tests; the same names as ``include/dpcs_probe.h``."""
from __future__ import annotations

import ctypes

from . import build as _build

_lib = None


class ProbeError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status}")
        self.status = status


def load_library():
    """Load libdpcs_probe.so, building it first if needed."""
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_probe())
        lib.dpcs_probe_l2_load.restype = ctypes.c_int32
        lib.dpcs_probe_l2_load.argtypes = [ctypes.c_int32, ctypes.c_size_t, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double)]
        lib.dpcs_probe_atomic4.restype = ctypes.c_int32
        lib.dpcs_probe_atomic4.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_double)]
        _lib = lib
    return _lib


def dpcs_probe_l2_load(device: int, nbytes: int = 32 << 20, passes: int = 64) -> float:
    """Measured L2 load bandwidth in GB/s (16-byte loads that bypass L1)."""
    out = ctypes.c_double()
    st = load_library().dpcs_probe_l2_load(int(device), int(nbytes), int(passes), ctypes.byref(out))
    if st != 0:
        raise ProbeError(st, "dpcs_probe_l2_load")
    return out.value


def dpcs_probe_atomic4(device: int, texels: int = 512 * 512, n_atomics: int = 1 << 28) -> float:
    """Measured scattered float4 atomic-add throughput in 1e9 adds per second."""
    out = ctypes.c_double()
    st = load_library().dpcs_probe_atomic4(int(device), int(texels), int(n_atomics), ctypes.byref(out))
    if st != 0:
        raise ProbeError(st, "dpcs_probe_atomic4")
    return out.value
