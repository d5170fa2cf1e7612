"""Binding of the roofline probe library (include/ht_probe.h, built as
_build/libht_probe.so): microbenchmarks the benchmark measures kernels
against.  Not part of libht."""
import ctypes

import torch

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build_probe())
        L.ht_probe_shared_atomic_rate.restype = ctypes.c_int32
        L.ht_probe_shared_atomic_rate.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.c_void_p]
        _lib = L
    return _lib


def shared_atomic_rate(iters=4096, stream=None):
    """Conflict-free shared-memory atomicAdd throughput of the current GPU
    (atomics per second, whole GPU)."""
    v = ctypes.c_double()
    s = torch.cuda.current_stream() if stream is None else stream
    st = lib().ht_probe_shared_atomic_rate(int(iters), ctypes.byref(v),
                                           ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise RuntimeError(f"ht_probe_shared_atomic_rate failed (status {st})")
    return v.value
