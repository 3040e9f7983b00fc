"""ctypes access to libne_probe.so (include/ne_probe.h), the instruction-rate
probe built beside libne.so for the benchmark's roofline denominators."""
import ctypes

_lib = None


def probe_lib():
    global _lib
    if _lib is None:
        from paper_1509_03838_gb300 import build
        build.build()
        L = ctypes.CDLL(build.PROBE_LIB)
        L.ne_probe_imad_rate.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
        L.ne_probe_imad_rate.restype = ctypes.c_int32
        _lib = L
    return _lib


def probe_rate(kind: int, iters: int):
    """(instructions per second, launch ms) of probe `kind`; raises on a
    non-zero status."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    st = probe_lib().ne_probe_imad_rate(kind, iters, ctypes.byref(rate),
                                        ctypes.byref(ms))
    if st != 0:
        raise RuntimeError(f"ne_probe_imad_rate({kind}, {iters}): status {st}")
    return rate.value, ms.value
