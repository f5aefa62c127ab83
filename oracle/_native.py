"""Build and load the oracle's C quadrature (TEST INFRASTRUCTURE ONLY).

gk_table.c is compiled with the host gcc into oracle/_gk_table.so next to it, with
OpenMP over the Gaussian-sum terms.  No compiler flag is machine specific, so the same
source builds on x86_64 and aarch64 hosts.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gk_table.c")
_LIB = os.path.join(_HERE, "_gk_table.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gk_table.c if the shared object is missing or older than the source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            h = ctypes.CDLL(build())
            h.oracle_a_table.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_void_p]
            h.oracle_a_table.restype = ctypes.c_long
            h.oracle_gk15_monomial.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double)]
            h.oracle_gk15_monomial.restype = None
            _lib = h
    return _lib
