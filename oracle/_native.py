"""Build and load the oracle's C parts (TEST INFRASTRUCTURE ONLY).

gk_table.c (the Gauss-Kronrod quadrature of the G-tensor factors) and fft.c (the oracle's
own FFT) are compiled with the host gcc into oracle/_gk_table.so and oracle/_fft.so next
to them, with OpenMP.  No compiler flag is machine specific, so the same sources build on
x86_64 and aarch64 hosts.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_PARTS = {
    "gk": (os.path.join(_HERE, "gk_table.c"), os.path.join(_HERE, "_gk_table.so")),
    "fft": (os.path.join(_HERE, "fft.c"), os.path.join(_HERE, "_fft.so")),
}
_lock = threading.Lock()
_libs = {}


def _build_one(src: str, out: str, force: bool) -> str:
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile every C part whose shared object is missing or older than its source."""
    for src, out in _PARTS.values():
        _build_one(src, out, force)
    return _PARTS["gk"][1]


def _load(name: str):
    with _lock:
        if name not in _libs:
            src, out = _PARTS[name]
            h = ctypes.CDLL(_build_one(src, out, False))
            if name == "gk":
                h.oracle_a_table.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_void_p]
                h.oracle_a_table.restype = ctypes.c_long
                h.oracle_gk15_monomial.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                   ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(ctypes.c_double)]
                h.oracle_gk15_monomial.restype = None
            else:
                h.oracle_fft_axis.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_long,
                                              ctypes.c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int]
                h.oracle_fft_axis.restype = ctypes.c_int
                h.oracle_fft_factors.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                 ctypes.c_int]
                h.oracle_fft_factors.restype = ctypes.c_int
            _libs[name] = h
    return _libs[name]


def lib():
    """The Gauss-Kronrod quadrature library."""
    return _load("gk")


def fft_lib():
    """The FFT library."""
    return _load("fft")
