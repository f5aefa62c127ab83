"""Oracle: its own FP64 discrete Fourier transform (TEST INFRASTRUCTURE ONLY).

The zero-padded transforms of Sec. 2 (convolution theorem on the padded grid) and the
unpadded transform pair of the correction's Laplacian run through ``fft.c``: a recursive
mixed-radix (5, 3, 2, and any other prime as a direct step) Cooley-Tukey FFT in FP64,
full complex, no pruning, along one axis at a time.

* ``fftn(x, s)`` -- x zero padded to shape s (data at the low corner of every axis), then
  the unnormalised forward DFT along every axis: X[k] = sum_j x[j] exp(-2 pi i j.k / n).
* ``ifftn(X)``   -- the inverse DFT along every axis, normalised by 1 / prod(shape).
* ``fft(x)``, ``ifft(x)`` -- one-dimensional forms (the same code).

Nothing here calls a library FFT.
"""
import ctypes
import math
import os

import numpy as np

from . import _native


def threads() -> int:
    """Host threads the transforms use: ORACLE_THREADS if set, else every core."""
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


def _as3d(a: np.ndarray) -> np.ndarray:
    if a.ndim > 3 or a.ndim == 0:
        raise ValueError("1 to 3 axes")
    return a.reshape((1,) * (3 - a.ndim) + a.shape)


def transform_axis(a: np.ndarray, axis: int, sign: int) -> None:
    """In place: the unnormalised DFT (sign -1) or inverse DFT (sign +1) of every line of
    the complex128 C-contiguous array a along `axis`."""
    if a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise ValueError("complex128, C-contiguous")
    ax = axis % a.ndim
    b = _as3d(a)
    ax3 = ax + 3 - a.ndim
    rc = _native.fft_lib().oracle_fft_axis(b.ctypes.data, b.shape[0], b.shape[1], b.shape[2],
                                           ax3, int(sign), threads())
    if rc != 0:
        raise RuntimeError("oracle_fft_axis failed (%d)" % rc)


def fftn(x: np.ndarray, s=None) -> np.ndarray:
    """Forward DFT over every axis of x zero padded to shape s (default: x's shape)."""
    x = np.asarray(x)
    s = tuple(x.shape) if s is None else tuple(int(v) for v in s)
    if len(s) != x.ndim or any(a < b for a, b in zip(s, x.shape)):
        raise ValueError("s must have x's rank and be at least x's shape")
    out = np.zeros(s, dtype=np.complex128)
    out[tuple(slice(0, m) for m in x.shape)] = x
    for ax in range(out.ndim):
        transform_axis(out, ax, -1)
    return out


def ifftn(X: np.ndarray, overwrite: bool = False) -> np.ndarray:
    """Inverse DFT over every axis, normalised by 1 / (number of points).  overwrite: X
    (complex128, C-contiguous) may be transformed in place and returned."""
    if overwrite and X.dtype == np.complex128 and X.flags.c_contiguous and X.flags.writeable:
        out = X
    else:
        out = np.array(X, dtype=np.complex128, order="C", copy=True)
    for ax in range(out.ndim):
        transform_axis(out, ax, +1)
    out *= 1.0 / math.prod(out.shape)
    return out


def fft(x: np.ndarray) -> np.ndarray:
    """Forward DFT of a 1-D sequence."""
    return fftn(np.asarray(x).reshape(-1))


def ifft(X: np.ndarray) -> np.ndarray:
    """Inverse DFT of a 1-D sequence (normalised by 1 / n)."""
    return ifftn(np.asarray(X).reshape(-1))


def factors(n: int):
    """The radices of the length-n transform, outermost first."""
    buf = (ctypes.c_int * 64)()
    nf = _native.fft_lib().oracle_fft_factors(int(n), buf, 64)
    if nf < 0:
        raise ValueError("cannot factor %d" % n)
    return [buf[i] for i in range(nf)]
