"""Oracle for the grid-selection pieces (TEST INFRASTRUCTURE ONLY).

Plain FP64 definitions (transforms by the oracle's own FFT) that the tests hold the GPU
kernels to:

* ``spectral_tail``  -- eta = sqrt(E_shell / E_total) of the zero-padded (2N)^3 DFT of the
  density, E_shell the energy where max(|kx|, |ky|, |kz|) >= N - N/8 (signed frequencies of
  the padded grid).  The method's error is driven by how well the finite Fourier series
  resolves the density (Sec. 3); the tail energy measures that.
* ``features32``     -- the 32^3 sample's DFT power averaged over 64 radial shells of
  |k| in [0, 16 sqrt 3] (shell index floor(|k| / (16 sqrt 3) * 64), capped at 63), as
  log10(P_b / P_0 + 1e-30) clamped to [-30, 0].
* ``mlp_forward`` / ``mlp_backward`` -- the 64 -> 64 -> 64 -> 64 -> K ReLU network with the
  parameter layout W1 (64x64), b1, W2, b2, W3, b3, W4 (K x 64), b4 (W[j, i] multiplies input
  i into unit j), and the mean-squared-error loss mean((y - t)^2) over all outputs.
"""
import math

import numpy as np

from . import fft

H = 64


def spectral_tail(rho):
    N = rho.shape[0]
    M = 2 * N
    F = fft.fftn(np.asarray(rho, np.float64), s=(M, M, M))
    e = np.abs(F) ** 2
    k = np.abs(np.where(np.arange(M) < N, np.arange(M), np.arange(M) - M))
    kinf = np.maximum(np.maximum(k[:, None, None], k[None, :, None]), k[None, None, :])
    shell = kinf >= N - N // 8
    return math.sqrt(e[shell].sum() / e.sum())


def features32(sample):
    s = np.asarray(sample, np.float64).reshape(32, 32, 32)
    F = fft.fftn(s)
    p = np.abs(F) ** 2
    idx = np.arange(32)
    k = np.where(idx < 16, idx, idx - 32).astype(np.float64)   # signed frequency
    kr = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    b = np.minimum((kr / (16 * math.sqrt(3.0)) * 64).astype(int), 63)
    pw = np.bincount(b.ravel(), weights=p.ravel(), minlength=64)
    cnt = np.bincount(b.ravel(), minlength=64).astype(np.float64)
    mean = np.where(cnt > 0, pw / np.maximum(cnt, 1), 0.0)
    v = np.log10(mean / max(mean[0], 1e-300) + 1e-30)
    return np.clip(v, -30.0, 0.0)


def nparams(K):
    return 3 * (H * H + H) + K * H + K


def unpack(p, K):
    p = np.asarray(p, np.float64)
    out, o = [], 0
    for l in range(3):
        W = p[o:o + H * H].reshape(H, H)
        o += H * H
        b = p[o:o + H]
        o += H
        out.append((W, b))
    W = p[o:o + K * H].reshape(K, H)
    o += K * H
    out.append((W, p[o:o + K]))
    return out


def mlp_forward(p, K, x):
    layers = unpack(p, K)
    a = [np.asarray(x, np.float64)]
    for W, b in layers[:3]:
        a.append(np.maximum(a[-1] @ W.T + b, 0.0))
    W, b = layers[3]
    return a[-1] @ W.T + b, a


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def mlp_backward(p, K, x, t):
    """Gradient of mse(forward(x), t) with respect to the parameter vector."""
    y, a = mlp_forward(p, K, x)
    dy = 2.0 * (y - t) / y.size
    layers = unpack(p, K)
    grads = []
    W4, _ = layers[3]
    grads.append((dy.T @ a[3], dy.sum(0)))
    d = (dy @ W4) * (a[3] > 0)
    for l in (2, 1, 0):
        W, _ = layers[l]
        grads.append((d.T @ a[l], d.sum(0)))
        if l > 0:
            d = (d @ W) * (a[l] > 0)
    grads = grads[::-1]       # layers 0..3
    return np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
