"""Oracle: the discrete convolution in real space (TEST INFRASTRUCTURE ONLY).

The FFT solve of Sec. 2/3 computes, for outputs m in [0, N)^3,

    u_m = lambda^2 sum_{m' in [0,N)^3} K_{m - m'} rho_{m'},
    K_d = (2N)^-3 sum_{k in [-N, N)^3} G_tot(k) exp(2 pi i k.d / (2N)),

because the zero padding makes the cyclic convolution of length 2N exact for
|m_q - m'_q| < N.  Every term of G_tot is a product over the axes (the Gaussian sum is
separable and |kappa|^2 is a sum), so K_d = sum_j w_j a_j(d_x) a_j(d_y) a_j(d_z)
+ C0 [d = 0] - C2 sum_q l(d_q) [d_other = 0], with 1-D kernels

    a_j(d) = (2N)^-1 sum_{k=-N}^{N-1} A_j(|k|) exp(2 pi i k d / (2N)),
    l(d)   = (2N)^-1 sum_{k=-N}^{N-1} (pi k / 2)^2 exp(2 pi i k d / (2N)).

This module evaluates that sum directly, with explicit phases and no FFT.  One output
line (fixed y, z; all x) costs (S+1) N^3 multiply-adds, done as a matrix product.
It serves two purposes: sampled outputs of grids too large for the FFT oracle, and a
brute-force check of the FFT oracle's padding, index map, crop and normalisation.
"""
import math

import numpy as np

from .gtensor import OraclePlan


def kernel_1d(plan: OraclePlan) -> np.ndarray:
    """a[j, d + N - 1] = a_j(d) for d = -(N-1)..(N-1), by the explicit cosine sum."""
    N = plan.N
    M = 2 * N
    d = np.arange(-(N - 1), N, dtype=np.float64)
    k = np.arange(-N, N, dtype=np.float64)
    phase = np.exp(2j * math.pi * np.outer(k, d) / M)              # (2N, 2N-1)
    Ak = plan.A[:, np.abs(k).astype(int)]                           # (S+1, 2N)
    return np.real(Ak @ phase) / M


def laplace_1d(N: int) -> np.ndarray:
    """l[d + N - 1] = l(d) for d = -(N-1)..(N-1)."""
    M = 2 * N
    d = np.arange(-(N - 1), N, dtype=np.float64)
    k = np.arange(-N, N, dtype=np.float64)
    phase = np.exp(2j * math.pi * np.outer(k, d) / M)
    return np.real(((0.5 * math.pi * k) ** 2) @ phase) / M


def sample_lines(rho: np.ndarray, plan: OraclePlan, lines) -> np.ndarray:
    """u[z, y, :] for each (z, y) in lines; rho is indexed [z, y, x]."""
    rho = np.asarray(rho, dtype=np.float64)
    N = plan.N
    a = kernel_1d(plan)                      # (S+1, 2N-1)
    lap = laplace_1d(N)
    w = plan.gs.w
    idx = np.arange(N)
    out = np.empty((len(lines), N), dtype=np.float64)
    by_z = {}
    for n, (z, y) in enumerate(lines):
        by_z.setdefault(int(z), []).append((n, int(y)))
    flat = rho.reshape(N, N * N)
    kx = a[:, idx[:, None] - idx[None, :] + N - 1] * w[:, None, None]   # (S+1, x, x')
    lapx = lap[idx[:, None] - idx[None, :] + N - 1]
    for z, items in by_z.items():
        kz = a[:, z - idx + N - 1]                                  # (S+1, N) over z'
        r1 = (kz @ flat).reshape(-1, N, N)                          # (S+1, y', x')
        for n, y in items:
            ky = a[:, y - idx + N - 1]                              # (S+1, N) over y'
            r2 = np.einsum("jy,jyx->jx", ky, r1)                    # (S+1, x')
            i1 = np.einsum("jxk,jk->x", kx, r2)
            # Near-zone terms: C0 rho_m - C2 sum_q (l * rho)_m along each axis.
            line = rho[z, y, :]
            lx = lapx @ line
            ly = lap[y - idx + N - 1] @ rho[z, :, :]
            lz = lap[z - idx + N - 1] @ rho[:, y, :]
            out[n] = plan.lam ** 2 * (i1 + plan.C0 * line - plan.C2 * (lx + ly + lz))
    return out


def brute_force(rho: np.ndarray, plan: OraclePlan) -> np.ndarray:
    """All N^3 outputs by the explicit triple sum with the full 3-D kernel (tiny N only)."""
    rho = np.asarray(rho, dtype=np.float64)
    N = plan.N
    if N > 12:
        raise ValueError("brute force is for N <= 12")
    a = kernel_1d(plan)
    lap = laplace_1d(N)
    w = plan.gs.w
    D = 2 * N - 1
    # K[dz, dy, dx] over d in [-(N-1), N-1]^3.
    K = np.einsum("j,jz,jy,jx->zyx", w, a, a, a)
    c = N - 1
    K[c, c, c] += plan.C0
    K[:, c, c] -= plan.C2 * lap
    K[c, :, c] -= plan.C2 * lap
    K[c, c, :] -= plan.C2 * lap
    u = np.zeros((N, N, N))
    for mz in range(N):
        for my in range(N):
            for mx in range(N):
                sub = K[mz - np.arange(N) + c][:, my - np.arange(N) + c][:, :, mx - np.arange(N) + c]
                u[mz, my, mx] = np.sum(sub * rho)
    assert K.shape == (D, D, D)
    return plan.lam ** 2 * u
