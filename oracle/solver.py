"""Oracle: the solve step (TEST INFRASTRUCTURE ONLY).

Sec. 2 and Sec. 3: u = lambda^2 (I_1 + I_delta).  I_1 is the convolution of the
density's finite Fourier series with U_GS, done by FFT with zero padding to twice the
length per axis; I_delta is the near-zone Taylor correction.

Normalisation (not printed in the paper; derived from Sec. 2).  On the padded period-4
scaled box the Fourier coefficients are rho_hat_k = DFT(P)_k / (2N)^3, where P is the
density zero padded to (2N)^3 with the data at indices 0..N-1 per axis, and
I_1(x_m) = sum_k rho_hat_k G_k exp(i kappa.(x_m - x_0)).  So, with the unnormalised
forward and 1/(2N)^3-normalised inverse transforms (the oracle's own FFT, ``fft``),

    u = lambda^2 * Re(IFFT(G_tot * FFT(P)))[0:N, 0:N, 0:N].

Arrays are indexed [z, y, x] (x fastest), the layout of the library's buffers.
"""
import numpy as np

from . import fft
from .gtensor import OraclePlan, make_plan, symbol


def solve(rho: np.ndarray, L: float, tol: float, plan: OraclePlan = None,
          correction: bool = True, G: np.ndarray = None) -> np.ndarray:
    """Potential of rho (N^3, FP64, cell-centred grid on [-L, L]^3), correction in the symbol.
    G: the padded symbol of this plan, if the caller already has it (several densities)."""
    rho = np.asarray(rho, dtype=np.float64)
    N = rho.shape[0]
    if rho.shape != (N, N, N):
        raise ValueError("rho must be N x N x N")
    if plan is None:
        plan = make_plan(N, L, tol)
    M = 2 * N
    if G is None:
        G = symbol(plan, correction=correction)
    spec = fft.fftn(rho, s=(M, M, M))
    spec *= G
    u = fft.ifftn(spec, overwrite=True)
    return plan.lam ** 2 * np.ascontiguousarray(u.real[:N, :N, :N])


def spectral_laplacian(rho: np.ndarray, L: float) -> np.ndarray:
    """Laplacian of the N-point (period 2 in scaled units) Fourier series of rho, in the
    scaled coordinates, by one forward and one inverse N^3 FFT (Sec. 2, last paragraph;
    Sec. 3 counts this FFT pair)."""
    N = rho.shape[0]
    idx = np.arange(N)
    k = np.where(idx < (N + 1) // 2, idx, idx - N)   # signed frequency of DFT index idx
    kap2 = (np.pi * k) ** 2                    # period 2: kappa = 2 pi k / 2
    lap = kap2[:, None, None] + kap2[None, :, None] + kap2[None, None, :]
    spec = fft.fftn(rho)
    spec *= -lap
    return np.ascontiguousarray(fft.ifftn(spec, overwrite=True).real)


def solve_literal_correction(rho: np.ndarray, L: float, tol: float,
                             plan: OraclePlan = None) -> np.ndarray:
    """The paper's literal order: I_1 by the padded FFT with G alone, then
    I_delta = C0 rho + C2 Laplace(rho) with the Laplacian from an unpadded FFT pair."""
    rho = np.asarray(rho, dtype=np.float64)
    N = rho.shape[0]
    if plan is None:
        plan = make_plan(N, L, tol)
    i1 = solve(rho, L, tol, plan=plan, correction=False) / plan.lam ** 2
    i_delta = plan.C0 * rho + plan.C2 * spectral_laplacian(rho, L)
    return plan.lam ** 2 * (i1 + i_delta)
