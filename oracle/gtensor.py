"""Oracle: G-tensor factors, near-zone constants and the padded symbol (TEST INFRASTRUCTURE ONLY).

Geometry.  The box is the cube [-L, L]^3 with N points per axis.  Sec. 2 scales it by
lambda = L to B_{1,lambda} = [-1, 1]^3 (l_q = 1).  Reading of the grid: cell centred,
x_i = -L + (i + 1/2) 2L/N.  The paper's listing samples with linspace (both ends), but its
G-tensor formula has the padded period 4 l_q = 2 N h', i.e. spacing 2 l_q / N in the
scaled box; the symbol depends on the spacing only, and the offset only moves the
sample points.

G-tensor (Sec. 2): G_k = sum_j w_j prod_q A_j(k_q), A_j(k) = 2 int_0^2 e^{-tau_j^2 t^2}
cos(pi k t / 2) dt, computed by adaptive Gauss-Kronrod quadrature (gk_table.c).

Near zone (Sec. 2, correction integral I_delta): the third-order Taylor polynomial of
the density at x' leaves, after the odd terms and the off-diagonal Hessian cancel,
I_delta = C0 rho + C2 Laplace(rho) with

    C0 = int_{B_delta} (U - U_GS) dy
       = delta^2/2 - 4 pi sum_j w_j int_0^delta r^2 e^{-tau_j^2 r^2} dr,
    C2 = (1/6) int_{B_delta} (U - U_GS) |y|^2 dy
       = (1/6) [delta^4/4 - 4 pi sum_j w_j int_0^delta r^4 e^{-tau_j^2 r^2} dr],

the radial integrals done analytically (closed forms through erf, or their power
series when tau delta < 1/2, where the closed forms cancel).

Symbol.  With kappa_q = pi k_q / 2 (period 4 of the padded scaled box) the Laplacian is
-|kappa|^2, so the correction joins the symbol: G_tot(k) = G_k + C0 - C2 |kappa|^2.
"""
from dataclasses import dataclass
import math

import numpy as np
from scipy.special import erf

from . import _native
from .gauss_sum import GaussSum, eps_from_tol, gauss_sum, near_zone_delta

GK_RTOL = 1e-15


@dataclass(frozen=True)
class OraclePlan:
    N: int
    L: float
    tol: float
    lam: float           # lambda = L (cube)
    delta: float
    eps: float
    gs: GaussSum
    A: np.ndarray        # (S+1, N+1): A_j(k), k = 0..N
    C0: float
    C2: float


def a_table(tau: np.ndarray, kmax: int, rtol: float = GK_RTOL) -> np.ndarray:
    """A[j, k] = 2 int_0^2 exp(-tau_j^2 t^2) cos(pi k t / 2) dt for k = 0..kmax."""
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    out = np.empty((tau.size, kmax + 1), dtype=np.float64)
    _native.lib().oracle_a_table(tau.ctypes.data, int(tau.size), int(kmax), float(rtol),
                                 out.ctypes.data)
    return out


def _r2_gauss_integral(tau: float, d: float) -> float:
    """int_0^d r^2 exp(-tau^2 r^2) dr."""
    x = tau * d
    if x < 0.5:
        total, n, term = 0.0, 0, 1.0
        while True:
            t = ((-1.0) ** n) * (tau ** (2 * n)) * d ** (2 * n + 3) / (math.factorial(n) * (2 * n + 3))
            total += t
            if abs(t) <= 1e-20 * abs(total) or n > 60:
                return total
            n += 1
    return math.sqrt(math.pi) * math.erf(x) / (4.0 * tau ** 3) - d * math.exp(-x * x) / (2.0 * tau ** 2)


def _r4_gauss_integral(tau: float, d: float) -> float:
    """int_0^d r^4 exp(-tau^2 r^2) dr."""
    x = tau * d
    if x < 0.5:
        total, n = 0.0, 0
        while True:
            t = ((-1.0) ** n) * (tau ** (2 * n)) * d ** (2 * n + 5) / (math.factorial(n) * (2 * n + 5))
            total += t
            if abs(t) <= 1e-20 * abs(total) or n > 60:
                return total
            n += 1
    return (3.0 * math.sqrt(math.pi) * math.erf(x) / (8.0 * tau ** 5)
            - math.exp(-x * x) * (d ** 3 / (2.0 * tau ** 2) + 3.0 * d / (4.0 * tau ** 4)))


def correction_constants(gs: GaussSum, delta: float):
    """(C0, C2) of the near-zone Taylor correction for this Gaussian sum and delta."""
    s2 = sum(w * _r2_gauss_integral(t, delta) for t, w in zip(gs.tau, gs.w))
    s4 = sum(w * _r4_gauss_integral(t, delta) for t, w in zip(gs.tau, gs.w))
    c0 = 0.5 * delta ** 2 - 4.0 * math.pi * s2
    c2 = (0.25 * delta ** 4 - 4.0 * math.pi * s4) / 6.0
    return c0, c2


def make_plan(N: int, L: float, tol: float) -> OraclePlan:
    """Setup phase (Sec. 3): delta, eps, the Gaussian sum, the A table and C0, C2."""
    N = int(N)
    L = float(L)
    lam = L
    delta = near_zone_delta([-L] * 3, [L] * 3, [N] * 3)
    if not delta < 1.0:
        raise ValueError("delta must lie below min_q l_q = 1 (Sec. 3 side condition)")
    eps = eps_from_tol(tol)
    gs = gauss_sum(eps, delta, 2.0 * math.sqrt(3.0))
    A = a_table(gs.tau, N)
    c0, c2 = correction_constants(gs, delta)
    return OraclePlan(N=N, L=L, tol=float(tol), lam=lam, delta=delta, eps=eps, gs=gs, A=A,
                      C0=c0, C2=c2)


def signed_freq(N: int) -> np.ndarray:
    """Integer frequency k_q in {-N, ..., N-1} of each padded FFT index 0..2N-1."""
    M = 2 * N
    idx = np.arange(M)
    return np.where(idx < N, idx, idx - M)


def symbol(plan: OraclePlan, correction: bool = True) -> np.ndarray:
    """G_tot on the padded (2N)^3 FFT grid (index order of numpy's fftn)."""
    N = plan.N
    M = 2 * N
    k = signed_freq(N)
    Ak = plan.A[:, np.abs(k)]                         # (S+1, M): A_j(|k|)
    # sum_j w_j A_j(kz) A_j(ky) A_j(kx) as one matrix product over j.
    zy = (plan.gs.w[:, None, None] * Ak[:, :, None] * Ak[:, None, :]).reshape(Ak.shape[0], M * M)
    G = (zy.T @ Ak).reshape(M, M, M)
    if correction:
        kap2 = (0.5 * math.pi * k.astype(np.float64)) ** 2
        G += plan.C0
        G -= plan.C2 * (kap2[:, None, None] + kap2[None, :, None] + kap2[None, None, :])
    return G
