"""Oracle: the method on a general rectangular box (TEST INFRASTRUCTURE ONLY).

Sec. 2, standardised form.  The box B = [a_1, b_1] x [a_2, b_2] x [a_3, b_3] is moved to
its centre c and scaled by lambda = max_q (b_q - a_q) / 2 to B_{1,lambda} = [-l_1, l_1] x
[-l_2, l_2] x [-l_3, l_3], l_q = (b_q - a_q) / (2 lambda) <= 1; u = lambda^2 (I_1 + I_delta)
in the scaled coordinates.  Axis q carries n_q cell-centred points (spacing 2 l_q / n_q
scaled), zero-padded to 2 n_q, so the padded period along q is 4 l_q and the Fourier
variable of padded frequency k is kappa_q = pi k / (2 l_q).

G-tensor (Sec. 2): G_k = sum_j w_j prod_q A^q_j(k_q) with the factor printed there,
A^q_j(k) = int_0^2 2 l_q exp(-(tau_j l_q)^2 y^2) cos(pi k y / 2) dy, i.e. l_q times the
cube's factor at tau_j l_q, taken from the same adaptive Gauss-Kronrod routine.

The Gaussian sum is fitted on [delta, 2 |l|] (the radii that 2 B_{1,lambda} reaches), delta
is the Sec. 3 heuristic min_q (b_q - a_q) / (50 n_q) floored at 1e-3 and must lie below
min_q l_q, and C0, C2 are the cube's (they depend on delta and the Gaussian sum only).  On
the cube [-L, L]^3 every step reduces to gtensor.make_plan / gtensor.symbol / solver.solve.
"""
from dataclasses import dataclass
import math

import numpy as np

from . import fft
from .gauss_sum import GaussSum, eps_from_tol, gauss_sum, near_zone_delta
from .gtensor import a_table, correction_constants, signed_freq


@dataclass(frozen=True)
class BoxPlan:
    n: tuple             # (n_x, n_y, n_z) points per axis
    lo: tuple            # (a_1, a_2, a_3)
    hi: tuple            # (b_1, b_2, b_3)
    tol: float
    lam: float           # lambda = max_q (b_q - a_q) / 2
    l: tuple             # (l_1, l_2, l_3)
    delta: float
    eps: float
    gs: GaussSum
    A: tuple             # per axis (S+1, n_q+1): A^q_j(k), k = 0..n_q
    C0: float
    C2: float


def axis(plan: BoxPlan, q: int) -> np.ndarray:
    """Cell-centred physical coordinates of axis q (0 = x)."""
    a, b, m = plan.lo[q], plan.hi[q], plan.n[q]
    return a + (np.arange(m, dtype=np.float64) + 0.5) * ((b - a) / m)


def make_box_plan(n, lo, hi, tol: float) -> BoxPlan:
    """Setup phase (Sec. 3) on the box [lo, hi] with n points per axis (x, y, z order)."""
    n = tuple(int(v) for v in (n if np.ndim(n) else (n, n, n)))
    lo = tuple(float(v) for v in lo)
    hi = tuple(float(v) for v in hi)
    half = [0.5 * (b - a) for a, b in zip(lo, hi)]
    lam = max(half)
    l = tuple(h / lam for h in half)
    delta = near_zone_delta(lo, hi, n)
    if not delta < min(l):
        raise ValueError("delta must lie below min_q l_q (Sec. 3 side condition)")
    eps = eps_from_tol(tol)
    gs = gauss_sum(eps, delta, 2.0 * math.sqrt(sum(v * v for v in l)))
    A = tuple(lq * a_table(gs.tau * lq, nq) for lq, nq in zip(l, n))
    c0, c2 = correction_constants(gs, delta)
    return BoxPlan(n=n, lo=lo, hi=hi, tol=float(tol), lam=lam, l=l, delta=delta, eps=eps, gs=gs,
                   A=A, C0=c0, C2=c2)


def box_symbol(plan: BoxPlan, correction: bool = True) -> np.ndarray:
    """G_tot on the padded (2 n_z, 2 n_y, 2 n_x) grid (numpy's fftn index order)."""
    kx, ky, kz = (signed_freq(m) for m in plan.n)
    Ax, Ay, Az = (plan.A[q][:, np.abs(k)] for q, k in enumerate((kx, ky, kz)))
    S = Ax.shape[0]
    zy = (plan.gs.w[:, None, None] * Az[:, :, None] * Ay[:, None, :]).reshape(S, -1)
    G = (zy.T @ Ax).reshape(kz.size, ky.size, kx.size)
    if correction:
        kap2 = [(0.5 * math.pi * k.astype(np.float64) / lq) ** 2 for k, lq in zip((kx, ky, kz), plan.l)]
        G += plan.C0
        G -= plan.C2 * (kap2[2][:, None, None] + kap2[1][None, :, None] + kap2[0][None, None, :])
    return G


def solve_box(rho: np.ndarray, plan: BoxPlan, G: np.ndarray = None,
              correction: bool = True) -> np.ndarray:
    """Potential of rho (shape (n_z, n_y, n_x), FP64, cell-centred grid of the box), the
    correction folded into the padded symbol (or left out: correction=False)."""
    rho = np.asarray(rho, dtype=np.float64)
    nx, ny, nz = plan.n
    if rho.shape != (nz, ny, nx):
        raise ValueError("rho must have shape (n_z, n_y, n_x)")
    if G is None:
        G = box_symbol(plan, correction=correction)
    spec = fft.fftn(rho, s=(2 * nz, 2 * ny, 2 * nx))
    spec *= G
    u = fft.ifftn(spec, overwrite=True)
    return plan.lam ** 2 * np.ascontiguousarray(u.real[:nz, :ny, :nx])


def spectral_laplacian_box(rho: np.ndarray, plan: BoxPlan) -> np.ndarray:
    """Laplacian, in the scaled coordinates, of the finite Fourier series of rho on the
    unpadded grid (Sec. 2, last paragraph): axis q has n_q points over the period 2 l_q,
    so DFT index k of that axis has kappa_q = 2 pi k_s / (2 l_q) = pi k_s / l_q with k_s
    the signed frequency; one forward and one inverse n_x n_y n_z transform."""
    rho = np.asarray(rho, dtype=np.float64)
    kap2 = []
    for m, lq in zip(plan.n, plan.l):
        idx = np.arange(m)
        ks = np.where(idx < (m + 1) // 2, idx, idx - m).astype(np.float64)
        kap2.append((math.pi * ks / lq) ** 2)
    lap = kap2[2][:, None, None] + kap2[1][None, :, None] + kap2[0][None, None, :]
    spec = fft.fftn(rho)
    spec *= -lap
    return np.ascontiguousarray(fft.ifftn(spec, overwrite=True).real)


def solve_box_literal(rho: np.ndarray, plan: BoxPlan) -> np.ndarray:
    """The paper's literal order on a box (Sec. 2): I_1 by the padded transform with the
    Gaussian-sum G-tensor alone, then I_delta = C0 rho + C2 Laplace(rho) with the
    Laplacian from the unpadded transform pair; u = lambda^2 (I_1 + I_delta)."""
    rho = np.asarray(rho, dtype=np.float64)
    i1 = solve_box(rho, plan, correction=False) / plan.lam ** 2
    i_delta = plan.C0 * rho + plan.C2 * spectral_laplacian_box(rho, plan)
    return plan.lam ** 2 * (i1 + i_delta)
