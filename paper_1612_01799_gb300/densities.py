"""Seeded synthetic densities on the solver's grid.

This module only samples inputs.  It holds none of the solver's arithmetic and imports
neither the CUDA library nor the oracle, so the tests can feed the same arrays to both.

Grid: the cube [-L, L]^3 with N cell-centred points per axis,
x_i = -L + (i + 1/2) * 2L/N, arrays indexed [z, y, x] (x fastest).

Workloads (shapes and value distributions of the paper's Sec. 5 test densities:
smooth, fast-decaying Gaussians and compact bumps):

* ``gaussian_iso``      normalised isotropic Gaussian (Sec. 5.1).
* ``gaussian_sum``      sum of normalised anisotropic Gaussians with charges q_g.
* ``poly_bump``         (1 - r^2/R^2)^4 on r < R.
* ``config_*``          the seeded parameter sets of the benchmark and parity workloads.
* ``paper_*``           the Sec. 5 densities, with the printed formulas of the bump
                        (Sec. 5.3) and the oscillating density (Sec. 5.5) replaced by
                        -Laplace(u*) of their stated exact solutions, because the printed
                        ones do not satisfy -Laplace(u*) = rho.
"""
from dataclasses import dataclass, field
import math
from typing import List

import numpy as np


def axis(N: int, L: float) -> np.ndarray:
    h = 2.0 * L / N
    return -L + (np.arange(N, dtype=np.float64) + 0.5) * h


@dataclass
class GaussianSum:
    """rho = sum_g q_g prod_q (2 pi s_gq^2)^{-1/2} exp(-(x_q - c_gq)^2 / (2 s_gq^2))."""
    centres: np.ndarray      # (G, 3) ordered (x, y, z)
    sigmas: np.ndarray       # (G, 3)
    charges: np.ndarray      # (G,)

    def sample(self, N: int, L: float, dtype=np.float64) -> np.ndarray:
        x = axis(N, L)
        rho = np.zeros((N, N, N), dtype=np.float64)
        for c, s, q in zip(self.centres, self.sigmas, self.charges):
            g = [np.exp(-np.square(x - c[a]) / (2.0 * s[a] ** 2)) / math.sqrt(2.0 * math.pi * s[a] ** 2)
                 for a in range(3)]
            rho += q * (g[2][:, None, None] * (g[1][:, None] * g[0][None, :])[None, :, :])
        return rho.astype(dtype, copy=False)


@dataclass
class Workload:
    name: str
    N: int
    L: float
    gaussians: GaussianSum
    bump_R: float = 0.0          # > 0: add (1 - r^2/R^2)^4 on r < R
    params: dict = field(default_factory=dict)

    def sample(self, dtype=np.float64) -> np.ndarray:
        rho = self.gaussians.sample(self.N, self.L)
        if self.bump_R > 0.0:
            rho += poly_bump(self.N, self.L, self.bump_R)
        return rho.astype(dtype, copy=False)


def gaussian_iso(N: int, L: float, sigma: float, centre=(0.0, 0.0, 0.0), Q: float = 1.0,
                 dtype=np.float64) -> np.ndarray:
    g = GaussianSum(np.array([centre], dtype=np.float64), np.full((1, 3), float(sigma)),
                    np.array([Q], dtype=np.float64))
    return g.sample(N, L, dtype)


def poly_bump(N: int, L: float, R: float) -> np.ndarray:
    x = axis(N, L)
    r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    t = np.clip(1.0 - r2 / R ** 2, 0.0, None)
    return t ** 4


def _draw_gaussians(rng, count, centre_lo, centre_hi, sigma_lo, sigma_hi, log_sigma=False,
                    iso=False, min_net=0.1):
    """Centres U[lo, hi]^3, widths U[sigma_lo, sigma_hi] (log-uniform if asked), charges
    U[-1, 1], redrawn until |sum q| >= min_net (so the net charge is not near zero)."""
    while True:
        c = rng.uniform(centre_lo, centre_hi, size=(count, 3))
        shape = (count, 1) if iso else (count, 3)
        if log_sigma:
            s = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), size=shape))
        else:
            s = rng.uniform(sigma_lo, sigma_hi, size=shape)
        s = np.broadcast_to(s, (count, 3)).copy()
        q = rng.uniform(-1.0, 1.0, size=count)
        if abs(q.sum()) >= min_net:
            return GaussianSum(c, s, q)


def config_single_gaussian() -> Workload:
    """Isotropic normalised Gaussian, sigma = 1, Q = 1, box [-8, 8]^3, N = 32."""
    g = GaussianSum(np.zeros((1, 3)), np.ones((1, 3)), np.ones(1))
    return Workload("gaussian_sigma1_N32", 32, 8.0, g, params={"sigma": 1.0})


def config_aniso4(N: int = 256, seed: int = 2) -> Workload:
    """4 anisotropic normalised Gaussians: centres U[-3,3]^3, widths U[0.5,1.5] per axis,
    charges U[-1,1] (|net| >= 0.1), box [-10, 10]^3."""
    rng = np.random.default_rng(seed)
    g = _draw_gaussians(rng, 4, -3.0, 3.0, 0.5, 1.5)
    return Workload("aniso4_N%d" % N, N, 10.0, g, params={"seed": seed})


def config_bump8(N: int = 512, seed: int = 3) -> Workload:
    """(1 - r^2/16)^4 on r < 4 plus 8 isotropic Gaussians (widths U[0.3, 1], charges
    U[-1, 1], centres U[-1.5, 1.5]^3), box [-6, 6]^3."""
    rng = np.random.default_rng(seed)
    g = _draw_gaussians(rng, 8, -1.5, 1.5, 0.3, 1.0, iso=True, min_net=0.0)
    return Workload("bump8_N%d" % N, N, 6.0, g, bump_R=4.0, params={"seed": seed, "R": 4.0})


BATCH_SIZES = (64, 96, 128, 160, 192)


def config_batch(count: int = 64, seed: int = 4, sizes=BATCH_SIZES) -> List[Workload]:
    """count densities, N uniform over sizes, each 1-6 anisotropic Gaussians drawn as in
    config_aniso4, box [-10, 10]^3."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.choice(sizes))
        k = int(rng.integers(1, 7))
        g = _draw_gaussians(rng, k, -3.0, 3.0, 0.5, 1.5)
        out.append(Workload("batch%d_N%d" % (i, N), N, 10.0, g, params={"seed": seed, "i": i}))
    return out


def config_selector(index: int, seed: int = 5, N: int = 64) -> Workload:
    """Density `index` of the selector set: 1-8 Gaussians, widths log-uniform [0.2, 2],
    charges U[-1, 1], centres U[-2, 2]^3, box [-16, 16]^3."""
    rng = np.random.default_rng([seed, index])
    k = int(rng.integers(1, 9))
    g = _draw_gaussians(rng, k, -2.0, 2.0, 0.2, 2.0, log_sigma=True, min_net=0.0)
    return Workload("selector%d" % index, N, 16.0, g, params={"seed": seed, "index": index})


# ---- Sec. 5 test densities ------------------------------------------------------------

def paper_two_gaussians(N: int, lo, hi, d=(0.1, -0.05, 0.05), s1=0.2, s2=0.1) -> np.ndarray:
    """Sec. 5.2: half the sum of normalised Gaussians at c + d (sigma1) and c - d (sigma2),
    c the box centre, on the box [lo, hi] (per-axis bounds; cube only here)."""
    c = 0.5 * (np.asarray(lo) + np.asarray(hi))
    L = 0.5 * (hi[0] - lo[0])
    g = GaussianSum(np.array([c + np.asarray(d), c - np.asarray(d)]),
                    np.array([[s1] * 3, [s2] * 3]), np.array([0.5, 0.5]))
    return g.sample(N, L)


def paper_bump(N: int, L: float, d: float, R: float) -> np.ndarray:
    """Sec. 5.3 density, as -Laplace of u* = exp(-d R^2/(R^2 - r^2)) on r < R:
    rho = 2 d R^2 (3R^4 - 2R^2 r^2 - r^4 - 2 d R^2 r^2) / (R^2 - r^2)^4 * u*."""
    x = axis(N, L)
    r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    out = np.zeros_like(r2)
    m = r2 < R * R
    a = R * R - r2[m]
    out[m] = (2.0 * d * R * R * (3 * R ** 4 - 2 * R * R * r2[m] - r2[m] ** 2 - 2 * d * R * R * r2[m])
              / a ** 4 * np.exp(-d * R * R / a))
    return out


def paper_aniso(N: int, L: float, sigma, c=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Sec. 5.4 density (as printed), -Laplace of exp(-sum (x_q - c_q)^2 / sigma_q^2)."""
    x = axis(N, L)
    X = [x - c[0], x - c[1], x - c[2]]
    e = [np.exp(-X[a] ** 2 / sigma[a] ** 2) for a in range(3)]
    p = [4.0 * X[a] ** 2 / sigma[a] ** 4 - 2.0 / sigma[a] ** 2 for a in range(3)]
    E = e[2][:, None, None] * e[1][None, :, None] * e[0][None, None, :]
    P = p[2][:, None, None] + p[1][None, :, None] + p[0][None, None, :]
    return -P * E


def paper_oscillating(N: int, L: float, sigma: float, omega: float) -> np.ndarray:
    """Sec. 5.5 density, as -Laplace of u* = e^{-r^2/sigma^2} cos(omega r^2) (the printed
    formula has the 4 omega^2 r^2 cos term with the wrong sign)."""
    x = axis(N, L)
    g = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    e = np.exp(-g / sigma ** 2)
    cs, sn = np.cos(omega * g), np.sin(omega * g)
    return (e * (6 * omega * sn + 4 * omega ** 2 * g * cs)
            - (4 * g / sigma ** 4 - 6 / sigma ** 2) * e * cs
            - 8 * omega * g / sigma ** 2 * e * sn)
