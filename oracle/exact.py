"""Closed-form potentials used to pin the oracle (TEST INFRASTRUCTURE ONLY).

Each function returns u = U * rho for a density that the tests sample with the input
generators.  None of them uses the method under test.

* Isotropic normalised Gaussian of charge Q (Sec. 5.1):  Q erf(r/(sqrt2 sigma))/(4 pi r).
* Anisotropic normalised Gaussian (centre c, widths sigma_q, charge Q): from
  1/(4 pi r) = (1/(2 pi^{3/2})) int_0^inf exp(-r^2 s^2) ds and the 1-D Gaussian
  convolution of exp(-(x-y)^2 s^2) with N(c_q, sigma_q^2),
      u(x) = Q/(2 pi^{3/2}) int_0^inf prod_q (1 + 2 sigma_q^2 s^2)^{-1/2}
                 exp(-sum_q (x_q - c_q)^2 s^2 / (1 + 2 sigma_q^2 s^2)) ds,
  done by composite Gauss-Legendre quadrature after s = v / (1 - v).
* Radial polynomial bump (1 - r^2/R^2)^4 on r < R: for a radial density
  u(r) = (1/r) int_0^r rho s^2 ds + int_r^R rho s ds, both polynomial integrals.
* Sec. 5 test potentials that the paper prescribes: the bump e^{-d/(1 - r^2/R^2)}, the
  anisotropic Gaussian e^{-sum (x_q - c_q)^2 / sigma_q^2} and the oscillating
  e^{-r^2/sigma^2} cos(omega r^2) are the exact solutions themselves.
"""
import math

import numpy as np
from scipy.special import erf


def gaussian_iso(r, sigma, Q=1.0):
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    small = r < 1e-8 * sigma
    rs = r[~small]
    out[~small] = Q * erf(rs / (math.sqrt(2.0) * sigma)) / (4.0 * math.pi * rs)
    out[small] = Q / (4.0 * math.pi) * math.sqrt(2.0 / math.pi) / sigma
    return out


def _gl_panels(n_panels=48, order=24):
    """Nodes and weights of composite Gauss-Legendre on v in [0, 1), panels graded
    towards both ends (geometric in v and in 1 - v)."""
    xg, wg = np.polynomial.legendre.leggauss(order)
    half = n_panels // 2
    edges_lo = np.concatenate([[0.0], 0.5 * np.geomspace(1e-7, 1.0, half)])
    edges_hi = 1.0 - edges_lo[::-1]
    edges = np.unique(np.concatenate([edges_lo, edges_hi]))
    nodes, weights = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        nodes.append(0.5 * (b - a) * xg + 0.5 * (a + b))
        weights.append(0.5 * (b - a) * wg)
    return np.concatenate(nodes), np.concatenate(weights)


def gaussian_aniso(points, centre, sigma, Q=1.0, chunk=4096):
    """Potential of Q * prod_q N(c_q, sigma_q^2) at points (P, 3) ordered (x, y, z)."""
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    c = np.asarray(centre, dtype=np.float64)
    sg = np.asarray(sigma, dtype=np.float64)
    v, wv = _gl_panels()
    s = v / (1.0 - v)
    ds = wv / (1.0 - v) ** 2
    den = 1.0 + 2.0 * np.square(sg)[None, :] * np.square(s)[:, None]       # (V, 3)
    pref = ds / np.sqrt(np.prod(den, axis=1))                              # (V,)
    fac = np.square(s)[:, None] / den                                      # (V, 3)
    out = np.empty(pts.shape[0])
    for i in range(0, pts.shape[0], chunk):
        d2 = np.square(pts[i:i + chunk] - c[None, :])                      # (P, 3)
        expo = d2 @ fac.T                                                   # (P, V)
        out[i:i + chunk] = np.exp(-expo) @ pref
    return Q * out / (2.0 * math.pi ** 1.5)


def poly_bump_radial(r, R):
    """Potential of (1 - r^2/R^2)^4 (r < R), zero outside."""
    r = np.asarray(r, dtype=np.float64)
    c = [math.comb(4, i) * (-1.0) ** i / R ** (2 * i) for i in range(5)]   # coefficients of r^{2i}
    out = np.empty_like(r)
    inside = r < R
    ri = r[inside]
    inner = sum(ci * ri ** (2 * i + 2) / (2 * i + 3) for i, ci in enumerate(c))   # (1/r) int_0^r rho s^2
    outer = sum(ci * (R ** (2 * i + 2) - ri ** (2 * i + 2)) / (2 * i + 2) for i, ci in enumerate(c))
    out[inside] = inner + outer
    ro = r[~inside]
    total = sum(ci * R ** (2 * i + 3) / (2 * i + 3) for i, ci in enumerate(c))   # int_0^R rho s^2
    out[~inside] = total / ro
    return out


def bump_exp(r, d, R):
    """Sec. 5.3 exact solution e^{-d/(1 - r^2/R^2)} for r < R, zero outside."""
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros_like(r)
    m = r < R
    out[m] = np.exp(-d / (1.0 - np.square(r[m] / R)))
    return out


def aniso_exp(x, y, z, c, sigma):
    """Sec. 5.4 exact solution exp(-sum_q (x_q - c_q)^2 / sigma_q^2)."""
    return np.exp(-(x - c[0]) ** 2 / sigma[0] ** 2 - (y - c[1]) ** 2 / sigma[1] ** 2
                  - (z - c[2]) ** 2 / sigma[2] ** 2)


def oscillating(r, sigma, omega):
    """Sec. 5.5 exact solution e^{-r^2/sigma^2} cos(omega r^2)."""
    r2 = np.square(np.asarray(r, dtype=np.float64))
    return np.exp(-r2 / sigma ** 2) * np.cos(omega * r2)
