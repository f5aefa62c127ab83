"""Oracle: Gaussian-sum approximation of the Newton kernel (TEST INFRASTRUCTURE ONLY).

Sec. 2 (eq. approx) replaces U(y) = 1/(4 pi |y|) on |y| in [delta, 2] by
U_GS(y) = sum_{j=0}^{S} w_j exp(-tau_j^2 |y|^2), obtained by sinc quadrature.  The paper
cites the construction but does not print it.  The reading used here:

    1/(4 pi r) = 1/(2 pi^{3/2}) * integral_R exp(-r^2 e^{2s} + s) ds

(from 1/r = (2/sqrt(pi)) int_0^inf exp(-r^2 t^2) dt with t = e^s), discretised by the
trapezoid rule on the grid s_j = j h, so tau_j = e^{s_j} and w_j = h e^{s_j}/(2 pi^{3/2}).

* Range.  The sum runs over every grid node in [s_lo, s_hi] widened to the grid: the
  lower tail cut at t_lo = e^{s_lo} changes 4 pi r U by at most erf(r t_lo) <=
  2 r t_lo / sqrt(pi), set to eps/4 at r = r_max; the upper cut at t_hi changes it by
  erfc(r t_hi) <= erfc(delta t_hi), set to eps/4.
* Step.  h runs down the ladder h = 2/m, m = 2, 3, ..., and the first h whose maximum
  of |4 pi r U_GS(r) - 1| over 4096 log-spaced r in [delta, r_max] is <= eps is taken.
* Fit range.  The paper states [delta, 2].  The convolution integral runs over
  2*B_{1,lambda}, whose points reach |y| = 2 |l|, 2 sqrt(3) for a cube, so the fit
  range here is [delta, 2 |l|].
* eps from the user tolerance: eps = clamp(tol / 10, 1e-14, 1e-7).  Sec. 3 puts the
  error of the approximations at max{eps, delta^6}; the tolerance is not mapped to eps
  in the paper.
* delta (Sec. 3 heuristic): min_q (b_q - a_q) / (50 n_q), at least 1e-3, read as the
  literal number in the scaled coordinates.  That reading is the one for which the
  paper's side condition delta < min_q l_q is the stated lambda <= 25 min_q n_q.
"""
from dataclasses import dataclass
import math

import numpy as np
from scipy.special import erfcinv

N_FIT = 4096


@dataclass(frozen=True)
class GaussSum:
    tau: np.ndarray      # (S+1,) exponent scales tau_j
    w: np.ndarray        # (S+1,) weights w_j
    h: float             # trapezoid step in s
    max_rel_err: float   # measured max |4 pi r U_GS - 1| on the fit grid
    delta: float
    r_max: float
    eps: float


def eps_from_tol(tol: float) -> float:
    """GS accuracy for a requested tolerance (reading: tol/10 clamped to [1e-14, 1e-7])."""
    return min(max(0.1 * float(tol), 1e-14), 1e-7)


def near_zone_delta(box_lo, box_hi, n) -> float:
    """delta of the Sec. 3 heuristic, min_q (b_q - a_q)/(50 n_q), floored at 1e-3."""
    d = min((float(b) - float(a)) / (50.0 * int(m)) for a, b, m in zip(box_lo, box_hi, n))
    return max(d, 1e-3)


def relative_error(tau, w, r):
    """|4 pi r U_GS(r) - 1| at the radii r."""
    r = np.asarray(r, dtype=np.float64)
    vals = np.exp(-np.square(r[:, None] * tau[None, :])) @ w
    return np.abs(4.0 * np.pi * r * vals - 1.0)


def gauss_sum(eps: float, delta: float, r_max: float) -> GaussSum:
    """Sinc-quadrature Gaussian sum with max relative error <= eps on [delta, r_max]."""
    t_lo = eps * math.sqrt(math.pi) / (8.0 * r_max)
    t_hi = float(erfcinv(eps / 4.0)) / delta
    s_lo, s_hi = math.log(t_lo), math.log(t_hi)
    r = np.geomspace(delta, r_max, N_FIT)
    for m in range(2, 4000):
        h = 2.0 / m
        j = np.arange(math.floor(s_lo / h), math.ceil(s_hi / h) + 1, dtype=np.float64)
        s = j * h
        tau = np.exp(s)
        w = h * np.exp(s) / (2.0 * math.pi ** 1.5)
        err = float(relative_error(tau, w, r).max())
        if err <= eps:
            return GaussSum(tau=tau, w=w, h=h, max_rel_err=err, delta=delta, r_max=r_max,
                            eps=eps)
    raise RuntimeError("no trapezoid step reaches the requested eps")
