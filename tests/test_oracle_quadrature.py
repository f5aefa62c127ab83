"""Pins of the oracle's setup phase: quadrature rule, G-tensor factors, Gaussian sum,
near-zone constants.  Each is checked against something other than the oracle itself:
polynomial exactness, a library special function (Faddeeva), arbitrary-precision
quadrature (mpmath), or the defining integral."""
import ctypes
import math

import numpy as np
import pytest
from scipy.special import erf, wofz

from oracle import _native, gauss_sum, gtensor


def test_gk15_rule_exactness():
    """K15 integrates degree <= 22 exactly and G7 degree <= 13 (and not 14): this pins
    every stored abscissa and weight of the G7/K15 pair."""
    lib = _native.lib()
    k, g = ctypes.c_double(), ctypes.c_double()
    for p in range(0, 23):
        lib.oracle_gk15_monomial(p, -0.3, 1.7, ctypes.byref(k), ctypes.byref(g))
        exact = (1.7 ** (p + 1) - (-0.3) ** (p + 1)) / (p + 1)
        assert abs(k.value - exact) <= 1e-14 * max(1.0, abs(exact)), p
        if p <= 13:
            assert abs(g.value - exact) <= 1e-14 * max(1.0, abs(exact)), p
    lib.oracle_gk15_monomial(14, -1.0, 1.0, ctypes.byref(k), ctypes.byref(g))
    assert abs(g.value - 2.0 / 15.0) > 1e-6


def faddeeva_a(tau, kmax):
    """A_j(k) = (sqrt(pi)/tau) Re[e^{-a^2} - e^{-b^2 - 2iab} w(-a + ib)], a = kappa/(2 tau),
    b = 2 tau: the integral written with the Faddeeva function w (scipy)."""
    kap = 0.5 * np.pi * np.arange(kmax + 1)
    a = kap[None, :] / (2 * tau[:, None])
    b = 2 * tau[:, None]
    return (np.sqrt(np.pi) / tau[:, None]) * np.real(np.exp(-a * a) - np.exp(-b * b - 2j * a * b) * wofz(-a + 1j * b))


@pytest.mark.parametrize("N", [8, 64, 200])
def test_a_table_matches_faddeeva(N):
    gs = gauss_sum.gauss_sum(1e-13, 1e-3, 2 * math.sqrt(3))
    A = gtensor.a_table(gs.tau, N)
    ref = faddeeva_a(gs.tau, N)
    # k = 0 from the erf form (the Faddeeva form cancels there for tiny tau).
    ref[:, 0] = np.sqrt(np.pi) * erf(2 * gs.tau) / gs.tau
    assert np.max(np.abs(A - ref)) <= 1e-13


def test_a_table_closed_form_limits():
    """Large tau: the Gaussian has left [0, 2], A = (sqrt(pi)/tau) exp(-kappa^2/(4 tau^2)).
    tau -> 0: A(0) = 4 and A(k != 0) = 4 sin(pi k)/(pi k) = 0."""
    tau = np.array([6.0, 40.0, 1e-9])
    A = gtensor.a_table(tau, 40)
    kap = 0.5 * np.pi * np.arange(41)
    for i in range(2):
        ref = np.sqrt(np.pi) / tau[i] * np.exp(-kap ** 2 / (4 * tau[i] ** 2))
        assert np.max(np.abs(A[i] - ref)) <= 1e-15 * np.sqrt(np.pi) / tau[i]
    assert abs(A[2, 0] - 4.0) <= 1e-14
    assert np.max(np.abs(A[2, 1:])) <= 1e-14


def test_a_table_matches_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    tau = np.array([np.exp(-5.15), np.exp(-0.5), 1.0, 2.7])
    ks = [0, 3, 77, 244]
    A = gtensor.a_table(tau, max(ks))
    for i, t in enumerate(tau):
        T = mp.mpf(t)
        for k in ks:
            kap = mp.pi * k / 2
            ref = 2 * mp.quad(lambda s: mp.exp(-T * T * s * s) * mp.cos(kap * s),
                              mp.linspace(0, 2, k + 2))
            assert abs(A[i, k] - float(ref)) <= 1e-13, (t, k)


@pytest.mark.parametrize("eps,delta", [(1e-7, 1e-3), (1e-10, 5e-3), (1e-13, 1e-2), (1e-14, 1e-3)])
def test_gauss_sum_relative_error(eps, delta):
    """max |4 pi r U_GS(r) - 1| <= eps on [delta, 2 sqrt 3], checked on a grid 12x denser
    than the construction's and at random radii."""
    r_max = 2 * math.sqrt(3)
    gs = gauss_sum.gauss_sum(eps, delta, r_max)
    dense = np.geomspace(delta, r_max, 50000)
    rnd = np.exp(np.random.default_rng(0).uniform(math.log(delta), math.log(r_max), 20000))
    assert gauss_sum.relative_error(gs.tau, gs.w, dense).max() <= 1.05 * eps
    assert gauss_sum.relative_error(gs.tau, gs.w, rnd).max() <= 1.05 * eps
    # Below delta the sum stays finite: U_GS(0) = sum w_j.
    assert np.isfinite(gs.w.sum())


def test_gauss_sum_more_terms_is_better():
    r_max = 2 * math.sqrt(3)
    errs = [gauss_sum.gauss_sum(e, 1e-3, r_max) for e in (1e-6, 1e-9, 1e-12)]
    assert len(errs[0].tau) < len(errs[1].tau) < len(errs[2].tau)
    r = np.geomspace(1e-3, r_max, 4096)
    m = [gauss_sum.relative_error(g.tau, g.w, r).max() for g in errs]
    assert m[0] > m[1] > m[2]


def test_eps_and_delta_readings():
    assert gauss_sum.eps_from_tol(1e-6) == pytest.approx(1e-7)
    assert gauss_sum.eps_from_tol(1e-20) == 1e-14
    assert gauss_sum.eps_from_tol(1.0) == 1e-7
    # Sec. 3: min_q (b_q - a_q)/(50 n_q), floored at 1e-3.
    assert gauss_sum.near_zone_delta([-8] * 3, [8] * 3, [32] * 3) == pytest.approx(0.01)
    assert gauss_sum.near_zone_delta([-6] * 3, [6] * 3, [512] * 3) == 1e-3


def test_correction_constants_match_definition():
    """C0 = int_{B_delta} (U - U_GS), C2 = (1/6) int_{B_delta} (U - U_GS)|y|^2, by mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for eps, delta in [(1e-13, 1e-2), (1e-7, 1e-3), (1e-10, 0.3)]:
        gs = gauss_sum.gauss_sum(eps, delta, 2 * math.sqrt(3))
        c0, c2 = gtensor.correction_constants(gs, delta)
        taus = [mp.mpf(t) for t in gs.tau]
        ws = [mp.mpf(w) for w in gs.w]

        def diff(r):
            return 1 / (4 * mp.pi * r) - mp.fsum(w * mp.exp(-t * t * r * r) for t, w in zip(taus, ws))
        pts = mp.linspace(0, delta, 9)
        ref0 = 4 * mp.pi * mp.quad(lambda r: diff(r) * r * r, pts)
        ref2 = 4 * mp.pi * mp.quad(lambda r: diff(r) * r ** 4, pts) / 6
        assert abs(c0 - float(ref0)) <= 1e-12 * abs(float(ref0)), (eps, delta)
        assert abs(c2 - float(ref2)) <= 1e-10 * abs(float(ref2)), (eps, delta)
