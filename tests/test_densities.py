"""The Sec. 5 densities: rho must equal -Laplace(u*) for the stated exact solutions u*.
The printed bump (Sec. 5.3) and oscillating (Sec. 5.5) densities do not; the generators
use the re-derived ones, checked here symbolically (sympy) and numerically."""
import math

import numpy as np
import pytest

from paper_1612_01799_gb300 import densities as D


def _neg_laplacian_radial(u_expr, r):
    import sympy as sp
    return sp.simplify(-(sp.diff(u_expr, r, 2) + 2 / r * sp.diff(u_expr, r)))


def test_bump_density_is_minus_laplacian():
    sp = pytest.importorskip("sympy")
    r, d, R = sp.symbols("r d R", positive=True)
    u = sp.exp(-d * R ** 2 / (R ** 2 - r ** 2))
    rho = _neg_laplacian_radial(u, r)
    ours = 2 * d * R ** 2 * (3 * R ** 4 - 2 * R ** 2 * r ** 2 - r ** 4 - 2 * d * R ** 2 * r ** 2) / (R ** 2 - r ** 2) ** 4 * u
    assert sp.simplify(rho - ours) == 0
    # The printed variant (-d R^2 r^2 in the numerator) is not the Laplacian.
    printed_num = 3 * R ** 4 - 2 * R ** 2 * r ** 2 - r ** 4 - d * R ** 2 * r ** 2
    printed = 2 * d * R ** 2 * printed_num / (R ** 2 - r ** 2) ** 4 * u
    assert sp.simplify(rho - printed) != 0
    # And the sampler matches the symbolic density.
    f = sp.lambdify((r, d, R), ours, "numpy")
    N, L = 12, 3.0
    x = D.axis(N, L)
    rr = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    got = D.paper_bump(N, L, 10.0, 2.0)
    m = rr < 2.0
    assert np.allclose(got[m], f(rr[m], 10.0, 2.0), rtol=1e-12, atol=0)
    assert np.all(got[~m] == 0)


def test_oscillating_density_is_minus_laplacian():
    sp = pytest.importorskip("sympy")
    r, s, w = sp.symbols("r sigma omega", positive=True)
    u = sp.exp(-r ** 2 / s ** 2) * sp.cos(w * r ** 2)
    rho = _neg_laplacian_radial(u, r)
    f = sp.lambdify((r, s, w), rho, "numpy")
    N, L = 10, 2.0
    x = D.axis(N, L)
    rr = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    assert np.allclose(D.paper_oscillating(N, L, 0.3, 20.0), f(rr, 0.3, 20.0), rtol=1e-10, atol=1e-9)


def test_aniso_density_is_minus_laplacian():
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("x y z", real=True)
    sg = (0.3, 0.2, 0.28)
    u = sp.exp(-X ** 2 / sg[0] ** 2 - Y ** 2 / sg[1] ** 2 - Z ** 2 / sg[2] ** 2)
    rho = -(sp.diff(u, X, 2) + sp.diff(u, Y, 2) + sp.diff(u, Z, 2))
    f = sp.lambdify((X, Y, Z), rho, "numpy")
    N, L = 8, 1.0
    x = D.axis(N, L)
    got = D.paper_aniso(N, L, sg)
    ref = f(x[None, None, :], x[None, :, None], x[:, None, None])
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_gaussian_sum_sampler_charge():
    """A normalised Gaussian well inside the box carries its charge: h^3 sum rho = q."""
    g = D.GaussianSum(np.array([[0.5, -0.3, 0.2]]), np.array([[0.8, 1.1, 0.9]]), np.array([-0.7]))
    N, L = 64, 8.0
    rho = g.sample(N, L)
    assert abs(rho.sum() * (2 * L / N) ** 3 - (-0.7)) <= 1e-12


def test_workloads_are_seeded():
    a, b = D.config_aniso4(N=16), D.config_aniso4(N=16)
    assert np.array_equal(a.sample(), b.sample())
    assert abs(a.gaussians.charges.sum()) >= 0.1
    batch = D.config_batch()
    assert len(batch) == 64 and {w.N for w in batch} <= set(D.BATCH_SIZES)
