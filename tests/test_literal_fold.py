"""The paper's literal near-field correction (Sec. 2: I_delta = C0 rho + C2 Laplace(rho), the
Laplacian from an unpadded N^3 transform pair) and the folded form the CUDA path uses for
it (POISSON_KNOB_CORRECTION = 1): the N-point DFT of rho is the zero-padded 2N-point DFT at
even frequencies, so 8 (C0 - C2 |kappa|^2) at the all-even padded frequencies, added to the
Gaussian-sum symbol, gives the same potential on the kept N^3 points.  These CPU tests pin
the oracle's spectral Laplacian to plane waves and the folding to the oracle's literal
solve, and check that the two correction placements differ enough for the GPU parity
tests to tell them apart."""
import math

import numpy as np
import pytest

from oracle import box as obox, fft, gtensor, solver


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def folded_solve(rho, plan, factor=8.0):
    """The literal correction placed in the padded symbol, written out from the reading above."""
    N = rho.shape[0]
    M = 2 * N
    k = gtensor.signed_freq(N)
    kap2 = (np.pi * k / 2.0) ** 2
    K2 = kap2[:, None, None] + kap2[None, :, None] + kap2[None, None, :]
    even = k % 2 == 0
    E = even[:, None, None] & even[None, :, None] & even[None, None, :]
    G = gtensor.symbol(plan, correction=False) + np.where(E, factor * (plan.C0 - plan.C2 * K2), 0.0)
    spec = fft.fftn(rho, s=(M, M, M)) * G
    return plan.lam ** 2 * fft.ifftn(spec).real[:N, :N, :N]


def densities(N, seed=1):
    rng = np.random.default_rng(seed)
    noise = rng.uniform(-1.0, 1.0, (N, N, N))
    checker = np.fromfunction(lambda i, j, l: (-1.0) ** (i + j + l), (N, N, N))
    return {"noise": noise, "checker": checker}


@pytest.mark.parametrize("N", [6, 8, 9, 12])
def test_spectral_laplacian_plane_waves(N):
    """cos(pi k x) on the period-2 scaled grid is an eigenfunction: Laplace = -(pi k)^2 (three axes)."""
    x = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
    for k in range(0, (N - 1) // 2 + 1):
        for axis in range(3):
            shape = [1, 1, 1]
            shape[axis] = N
            f = np.broadcast_to(np.cos(np.pi * k * x).reshape(shape), (N, N, N)).copy()
            lap = solver.spectral_laplacian(f, 1.0)
            np.testing.assert_allclose(lap, -(np.pi * k) ** 2 * f, atol=1e-11 * max(1.0, (np.pi * k) ** 2))


@pytest.mark.parametrize("N,L", [(8, 8.0), (9, 8.0), (12, 6.0), (16, 8.0)])
def test_folded_symbol_equals_literal_transform_pair(N, L):
    plan = gtensor.make_plan(N, L, 1e-10)
    for name, rho in densities(N).items():
        lit = solver.solve_literal_correction(rho, L, 1e-10, plan=plan)
        assert rel_l2(folded_solve(rho, plan), lit) < 1e-14, name


@pytest.mark.parametrize("N,L", [(8, 8.0), (16, 8.0)])
def test_fused_and_literal_placements_differ(N, L):
    """Far above the FP64 parity tolerance (1e-12) for densities with high frequencies."""
    plan = gtensor.make_plan(N, L, 1e-10)
    for name, rho in densities(N).items():
        lit = solver.solve_literal_correction(rho, L, 1e-10, plan=plan)
        fused = solver.solve(rho, L, 1e-10, plan=plan)
        assert rel_l2(fused, lit) > 1e-9, name


def test_planted_missing_factor_8_is_caught():
    """Dropping the 8 (the unpadded 1/N^3 against the padded 1/(2N)^3) must fail the pin."""
    N, L = 8, 8.0
    plan = gtensor.make_plan(N, L, 1e-10)
    rho = densities(N)["noise"]
    lit = solver.solve_literal_correction(rho, L, 1e-10, plan=plan)
    assert rel_l2(folded_solve(rho, plan, factor=1.0), lit) > 1e-9


def folded_box_solve(rho, plan, factor=8.0):
    """The same reading on a box: 8 (C0 - C2 |kappa|^2) at the padded frequencies whose three
    indices are all even, kappa_q = pi k / (2 l_q) per axis."""
    nx, ny, nz = plan.n
    ks = [gtensor.signed_freq(m) for m in (nx, ny, nz)]
    kap2 = [(0.5 * math.pi * k / lq) ** 2 for k, lq in zip(ks, plan.l)]
    ev = [k % 2 == 0 for k in ks]
    E = ev[2][:, None, None] & ev[1][None, :, None] & ev[0][None, None, :]
    K2 = kap2[2][:, None, None] + kap2[1][None, :, None] + kap2[0][None, None, :]
    G = obox.box_symbol(plan, correction=False) + np.where(E, factor * (plan.C0 - plan.C2 * K2), 0.0)
    spec = fft.fftn(rho, s=(2 * nz, 2 * ny, 2 * nx)) * G
    return plan.lam ** 2 * fft.ifftn(spec).real[:nz, :ny, :nx]


@pytest.mark.parametrize("n", [(8, 8, 8), (8, 10, 12), (12, 9, 16)])
def test_box_folded_symbol_equals_box_literal_transform_pair(n):
    """On the box of Table 2 with n_q per axis: the folded placement against the oracle's
    literal box solve (its own unpadded transform pair with kappa_q = pi k / l_q)."""
    plan = obox.make_box_plan(n, (-3.0, -2.0, -1.0), (2.0, 3.5, 5.0), 1e-10)
    rng = np.random.default_rng(12)
    checker = np.fromfunction(lambda i, j, l: (-1.0) ** (i + j + l), (n[2], n[1], n[0]))
    for rho in (rng.uniform(-1, 1, (n[2], n[1], n[0])), checker):
        lit = obox.solve_box_literal(rho, plan)
        assert rel_l2(folded_box_solve(rho, plan), lit) < 1e-14
        assert rel_l2(folded_box_solve(rho, plan, factor=1.0), lit) > 1e-10
