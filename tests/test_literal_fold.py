"""The paper's literal near-field correction (Sec. 2: I_delta = C0 rho + C2 Laplace(rho), the
Laplacian from an unpadded N^3 transform pair) and the folded form the CUDA path uses for
it (POISSON_KNOB_CORRECTION = 1): the N-point DFT of rho is the zero-padded 2N-point DFT at
even frequencies, so 8 (C0 - C2 |kappa|^2) at the all-even padded frequencies, added to the
Gaussian-sum symbol, gives the same potential on the kept N^3 points.  These CPU tests pin
the oracle's spectral Laplacian to plane waves and the folding to the oracle's literal
solve, and check that the two correction placements differ enough for the GPU parity
tests to tell them apart."""
import numpy as np
import pytest
import scipy.fft as sfft

from oracle import gtensor, solver


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
    spec = sfft.fftn(rho, s=(M, M, M)) * G
    return plan.lam ** 2 * sfft.ifftn(spec).real[:N, :N, :N]


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
