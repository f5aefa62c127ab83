"""Pins of the oracle's own FFT (oracle/fft.c): the O(n^2) DFT for every transform length the
library's grids use (2N for every supported N, the unpadded N of the correction's
Laplacian, the 32-point selector sample) and for lengths with other prime factors;
Parseval; impulses and plane waves; inversion; Hermitian symmetry of real input; the
three-axis zero-padded transform against the DFT applied axis by axis; and scipy's FFT as
an outside cross-check."""
import math

import numpy as np
import pytest

from oracle import fft


def five_smooth(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


# 2N for N = 4 ... 1024 with 2N 5-smooth, and lengths with primes 7, 11 and 13.
PADDED = [2 * n for n in range(4, 1025) if five_smooth(2 * n)]
OTHER = [1, 2, 3, 5, 7, 9, 11, 15, 25, 27, 49, 77, 143, 169, 210]


def dft(x):
    """The defining O(n^2) sum, each phase reduced mod n before the exponential."""
    n = x.shape[-1]
    j = np.arange(n)
    D = np.exp(-2j * math.pi * (np.outer(j, j) % n) / n)
    return x @ D.T


def rand_c(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n", PADDED[::7] + [8, 16, 24, 96, 128, 192, 256, 320, 324, 384, 512, 1024, 2048] + OTHER)
def test_against_direct_dft(n):
    x = rand_c((3, n), n)
    X = np.stack([fft.fft(v) for v in x])
    ref = dft(x)
    err = np.abs(X - ref).max() / np.abs(ref).max()
    assert err < 4e-15 * max(1.0, math.log2(max(n, 2))), (n, err)


def test_every_padded_length_against_direct_dft():
    """All 2N with 4 <= N <= 1024 and 2N 5-smooth, one random vector each."""
    worst = 0.0
    for n in PADDED:
        x = rand_c(n, 1000 + n)
        ref = dft(x)
        worst = max(worst, np.abs(fft.fft(x) - ref).max() / np.abs(ref).max())
    assert worst < 5e-14, worst


@pytest.mark.parametrize("n", [8, 30, 162, 324, 1000, 2048])
def test_parseval_and_inversion(n):
    x = rand_c(n, 7 * n)
    X = fft.fft(x)
    assert abs(np.vdot(X, X).real / n - np.vdot(x, x).real) <= 1e-13 * np.vdot(x, x).real
    assert np.abs(fft.ifft(X) - x).max() <= 1e-14 * np.abs(x).max() * math.log2(n)


@pytest.mark.parametrize("n", [12, 64, 250, 486])
def test_impulse_and_plane_wave(n):
    """An impulse at j0 gives the plane wave exp(-2 pi i j0 k / n); the plane wave of
    frequency k0 gives n at k0 and zero elsewhere."""
    k = np.arange(n)
    for j0 in (0, 1, n // 3, n - 1):
        x = np.zeros(n, complex)
        x[j0] = 1.0
        np.testing.assert_allclose(fft.fft(x), np.exp(-2j * math.pi * ((j0 * k) % n) / n), atol=1e-15)
    for k0 in (0, 1, n // 2, n - 2):
        x = np.exp(2j * math.pi * ((k0 * k) % n) / n)
        X = fft.fft(x)
        spike = np.zeros(n, complex)
        spike[k0] = n
        np.testing.assert_allclose(X, spike, atol=1e-12 * n)


def test_real_input_is_hermitian():
    n = 360
    x = np.random.default_rng(3).standard_normal(n)
    X = fft.fft(x)
    idx = (-np.arange(n)) % n
    np.testing.assert_allclose(X[idx], np.conj(X), atol=1e-13)


def test_padded_three_axis_transform_against_dft_per_axis():
    """fftn(x, s) with x (5, 6, 7) zero padded to (10, 12, 14): the DFT applied axis by axis."""
    x = np.random.default_rng(4).standard_normal((5, 6, 7))
    s = (10, 12, 14)
    P = np.zeros(s)
    P[:5, :6, :7] = x
    ref = P.astype(complex)
    for ax in range(3):
        ref = np.moveaxis(dft(np.moveaxis(ref, ax, -1)), -1, ax)
    got = fft.fftn(x, s=s)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    back = fft.ifftn(got)
    assert np.abs(back[:5, :6, :7] - x).max() < 1e-14
    assert np.abs(back[5:, :, :]).max() < 1e-14


def test_matches_library_fft_as_outside_check():
    sfft = pytest.importorskip("scipy.fft")
    x = np.random.default_rng(5).standard_normal((12, 20, 18))
    s = (24, 40, 36)
    ref = sfft.fftn(x, s=s)
    assert np.abs(fft.fftn(x, s=s) - ref).max() < 1e-13 * np.abs(ref).max()


def test_factors_and_bad_lengths():
    assert fft.factors(2048) == [2] * 11
    assert fft.factors(324) == [3, 3, 3, 3, 2, 2]
    assert fft.factors(1500) == [5, 5, 5, 3, 2, 2]
    assert fft.factors(143) == [11, 13]
    with pytest.raises(ValueError):
        fft.transform_axis(np.zeros((4, 4), np.float64), 0, -1)


def test_planted_wrong_twiddle_sign_is_caught():
    """Conjugating the forward transform (a sign slip in the twiddles) fails the DFT pin."""
    x = rand_c(48, 11)
    wrong = np.conj(fft.fft(np.conj(x)))          # the inverse (unnormalised) transform
    assert np.abs(wrong - dft(x)).max() > 1.0
