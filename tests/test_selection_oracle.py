"""Pins of the grid-selection oracle: MLP backprop against central differences, features
and the spectral tail on inputs whose answer is known."""
import math

import numpy as np

from oracle import selection as S


def test_mlp_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    K = 5
    p = rng.normal(scale=0.3, size=S.nparams(K))
    x = rng.normal(size=(7, 64))
    t = rng.normal(size=(7, K))
    g = S.mlp_backward(p, K, x, t)
    h = 1e-6
    for i in rng.choice(p.size, size=60, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        num = (S.mse(S.mlp_forward(p + e, K, x)[0], t) - S.mse(S.mlp_forward(p - e, K, x)[0], t)) / (2 * h)
        assert abs(num - g[i]) <= 1e-7 + 1e-6 * abs(num), i


def test_features_of_a_constant_and_a_plane_wave():
    f = S.features32(np.ones(32 ** 3))
    assert f[0] == 0.0 and np.all(f[1:] == -30.0)
    x = np.arange(32)
    k0 = 5
    wave = 1.0 + np.cos(2 * np.pi * k0 * x / 32)[None, None, :] * np.ones((32, 32, 1))
    f = S.features32(wave)
    b = min(int(k0 / (16 * math.sqrt(3)) * 64), 63)
    # the two modes (+-k0, 0, 0) carry power 1/4 of the mean at k = 0; the shell's mean
    # divides it among all the shell's modes
    assert -4.0 < f[b] < -1.0
    others = [i for i in range(64) if i not in (0, b)]
    assert np.all(f[others] <= -29.0)                # round-off power only


def test_spectral_tail_limits():
    rng = np.random.default_rng(1)
    N = 16
    noise = rng.standard_normal((N, N, N))
    frac = 1 - (1 - 1 / 8) ** 3                     # shell share of the padded frequencies
    assert abs(S.spectral_tail(noise) ** 2 - frac) < 0.08
    # a Gaussian resolved by the grid (sigma = 2.7 h) and negligible at the box edge
    N = 32
    x = (np.arange(N) + 0.5) / N * 12 - 6
    g = np.exp(-(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2) / 2)
    assert S.spectral_tail(g) < 1e-6
