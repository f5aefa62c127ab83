"""GPU kernels of the a-posteriori check and the grid selector against the oracle: the
density sampler, exact potentials, FP64 comparisons, the spectral-tail indicator, the
power-spectrum features, and the MLP forward / backward / Adam; then a small end-to-end
training run through the selector file and poisson_select_n."""
import ctypes
import math
import os

import numpy as np
import pytest

from oracle import exact, selection as OS
from paper_1612_01799_gb300 import densities as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01799_gb300 import _lib, build
    build.build()
    return torch, _lib.load()


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def params_of(g):
    from paper_1612_01799_gb300.selector import gaussian_params
    return gaussian_params(g)


def test_sampler_matches_generator(env):
    torch, lib = env
    g = D._draw_gaussians(np.random.default_rng(3), 5, -2, 2, 0.4, 1.5)
    N, L = 40, 6.0
    P = params_of(g)
    ref = g.sample(N, L)
    for code, dt, tol in ((1, torch.float64, 1e-13), (0, torch.float32, 2e-6)):
        out = torch.empty(N ** 3, dtype=dt, device="cuda")
        assert lib.poisson_sample_gaussians(N, L, P.shape[0], P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            code, ptr(out), None) == 0
        got = out.cpu().numpy().reshape(N, N, N)
        assert np.max(np.abs(got - ref)) <= tol * np.abs(ref).max()


def test_exact_potential_matches_oracle(env):
    torch, lib = env
    g = D._draw_gaussians(np.random.default_rng(4), 3, -2, 2, 0.3, 2.0)
    N, L = 64, 16.0
    P = params_of(g)
    idx = np.random.default_rng(5).integers(0, N, size=(300, 3)).astype(np.int32)
    idx_d = torch.from_numpy(idx.ravel()).cuda()
    out = torch.empty(300, dtype=torch.float64, device="cuda")
    assert lib.poisson_gaussian_potential(N, L, P.shape[0], P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          300, ptr(idx_d), ptr(out), None) == 0
    x = D.axis(N, L)
    pts = np.stack([x[idx[:, 0]], x[idx[:, 1]], x[idx[:, 2]]], axis=1)
    ref = sum(exact.gaussian_aniso(pts, c, s, q) for c, s, q in zip(g.centres, g.sigmas, g.charges))
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-11 * np.abs(ref).max()


def test_compare_kernels(env):
    torch, lib = env
    rng = np.random.default_rng(6)
    b = rng.standard_normal(100003)
    a = b + 1e-3 * rng.standard_normal(b.size)
    ad = torch.from_numpy(a.astype(np.float32)).cuda()
    bd = torch.from_numpy(b).cuda()
    l2, li = ctypes.c_double(), ctypes.c_double()
    assert lib.poisson_compare(ptr(ad), 0, ptr(bd), 1, b.size, ctypes.byref(l2), ctypes.byref(li), None) == 0
    a32 = a.astype(np.float32).astype(np.float64)
    assert l2.value == pytest.approx(np.linalg.norm(a32 - b) / np.linalg.norm(b), rel=1e-12)
    assert li.value == pytest.approx(np.abs(a32 - b).max() / np.abs(b).max(), rel=1e-12)
    N = 16
    u = rng.standard_normal(N ** 3)
    idx = rng.integers(0, N, size=(50, 3)).astype(np.int32)
    ref = rng.standard_normal(50)
    ud, id_, rd = torch.from_numpy(u).cuda(), torch.from_numpy(idx.ravel()).cuda(), torch.from_numpy(ref).cuda()
    assert lib.poisson_compare_points(ptr(ud), 1, N, 50, ptr(id_), ptr(rd), ctypes.byref(l2), None) == 0
    got = u.reshape(N, N, N)[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert l2.value == pytest.approx(np.linalg.norm(got - ref) / np.linalg.norm(ref), rel=1e-12)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_checked_solve(env, dtype):
    """Same potential as poisson_solve, and eta as defined on the padded spectrum."""
    torch, lib = env
    from paper_1612_01799_gb300 import Plan
    for N, L, seed in ((64, 10.0, 21), (48, 3.0, 22), (8, 4.0, 23)):
        rho = D.config_aniso4(N=N, seed=seed).gaussians.sample(N, L)
        with Plan(N, L, 1e-6, dtype) as p:
            t = torch.from_numpy(rho.astype(p.np_dtype)).cuda()
            u1 = p.solve(t)
            u2 = torch.empty_like(t)
            eta = ctypes.c_double()
            assert lib.poisson_solve_checked(p.handle, ptr(t), ptr(u2), ctypes.byref(eta), None) == 0
            torch.cuda.synchronize()
            assert torch.equal(u1, u2)
        ref = OS.spectral_tail(rho.astype(np.float32 if dtype == "f32" else np.float64))
        assert eta.value == pytest.approx(ref, rel=2e-3 if dtype == "f32" else 1e-6, abs=1e-12)


def test_features_kernel(env):
    torch, lib = env
    rng = np.random.default_rng(7)
    samples = [D.config_selector(i, N=32).sample(np.float32) for i in range(6)]
    samples.append(rng.standard_normal((32, 32, 32)).astype(np.float32))
    s = torch.from_numpy(np.stack(samples).ravel()).cuda()
    f = torch.empty(len(samples) * 64, dtype=torch.float32, device="cuda")
    assert lib.poisson_features32(ptr(s), len(samples), ptr(f), None) == 0
    got = f.cpu().numpy().reshape(len(samples), 64)
    for i, smp in enumerate(samples):
        ref = OS.features32(smp)
        m = ref > -9.0                       # bins above the FP32 round-off floor
        assert np.max(np.abs(got[i][m] - ref[m])) <= 2e-3, i


def test_mlp_kernels_against_oracle(env):
    torch, lib = env
    from paper_1612_01799_gb300.selector import Network
    K = 12
    rng = np.random.default_rng(8)
    net = Network(K, seed=3)
    B = 37
    x = rng.standard_normal((B, 64)).astype(np.float32)
    t = rng.standard_normal((B, K)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t.ravel()).cuda()
    p = net.params.cpu().numpy().astype(np.float64)
    y = net.forward(xd).cpu().numpy()
    yref, _ = OS.mlp_forward(p, K, x.astype(np.float64))
    assert np.max(np.abs(y - yref)) <= 1e-5 * (1 + np.abs(yref).max())
    loss = net.gradient(xd, td)
    torch.cuda.synchronize()
    assert loss.item() == pytest.approx(OS.mse(yref, t), rel=1e-5)
    gref = OS.mlp_backward(p, K, x.astype(np.float64), t.astype(np.float64))
    g = net.grad.cpu().numpy()
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
    # one Adam step from zero moments: p - lr * sign-like update g / (|g| + eps')
    before = net.params.clone()
    lr = 1e-3
    assert lib.poisson_mlp_adam(ptr(net.params), ptr(net.grad), ptr(net.m), ptr(net.v), net.n, ctypes.c_float(lr),
                                ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-8), 1, None) == 0
    gg = net.grad.double()
    expect = before.double() - lr * gg / (gg.abs() + 1e-8)
    assert torch.allclose(net.params.double(), expect, rtol=0, atol=2e-7)


def test_selector_end_to_end_small(env, tmp_path):
    torch, lib = env
    from paper_1612_01799_gb300 import selector as S
    ws = S.Workspace(candidates=(32, 64, 128))
    try:
        path = str(tmp_path / "sel.bin")
        info = S.fit(list(range(24)), ws, path, epochs=600, lr=3e-3)
        assert info["losses"][-1] < 0.1 * info["losses"][0]
        sel = S.Selector(path, capacity=32)
        params = [S.gaussian_params(S.density(i)) for i in range(24, 32)]
        _, s32 = ws.features(params)
        Ns, pred = sel.select(s32, len(params), 1e-6)
        goal = math.log10(1e-6) - 0.3
        for n, row in zip(Ns, pred):
            ok = [k for k in range(3) if row[k] <= goal]
            assert n == (ws.candidates[ok[0]] if ok else ws.candidates[-1])
        # The batched refinement ends where the one-at-a-time refinement ends.
        starts = [ws.candidates.index(n) for n in Ns]
        batched = S.solve_batched_until_checked(ws, sel, params, starts, 1e-6)
        single = [S._solve_until_checked(ws, sel, p, k, 1e-6) for p, k in zip(params, starts)]
        assert batched == single
        sel.close()
    finally:
        ws.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_checked_batched_equals_checked_singles(env, dtype):
    """poisson_solve_checked_batched: each density's potential and eta as its own checked solve."""
    torch, lib = env
    from paper_1612_01799_gb300 import Plan
    N, L = 48, 4.0
    rhos = [D.config_aniso4(N=N, seed=s).gaussians.sample(N, L) for s in (31, 32, 33)]
    with Plan(N, L, 1e-6, dtype, max_batch=3) as p:
        ts = [torch.from_numpy(r.astype(p.np_dtype)).cuda() for r in rhos]
        us = [torch.empty_like(t) for t in ts]
        rp = (ctypes.c_void_p * 3)(*[t.data_ptr() for t in ts])
        up = (ctypes.c_void_p * 3)(*[u.data_ptr() for u in us])
        eta = (ctypes.c_double * 3)()
        assert lib.poisson_solve_checked_batched(p.handle, 3, rp, up, eta, None) == 0
        assert lib.poisson_solve_checked_batched(p.handle, 4, rp, up, eta, None) == -1   # above max_batch
        for t, u, e in zip(ts, us, eta):
            u1 = torch.empty_like(t)
            e1 = ctypes.c_double()
            assert lib.poisson_solve_checked(p.handle, ptr(t), ptr(u1), ctypes.byref(e1), None) == 0
            torch.cuda.synchronize()
            assert torch.equal(u, u1)
            assert e == pytest.approx(e1.value, rel=1e-12)
