"""Both forms of the fused z pass against the oracle: the length-2N transforms and the
split into even- and odd-frequency length-N transforms (forced through the plan's knob,
whatever the autotuner chose), the knob API's error codes, and the split form's
spectral-tail sums."""
import ctypes

import numpy as np
import pytest

from oracle import direct, gtensor, selection as OS, solver as osolver
from paper_1612_01799_gb300 import densities as D

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
SPLIT_N = (16, 80, 256, 320, 384)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01799_gb300 import build
    build.build()
    return torch


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def solve_form(torch, N, L, tol, dtype, rho, form):
    from paper_1612_01799_gb300 import Plan
    with Plan(N, L, tol, dtype) as p:
        assert p.z_split in (0, 1)
        p.z_split = form
        assert p.z_split == form
        t = torch.from_numpy(np.ascontiguousarray(rho, dtype=p.np_dtype)).cuda()
        u = p.solve(t)
        torch.cuda.synchronize()
        return u.cpu().numpy().astype(np.float64)


def test_knob_codes(torch_cuda):
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    for N in (4, 8, 16, 32, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384):
        with Plan(N, 4.0, 1e-6, "f32") as p:
            if N in SPLIT_N:
                p.z_split = 1
                p.z_split = 0
            else:
                assert p.z_split == 0
                assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_Z_SPLIT, 1) == -4
            assert lib.poisson_plan_set_knob(p.handle, 7, 0) == -1
            assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_Z_SPLIT, 2) == -1
            v = ctypes.c_int()
            assert lib.poisson_plan_get_knob(p.handle, 7, ctypes.byref(v)) == -1
            assert lib.poisson_plan_get_knob(None, _lib.KNOB_Z_SPLIT, ctypes.byref(v)) == -1


def test_tuning_is_per_shape(torch_cuda):
    """Every plan of one (N, dtype) gets the autotuner's first decision."""
    from paper_1612_01799_gb300 import Plan
    for dtype in ("f32", "f64"):
        with Plan(256, 10.0, 1e-6, dtype) as a, Plan(256, 3.0, 1e-9, dtype, max_batch=2) as b:
            assert a.z_split == b.z_split


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [16, 80])
def test_forms_full_grid_small(torch_cuda, plan_cache, N, dtype):
    L = 10.0 if N >= 32 else 4.0
    tol = 1e-12 if dtype == "f64" else 1e-6
    rho = D.config_aniso4(N=N, seed=200 + N).gaussians.sample(N, L)
    uo = osolver.solve(rho, L, tol, plan=plan_cache(N, L, tol))
    for form in (0, 1):
        u = solve_form(torch_cuda, N, L, tol, dtype, rho, form)
        assert rel_l2(u, uo) <= TOL[dtype], form
        assert np.max(np.abs(u - uo)) <= 50 * TOL[dtype] * np.abs(uo).max(), form


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_forms_full_grid_n256(torch_cuda, plan_cache, dtype):
    """The 4-Gaussian density on [-10,10]^3 at N = 256, both forms, every grid point."""
    rho = D.config_aniso4().sample()
    tol = 1e-12 if dtype == "f64" else 1e-6
    uo = osolver.solve(rho, 10.0, tol, plan=plan_cache(256, 10.0, tol))
    for form in (0, 1):
        u = solve_form(torch_cuda, 256, 10.0, tol, dtype, rho, form)
        assert rel_l2(u, uo) <= TOL[dtype], form


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [320, 384])
def test_forms_sampled_large(torch_cuda, N, dtype):
    """Output lines against the oracle's real-space evaluation of the same discrete
    convolution (the full 2N-cube FFT oracle is too large here)."""
    L = 10.0
    tol = 1e-12 if dtype == "f64" else 1e-6
    rho = D.config_aniso4(N=N, seed=300 + N).gaussians.sample(N, L)
    lines = [(0, 0), (N // 2, N // 2 - 1), (N - 1, N - 1), (N // 3, 2 * N // 3), (N - 2, 1)]
    ref = direct.sample_lines(rho, gtensor.make_plan(N, L, tol), lines)
    for form in (0, 1):
        u = solve_form(torch_cuda, N, L, tol, dtype, rho, form)
        got = np.stack([u[z, y] for z, y in lines])
        assert rel_l2(got, ref) <= TOL[dtype], form


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_split_form_tail(torch_cuda, dtype):
    """The checked solve in the split form: same potential as the unchecked one, and eta
    as defined on the padded spectrum."""
    torch = torch_cuda
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    N, L = 80, 6.0
    rho = D.config_aniso4(N=N, seed=31).gaussians.sample(N, L)
    with Plan(N, L, 1e-6, dtype) as p:
        p.z_split = 1
        t = torch.from_numpy(rho.astype(p.np_dtype)).cuda()
        u1 = p.solve(t)
        u2 = torch.empty_like(t)
        eta = ctypes.c_double()
        assert lib.poisson_solve_checked(p.handle, ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(u2.data_ptr()),
                                         ctypes.byref(eta), None) == 0
        torch.cuda.synchronize()
        assert torch.equal(u1, u2)
    ref = OS.spectral_tail(rho.astype(np.float32 if dtype == "f32" else np.float64))
    assert eta.value == pytest.approx(ref, rel=2e-3 if dtype == "f32" else 1e-6, abs=1e-12)
