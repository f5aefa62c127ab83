"""The FP64 plans' two arithmetics against the FP64 oracle: FP64 on the FP64 pipe and
double-float (each real hi + lo of two FP32 numbers, on the FP32 pipe; POISSON_KNOB_ARITH).
Both must meet the FP64 parity bar (rel-L2 <= 1e-12) on the full grid at every compiled
radix path, on sampled lines of the N = 512 workload, on rectangular boxes, with the
literal correction, in batched solves and in the checked solve."""
import math

import numpy as np
import pytest

from oracle import box as obox, direct, gtensor, selection, solver as osolver
from paper_1612_01799_gb300 import densities as D

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def solve(torch, p, rho):
    t = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float64)).cuda()
    u = p.solve(t)
    torch.cuda.synchronize()
    p.last_status()
    return u.cpu().numpy()


@pytest.mark.parametrize("arith", ["df", "f64"])
@pytest.mark.parametrize("N", [4, 8, 16, 32, 48, 64, 80, 96, 128, 160, 192, 256])
def test_full_grid(torch_cuda, plan_cache, N, arith):
    from paper_1612_01799_gb300 import Plan
    L = 10.0 if N >= 32 else 4.0
    rho = D.config_aniso4(N=N, seed=200 + N).gaussians.sample(N, L)
    uo = osolver.solve(rho, L, 1e-12, plan=plan_cache(N, L, 1e-12))
    with Plan(N, L, 1e-12, "f64") as p:
        p.arith = arith
        assert p.arith == arith
        for z in ([0, 1] if arith == "f64" and N in (16, 80, 256) else [0]):
            p.z_form = z
            u = solve(torch_cuda, p, rho)
            assert rel_l2(u, uo) <= TOL, (z, rel_l2(u, uo))
            assert np.abs(u - uo).max() <= 50 * TOL * np.abs(uo).max()


@pytest.mark.parametrize("N", [320, 384])
def test_full_grid_large(torch_cuda, N):
    from paper_1612_01799_gb300 import Plan
    L = 10.0
    rho = D.config_aniso4(N=N, seed=200 + N).gaussians.sample(N, L)
    uo = osolver.solve(rho, L, 1e-12)
    with Plan(N, L, 1e-12, "f64") as p:
        p.arith = "df"
        assert rel_l2(solve(torch_cuda, p, rho), uo) <= TOL


def test_n512_sampled_lines(torch_cuda):
    """Config 3 (bump plus 8 Gaussians, N = 512) against the oracle's real-space sum on
    lines crossing the column tiles and the box faces."""
    from paper_1612_01799_gb300 import Plan
    w = D.config_bump8(N=512)
    rho = w.sample()
    lines = [(0, 0), (7, 300), (255, 256), (256, 17), (448, 447), (511, 511)]
    ref = direct.sample_lines(rho, gtensor.make_plan(512, w.L, 1e-12), lines)
    with Plan(512, w.L, 1e-12, "f64") as p:
        p.arith = "df"
        u = solve(torch_cuda, p, rho)
    got = np.stack([u[z, y, :] for z, y in lines])
    assert rel_l2(got, ref) <= TOL


def test_arithmetics_agree_and_switch_back(torch_cuda):
    from paper_1612_01799_gb300 import Plan
    N, L = 64, 10.0
    rho = np.random.default_rng(3).standard_normal((N, N, N))
    with Plan(N, L, 1e-12, "f64") as p:
        p.arith = "df"
        a = solve(torch_cuda, p, rho)
        p.arith = "f64"
        b = solve(torch_cuda, p, rho)
        p.arith = "df"
        c = solve(torch_cuda, p, rho)
    assert rel_l2(a, b) < 1e-13
    assert np.array_equal(a, c)
    with Plan(N, L, 1e-6, "f32") as q:
        with pytest.raises(ValueError):
            q.arith = "df"


@pytest.mark.parametrize("n", [16, 32])
def test_box_and_literal(torch_cuda, n):
    """Table 6's box and the literal correction (the oracle's own unpadded transform pair)."""
    from paper_1612_01799_gb300 import Plan
    lo, hi = (-2.0, -4.0, -6.0), (2.0, 4.0, 6.0)
    op = obox.make_box_plan(n, lo, hi, 1e-12)
    rho = np.random.default_rng(n).uniform(-1, 1, (n, n, n))
    with Plan(n, (2.0, 4.0, 6.0), 1e-12, "f64") as p:
        p.arith = "df"
        assert rel_l2(solve(torch_cuda, p, rho), obox.solve_box(rho, op)) <= TOL
        p.correction = "literal"
        assert rel_l2(solve(torch_cuda, p, rho), obox.solve_box_literal(rho, op)) <= TOL


def test_batched_equals_single(torch_cuda):
    from paper_1612_01799_gb300 import Plan, solve_batched
    torch = torch_cuda
    N, L = 48, 10.0
    rhos = [torch.from_numpy(D.config_aniso4(N=N, seed=s).gaussians.sample(N, L)).cuda() for s in (1, 2, 3)]
    with Plan(N, L, 1e-12, "f64", max_batch=3) as p:
        p.arith = "df"
        outs = [torch.empty_like(r) for r in rhos]
        solve_batched([p] * 3, rhos, outs)
        torch.cuda.synchronize()
        for r, o in zip(rhos, outs):
            assert torch.equal(p.solve(r), o)


def test_checked_solve_tail(torch_cuda):
    """The a-posteriori indicator of a double-float solve against the oracle's spectral tail."""
    import ctypes
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    torch = torch_cuda
    N, L = 32, 4.0
    rho = D.config_aniso4(N=N, seed=9).gaussians.sample(N, L)
    with Plan(N, L, 1e-12, "f64") as p:
        p.arith = "df"
        t = torch.from_numpy(rho).cuda()
        u = torch.empty_like(t)
        eta = ctypes.c_double()
        assert lib.poisson_solve_checked(p.handle, ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.byref(eta), None) == 0
        torch.cuda.synchronize()
    ref = selection.spectral_tail(rho)
    assert abs(eta.value - ref) <= 1e-3 * ref + 1e-12
    assert rel_l2(u.cpu().numpy(), osolver.solve(rho, L, 1e-12)) <= TOL
