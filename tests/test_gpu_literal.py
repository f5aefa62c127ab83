"""GPU parity of the paper's literal near-field correction (POISSON_KNOB_CORRECTION = 1,
Sec. 2: I_delta = C0 rho + C2 Laplace(rho) with the Laplacian of the N-periodic series)
against the oracle's literal solve, which takes the Laplacian from its own unpadded N^3
FFT pair.  The densities (uniform noise, a checkerboard) have high frequencies, where the
two placements of the correction differ by far more than the FP64 tolerance, so the FP64
cases also check that the knob changes the symbol."""
import numpy as np
import pytest

from oracle import gtensor, solver as osolver

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
SPLIT_N = (16, 80, 256, 320, 384)
WARP_N = (64, 96, 128, 160, 192, 256)


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


def densities(N, seed=7):
    rng = np.random.default_rng(seed)
    return {"noise": rng.uniform(-1.0, 1.0, (N, N, N)),
            "checker": np.fromfunction(lambda i, j, l: (-1.0) ** (i + j + l), (N, N, N))}


def run(torch, p, rho):
    t = torch.from_numpy(np.ascontiguousarray(rho, dtype=p.np_dtype)).cuda()
    u = p.solve(t)
    torch.cuda.synchronize()
    p.last_status()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,L", [(16, 8.0), (32, 8.0), (48, 6.0)])
def test_literal_f64_matches_oracle_and_differs_from_fused(torch_cuda, N, L):
    from paper_1612_01799_gb300 import Plan
    tol = 1e-10
    plan = gtensor.make_plan(N, L, tol)
    with Plan(N, L, tol, "f64") as p:
        assert p.correction == "fused"
        p.correction = "literal"
        assert p.correction == "literal"
        for name, rho in densities(N).items():
            lit = osolver.solve_literal_correction(rho, L, tol, plan=plan)
            fused = osolver.solve(rho, L, tol, plan=plan)
            u = run(torch_cuda, p, rho)
            assert rel_l2(u, lit) <= TOL["f64"], name
            assert rel_l2(u, fused) > 1e-9, name


def test_switching_back_restores_the_fused_symbol(torch_cuda):
    from paper_1612_01799_gb300 import Plan
    N, L, tol = 32, 8.0, 1e-10
    rho = densities(N)["noise"]
    with Plan(N, L, tol, "f64") as ref:
        u_ref = run(torch_cuda, ref, rho)
    with Plan(N, L, tol, "f64") as p:
        p.correction = "literal"
        u_lit = run(torch_cuda, p, rho)
        p.correction = "literal"   # no change: no rebuild
        assert np.array_equal(run(torch_cuda, p, rho), u_lit)
        p.correction = "fused"
        assert p.correction == "fused"
        assert np.array_equal(run(torch_cuda, p, rho), u_ref)


@pytest.mark.parametrize("N", [64, 80, 128])
def test_literal_f32_every_form(torch_cuda, N):
    from paper_1612_01799_gb300 import Plan
    L, tol = 8.0, 1e-6
    plan = gtensor.make_plan(N, L, tol)
    rho = densities(N)["noise"]
    lit = osolver.solve_literal_correction(rho, L, tol, plan=plan)
    zf = [0] + ([1] if N in SPLIT_N else []) + ([2] if N in WARP_N else [])
    yf = [0] + ([1] if N in WARP_N else [])
    with Plan(N, L, tol, "f32") as p:
        p.correction = "literal"
        for z in zf:
            for y in yf:
                p.z_form, p.y_form, p.x_form = z, y, y
                assert rel_l2(run(torch_cuda, p, rho), lit) <= TOL["f32"], (z, y)


def test_knob_codes(torch_cuda):
    from paper_1612_01799_gb300 import Plan, _lib
    import ctypes
    lib = _lib.load()
    with Plan(16, 4.0, 1e-6, "f32") as p:
        v = ctypes.c_int(-1)
        assert lib.poisson_plan_get_knob(p.handle, _lib.KNOB_CORRECTION, ctypes.byref(v)) == 0
        assert v.value == 0
        assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_CORRECTION, 2) == -1
        assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_CORRECTION, -1) == -1
        assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_CORRECTION, 1) == 0
        assert lib.poisson_plan_get_knob(p.handle, _lib.KNOB_CORRECTION, ctypes.byref(v)) == 0
        assert v.value == 1
        with pytest.raises(ValueError):
            p.correction = "other"
