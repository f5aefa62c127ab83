"""Every form of the fused z pass against the oracle: the length-2N transforms, the split
into even- and odd-frequency length-N transforms and the warp form (forced through the
plan's knob, whatever the autotuner chose), the knob API's error codes, and the split and
warp forms' spectral-tail sums and batched solves."""
import ctypes

import numpy as np
import pytest

from oracle import direct, gtensor, selection as OS, solver as osolver
from paper_1612_01799_gb300 import densities as D

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
SPLIT_N = (16, 80, 256, 320, 384)
WARP_N = (64, 96, 128, 160, 192, 256)


def forms(N, dtype, arith=None):
    """z forms of (N, dtype); an FP64 plan's split form exists in FP64 arithmetic only, so
    with arith None (whichever the plan chose) it is left out for FP64."""
    split = N in SPLIT_N and (dtype == "f32" or arith == "f64")
    return [0] + ([1] if split else []) + ([2] if dtype == "f32" and (N in WARP_N or N == 512) else [])


def yforms(N, dtype):
    return [0] + ([1] if dtype == "f32" and (N in WARP_N or N == 512) else [])


def xforms(N, dtype):
    return [0] + ([1] if dtype == "f32" and (N in WARP_N or N == 512) else [])


def xyforms(N, dtype):
    return [0] + ([1] if dtype == "f32" and N in WARP_N else [])


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


def solve_form(torch, N, L, tol, dtype, rho, form, yform=None, xform=None, xyform=0):
    from paper_1612_01799_gb300 import Plan
    with Plan(N, L, tol, dtype) as p:
        assert p.z_form in forms(N, dtype, p.arith)
        if dtype == "f64" and form == 1:
            p.arith = "f64"             # the split form exists in FP64 arithmetic only
        assert p.y_form in yforms(N, dtype)
        assert p.x_form in xforms(N, dtype)
        assert p.xy_form in xyforms(N, dtype)
        p.z_form = form
        assert p.z_form == form
        p.xy_form = xyform
        assert p.xy_form == xyform
        if yform is not None:
            p.y_form = yform
            assert p.y_form == yform
        if xform is not None:
            p.x_form = xform
            assert p.x_form == xform
        t = torch.from_numpy(np.ascontiguousarray(rho, dtype=p.np_dtype)).cuda()
        u = p.solve(t)
        torch.cuda.synchronize()
        p.last_status()
        return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_knob_codes(torch_cuda, dtype):
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    for N in (4, 8, 16, 32, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512):
        with Plan(N, 4.0, 1e-6, dtype) as p:
            assert p.z_form in forms(N, dtype, p.arith)
            if dtype == "f64":
                p.arith = "f64" if N % 2 == 0 and (N // 2) % 2 == 0 else "df"
            have = forms(N, dtype, p.arith)
            assert p.z_form in have
            for f in (0, 1, 2):
                if f in have:
                    p.z_form = f
                    assert p.z_form == f
                else:
                    assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_Z_FORM, f) == -4
            for f in (0, 1):
                if f in yforms(N, dtype):
                    p.y_form = f
                    assert p.y_form == f
                else:
                    assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_Y_FORM, f) == -4
            assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_Y_FORM, 2) == -1
            for f in (0, 1):
                if f in xforms(N, dtype):
                    p.x_form = f
                    assert p.x_form == f
                else:
                    assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_X_FORM, f) == -4
            assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_X_FORM, 2) == -1
            for f in (0, 1):
                if f in xyforms(N, dtype):
                    p.xy_form = f
                    assert p.xy_form == f
                else:
                    assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_XY_FORM, f) == -4
            assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_XY_FORM, 2) == -1
            assert lib.poisson_plan_set_knob(p.handle, 7, 0) == -1
            assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_Z_FORM, 3) == -1
            assert lib.poisson_plan_set_knob(p.handle, _lib.KNOB_Z_FORM, -1) == -1
            v = ctypes.c_int()
            assert lib.poisson_plan_get_knob(p.handle, 7, ctypes.byref(v)) == -1
            assert lib.poisson_plan_get_knob(None, _lib.KNOB_Z_FORM, ctypes.byref(v)) == -1


def test_tuning_is_per_shape(torch_cuda):
    """Every plan of one (N, dtype) gets the autotuner's first decision."""
    from paper_1612_01799_gb300 import Plan
    for dtype in ("f32", "f64"):
        with Plan(256, 10.0, 1e-6, dtype) as a, Plan(256, 3.0, 1e-9, dtype, max_batch=2) as b:
            assert a.z_form == b.z_form and a.y_form == b.y_form and a.x_form == b.x_form
            assert a.xy_form == b.xy_form


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N", [16, 80])
def test_forms_full_grid_small(torch_cuda, plan_cache, N, dtype):
    L = 10.0 if N >= 32 else 4.0
    tol = 1e-12 if dtype == "f64" else 1e-6
    rho = D.config_aniso4(N=N, seed=200 + N).gaussians.sample(N, L)
    uo = osolver.solve(rho, L, tol, plan=plan_cache(N, L, tol))
    for form in forms(N, dtype, "f64"):
        u = solve_form(torch_cuda, N, L, tol, dtype, rho, form)
        assert rel_l2(u, uo) <= TOL[dtype], form
        assert np.max(np.abs(u - uo)) <= 50 * TOL[dtype] * np.abs(uo).max(), form


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_forms_full_grid_n256(torch_cuda, plan_cache, dtype):
    """The 4-Gaussian density on [-10,10]^3 at N = 256, both forms, every grid point."""
    rho = D.config_aniso4().sample()
    tol = 1e-12 if dtype == "f64" else 1e-6
    uo = osolver.solve(rho, 10.0, tol, plan=plan_cache(256, 10.0, tol))
    combos = [(f, 0, 0, 0) for f in forms(256, dtype, "f64")] + [(f, 1, x, 0) for f in forms(256, dtype)
                                                                  for x in xforms(256, dtype) if dtype == "f32"]
    combos += [(f, 0, 0, 1) for f in forms(256, dtype) if dtype == "f32"]
    for form, yform, xform, xyform in combos:
        u = solve_form(torch_cuda, 256, 10.0, tol, dtype, rho, form, yform, xform, xyform)
        assert rel_l2(u, uo) <= TOL[dtype], (form, yform, xform, xyform)
        assert np.max(np.abs(u - uo)) <= 50 * TOL[dtype] * np.abs(uo).max(), (form, yform, xform, xyform)


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
    for form in forms(N, dtype, "f64"):
        u = solve_form(torch_cuda, N, L, tol, dtype, rho, form)
        got = np.stack([u[z, y] for z, y in lines])
        assert rel_l2(got, ref) <= TOL[dtype], form


@pytest.mark.parametrize("form,N,dtype", [(1, 80, "f64"), (1, 80, "f32"), (2, 256, "f32"), (2, 192, "f32"),
                                          (2, 160, "f32")])
def test_form_tail(torch_cuda, form, N, dtype):
    """The checked solve in a non-default form: same potential as the unchecked one, and
    eta as defined on the padded spectrum.  The box [-6,6]^3 truncates the Gaussians, so
    eta (2.5e-4 at N = 256) stands far above the FP32 transforms' rounding floor (about
    1e-7 here; on [-10,10]^3 the exact eta, 1.6e-8, lies below it)."""
    torch = torch_cuda
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    L = 6.0
    rho = D.config_aniso4(N=N, seed=31).gaussians.sample(N, L)
    with Plan(N, L, 1e-6, dtype) as p:
        if dtype == "f64":
            p.arith = "f64"             # the split form exists in FP64 arithmetic only
        p.z_form = form
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


@pytest.mark.parametrize("N,yform,xform", [(256, 0, 0), (256, 1, 0), (256, 1, 1), (192, 1, 1), (160, 1, 1),
                                           (128, 1, 1), (96, 1, 1), (64, 1, 1)])
def test_warp_form_batched(torch_cuda, N, yform, xform):
    """Three densities through one grouped launch sequence in the warp forms: each equals
    its single solve bit for bit, and the plan reports no timed-out wait."""
    torch = torch_cuda
    from paper_1612_01799_gb300 import Plan, solve_batched
    L = 10.0
    rhos = [torch.from_numpy(D.config_aniso4(N=N, seed=40 + i).gaussians.sample(N, L).astype(np.float32)).cuda()
            for i in range(3)]
    with Plan(N, L, 1e-6, "f32", max_batch=3) as p:
        p.z_form = 2
        p.y_form = yform
        p.x_form = xform
        outs = [torch.empty_like(r) for r in rhos]
        solve_batched([p] * 3, rhos, outs)
        torch.cuda.synchronize()
        for r, o in zip(rhos, outs):
            assert torch.equal(p.solve(r), o)
        p.last_status()


@pytest.mark.parametrize("zform,yform,xform", [(0, 0, 0), (0, 0, 1), (2, 1, 1), (2, 0, 0), (0, 1, 0)])
def test_forms_sampled_n512(torch_cuda, zform, yform, xform):
    """N = 512 (the padded 1024^3 grid), FP32, the z and y passes in their block forms and
    their warp forms (one warp per column, 1024 = 32 x 32) with both x forms: output lines
    against the oracle's real-space evaluation of the discrete convolution.  The lines
    cross every z, so each crosses all 16 output registers of the z warp form."""
    N, L, tol = 512, 10.0, 1e-6
    rho = D.config_aniso4(N=N, seed=512).gaussians.sample(N, L)
    lines = [(0, 0), (N // 2, N // 2 - 1), (N - 1, N - 1), (N // 3, 2 * N // 3), (7, 505)]
    ref = direct.sample_lines(rho, gtensor.make_plan(N, L, tol), lines)
    u = solve_form(torch_cuda, N, L, tol, "f32", rho, zform, yform, xform)
    got = np.stack([u[z, y] for z, y in lines])
    assert rel_l2(got, ref) <= TOL["f32"]


def test_w512_tail_matches_block_form(torch_cuda):
    """The checked solve at N = 512 in the z warp form: the same potential as its unchecked
    solve and the same eta as the block form (both sum the same forward spectrum; they
    differ only by FP32 rounding of the transforms)."""
    torch = torch_cuda
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    N, L = 512, 6.0
    rho = torch.from_numpy(D.config_aniso4(N=N, seed=33).gaussians.sample(N, L).astype(np.float32)).cuda()
    etas = {}
    with Plan(N, L, 1e-6, "f32") as p:
        for form in (0, 2):
            p.z_form = form
            u1 = p.solve(rho)
            u2 = torch.empty_like(rho)
            eta = ctypes.c_double()
            assert lib.poisson_solve_checked(p.handle, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u2.data_ptr()),
                                             ctypes.byref(eta), None) == 0
            torch.cuda.synchronize()
            assert torch.equal(u1, u2)
            etas[form] = eta.value
        p.last_status()
    assert etas[2] == pytest.approx(etas[0], rel=1e-3)


@pytest.mark.parametrize("N", [64, 96, 128, 160, 192])
def test_warp_forms_full_grid(torch_cuda, plan_cache, N):
    """N = 64 ... 192 (first-stage lengths 4 ... 12 of the warp forms), FP32: every form
    combination against the oracle on the whole grid."""
    L, tol = 10.0, 1e-6
    rho = D.config_aniso4(N=N, seed=400 + N).gaussians.sample(N, L)
    uo = osolver.solve(rho, L, tol, plan=plan_cache(N, L, tol))
    for form, yform, xform, xyform in [(0, 0, 0, 0), (2, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (2, 1, 1, 0),
                                       (2, 0, 0, 1), (0, 0, 0, 1)]:
        u = solve_form(torch_cuda, N, L, tol, "f32", rho, form, yform, xform, xyform)
        assert rel_l2(u, uo) <= TOL["f32"], (form, yform, xform, xyform)
        assert np.max(np.abs(u - uo)) <= 50 * TOL["f32"] * np.abs(uo).max(), (form, yform, xform, xyform)


@pytest.mark.parametrize("N,count", [(256, 1), (256, 3), (192, 2), (160, 2), (128, 3), (96, 4), (64, 1), (64, 6)])
def test_xy_fused_equals_separate_warp_forms(torch_cuda, N, count):
    """The fused x-y passes run the arithmetic of the separate warp-form x and y passes, so
    a batch through them equals, bit for bit, the same batch through the separate passes.
    Batches of several densities cycle every ring slot through several planes (the ring
    holds at most 2N planes per density and often fewer), so this also checks the slot
    hand-over between producers and consumers; the second fused run checks that the
    counters return to zero after a launch."""
    torch = torch_cuda
    from paper_1612_01799_gb300 import Plan, solve_batched
    L = 10.0
    rhos = [torch.from_numpy(D.config_aniso4(N=N, seed=70 + i).gaussians.sample(N, L).astype(np.float32)).cuda()
            for i in range(count)]
    with Plan(N, L, 1e-6, "f32", max_batch=count) as p:
        p.z_form = 2
        p.y_form = 1
        p.x_form = 1
        p.xy_form = 0
        ref = [torch.empty_like(r) for r in rhos]
        solve_batched([p] * count, rhos, ref)
        p.xy_form = 1
        for _ in range(2):
            outs = [torch.full_like(r, float("nan")) for r in rhos]
            solve_batched([p] * count, rhos, outs)
            torch.cuda.synchronize()
            for r, o in zip(ref, outs):
                assert torch.equal(r, o)
        p.last_status()


def test_xy_fused_timed_passes(torch_cuda):
    """With the fused x-y form the timed solve reports the forward x-y kernel in the x
    forward entry and the inverse one in the y inverse entry; the folded entries are 0."""
    torch = torch_cuda
    from paper_1612_01799_gb300 import Plan
    N = 128
    rho = torch.from_numpy(D.config_aniso4(N=N, seed=5).gaussians.sample(N, 10.0).astype(np.float32)).cuda()
    with Plan(N, 10.0, 1e-6, "f32") as p:
        p.xy_form = 1
        u = torch.empty_like(rho)
        ms = p.solve_timed(rho, u)
        assert ms[0] > 0 and ms[2] > 0 and ms[3] > 0
        assert ms[1] < 0.02 and ms[4] < 0.02
        assert torch.equal(u, p.solve(rho))
        p.last_status()


def test_w512_batched(torch_cuda):
    """Two densities at N = 512 through one grouped launch sequence in the N = 512 warp forms
    of the z and y passes: each equals its single solve bit for bit (the kernels take the
    density from the tile index)."""
    torch = torch_cuda
    from paper_1612_01799_gb300 import Plan, solve_batched
    N, L = 512, 10.0
    rhos = [torch.from_numpy(D.config_aniso4(N=N, seed=80 + i).gaussians.sample(N, L).astype(np.float32)).cuda()
            for i in range(2)]
    with Plan(N, L, 1e-6, "f32", max_batch=2) as p:
        p.z_form, p.y_form, p.x_form = 2, 1, 1
        outs = [torch.empty_like(r) for r in rhos]
        solve_batched([p, p], rhos, outs)
        torch.cuda.synchronize()
        for r, o in zip(rhos, outs):
            assert torch.equal(p.solve(r), o)
        p.last_status()
