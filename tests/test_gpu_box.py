"""GPU parity of rectangular-box plans (poisson_plan_create_box: N points on every axis,
half-lengths Lx, Ly, Lz; Sec. 2 standardised form) with the oracle's box solve, the
paper's Tables 2 and 6 through the CUDA path, and the cube as a special case."""
import math

import numpy as np
import pytest

from oracle import box as obox, exact

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
T2 = ((-3.0, -2.0, -1.0), (2.0, 3.5, 5.0))     # Table 2's box, sigma = 0.2 Gaussian at its centre
T6 = ((-2.0, -4.0, -6.0), (2.0, 4.0, 6.0))     # Table 6's box, anisotropic density


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


def rel_inf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def half(lo, hi):
    return tuple(0.5 * (b - a) for a, b in zip(lo, hi))


def coords(plan):
    x, y, z = (obox.axis(plan, q) for q in range(3))
    return x[None, None, :], y[None, :, None], z[:, None, None]


def t2_case(plan, sigma=0.2):
    c = [0.5 * (a + b) for a, b in zip(plan.lo, plan.hi)]
    x, y, z = coords(plan)
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    rho = np.exp(-r ** 2 / (2 * sigma ** 2)) / ((2 * math.pi) ** 1.5 * sigma ** 3)
    return rho, exact.gaussian_iso(r, sigma)


def t6_case(plan, s=(0.10, 0.20, 0.30)):
    X = coords(plan)
    E = np.exp(-sum(X[q] ** 2 / s[q] ** 2 for q in range(3)))
    P = sum(4 * X[q] ** 2 / s[q] ** 4 - 2 / s[q] ** 2 for q in range(3))
    return -P * E, E


def gpu(torch, p, rho):
    t = torch.from_numpy(np.ascontiguousarray(rho, dtype=p.np_dtype)).cuda()
    u = p.solve(t)
    torch.cuda.synchronize()
    p.last_status()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,geom", [(16, T2), (32, T2), (32, T6), (48, T6)])
def test_box_f64_matches_oracle(torch_cuda, N, geom):
    from paper_1612_01799_gb300 import Plan
    op = obox.make_box_plan(N, geom[0], geom[1], 1e-12)
    rho, _ = (t2_case if geom is T2 else t6_case)(op)
    uo = obox.solve_box(rho, op)
    with Plan(N, half(*geom), 1e-12, "f64") as p:
        assert rel_l2(gpu(torch_cuda, p, rho), uo) <= TOL["f64"]


@pytest.mark.parametrize("N", [64, 80, 128, 256])
def test_box_f32_every_form(torch_cuda, N):
    """Every z form, the warp forms reading the box symbol's kz-innermost copy."""
    from paper_1612_01799_gb300 import Plan
    op = obox.make_box_plan(N, T6[0], T6[1], 1e-6)
    rho, _ = t6_case(op)
    uo = obox.solve_box(rho, op)
    warp = (64, 96, 128, 160, 192, 256)
    with Plan(N, half(*T6), 1e-6, "f32") as p:
        zf = [0] + ([1] if N in (16, 80, 256, 320, 384) else []) + ([2] if N in warp else [])
        yf = [0] + ([1] if N in warp else [])
        for z in zf:
            for y in yf:
                p.z_form, p.y_form, p.x_form = z, y, y
                assert rel_l2(gpu(torch_cuda, p, rho), uo) <= TOL["f32"], (z, y)


def test_box_literal_correction_and_warp_form(torch_cuda):
    """The literal correction on a box (all-even frequencies, per-axis kappa) and the z warp
    form reading the rebuilt transposed copy give the same potential as the block form."""
    from paper_1612_01799_gb300 import Plan
    N = 64
    rho = np.random.default_rng(6).uniform(-1, 1, (N, N, N))
    with Plan(N, half(*T2), 1e-6, "f32") as p:
        p.correction = "literal"
        p.z_form = 0
        u0 = gpu(torch_cuda, p, rho)
        p.z_form = 2
        u2 = gpu(torch_cuda, p, rho)
        assert rel_l2(u2, u0) < 1e-6


def test_box_literal_f64(torch_cuda):
    """The literal correction on a box against the oracle's literal box solve (the Gaussian-sum
    convolution plus C0 rho + C2 Laplace(rho) from its own unpadded transform pair)."""
    from paper_1612_01799_gb300 import Plan
    N, tol = 32, 1e-10
    op = obox.make_box_plan(N, T2[0], T2[1], tol)
    rng = np.random.default_rng(8)
    checker = np.fromfunction(lambda i, j, l: (-1.0) ** (i + j + l), (N, N, N))
    with Plan(N, half(*T2), tol, "f64") as p:
        p.correction = "literal"
        for rho in (rng.uniform(-1, 1, (N, N, N)), checker):
            u = gpu(torch_cuda, p, rho)
            assert rel_l2(u, obox.solve_box_literal(rho, op)) <= TOL["f64"]
            assert rel_l2(u, obox.solve_box(rho, op)) > 2e-11   # the placements differ by 2e-10 and 1e-8


def test_cube_shaped_box_equals_cube_plan(torch_cuda):
    from paper_1612_01799_gb300 import Plan
    N, L = 32, 4.0
    rho = np.random.default_rng(5).uniform(-1, 1, (N, N, N))
    with Plan(N, L, 1e-10, "f64") as pc, Plan(N, (L, L, L), 1e-10, "f64") as pb:
        pb.z_form = pc.z_form = 0
        pb.y_form = pc.y_form = 0
        pb.x_form = pc.x_form = 0
        assert rel_l2(gpu(torch_cuda, pb, rho), gpu(torch_cuda, pc, rho)) < 1e-14


@pytest.mark.parametrize("N", [16, 32, 64])
def test_paper_tables_2_and_6_on_gpu(torch_cuda, N):
    """Within a factor 5 of the printed E (the paper above 1e-8 at these n)."""
    from paper_1612_01799_gb300 import Plan
    printed = {"T2": {16: 4.417e-02, 32: 1.857e-05}, "T6": {16: 1.011e+02, 32: 9.529e-01, 64: 1.544e-04}}
    for name, geom, case in (("T2", T2, t2_case), ("T6", T6, t6_case)):
        op = obox.make_box_plan(N, geom[0], geom[1], 1e-12)
        rho, ue = case(op)
        with Plan(N, half(*geom), 1e-12, "f64") as p:
            E = rel_inf(gpu(torch_cuda, p, rho), ue)
        ref = printed[name].get(N)
        if ref is None:
            assert E < 1e-12, (name, N, E)      # the paper stagnates at 3e-12 there; the method does not
        else:
            assert abs(math.log10(E / ref)) <= math.log10(5.0), (name, N, E, ref)


def test_box_n512_warp_form_against_block_form_and_oracle(torch_cuda):
    """N = 512 on Table 6's box: the one-warp-per-column z form (reading the box symbol's
    kz-innermost copy through its own tensor map) against the block form, and both against
    the oracle's box solve on the whole grid (a 1024^3 transform pair on the host)."""
    from paper_1612_01799_gb300 import Plan
    N = 512
    rng = np.random.default_rng(51)
    rho = rng.uniform(-1, 1, (N, N, N))
    with Plan(N, half(*T6), 1e-6, "f32") as p:
        p.z_form, p.y_form, p.x_form = 2, 1, 1
        u2 = gpu(torch_cuda, p, rho)
        p.z_form, p.y_form, p.x_form = 0, 0, 0
        u0 = gpu(torch_cuda, p, rho)
    assert rel_l2(u2, u0) < 2e-6
    avail = 0.0
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) / 2 ** 20
    if avail < 80:
        pytest.skip("the N = 512 box oracle needs about 30 GB of host memory")
    uo = obox.solve_box(rho, obox.make_box_plan(N, T6[0], T6[1], 1e-6))
    assert rel_l2(u2, uo) <= TOL["f32"]
    assert rel_l2(u0, uo) <= TOL["f32"]
