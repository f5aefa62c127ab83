"""The slab stages of the C-ABI (poisson_slab_forward / _z / _inverse, poisson_plan_spectrum)
on one GPU: P ranks emulated in turn, one plan each, the two exchanges of the slab
decomposition done as block copies between the plans' spectrum buffers (the blocks an
all-to-all would move), the assembled potential against the FP64 oracle (FP32 <= 1e-5,
FP64 <= 1e-12 rel-L2, element by element) and against each plan's own whole solve."""
import numpy as np
import pytest

from oracle import box as obox, solver as osolver
from paper_1612_01799_gb300 import densities as D

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


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


def emulated(torch, plans, rho):
    """u from P plans as P slab ranks (rho: [nz][ny][nx] numpy)."""
    from paper_1612_01799_gb300 import slab
    P = len(plans)
    nx, ny, nz = plans[0].n
    st = [slab.PlanStages(torch, p) for p in plans]
    zb = [slab.bounds(nz, P, r) for r in range(P)]
    kb = [slab.bounds(2 * ny, P, r) for r in range(P)]
    dt = plans[0].torch_dtype
    for r in range(P):
        z0, z1 = zb[r]
        st[r].forward(torch.from_numpy(np.ascontiguousarray(rho[z0:z1])).to("cuda", dt).reshape(-1), z0, z1 - z0)
    w = [s.spectrum(0) for s in st]
    for r in range(P):                     # rank s receives [z of r][ky of s] from rank r
        for s in range(P):
            if s != r:
                (z0, z1), (k0, k1) = zb[r], kb[s]
                w[s][z0:z1, k0:k1].copy_(w[r][z0:z1, k0:k1])
    for r in range(P):
        st[r].z(kb[r][0], kb[r][1] - kb[r][0])
    w = [s.spectrum(1) for s in st]
    for r in range(P):                     # rank s receives [z of s][ky of r] from rank r
        for s in range(P):
            if s != r:
                (z0, z1), (k0, k1) = zb[s], kb[r]
                w[s][z0:z1, k0:k1].copy_(w[r][z0:z1, k0:k1])
    parts = [st[r].inverse(zb[r][0], zb[r][1] - zb[r][0]) for r in range(P)]
    torch.cuda.synchronize()
    for p in plans:
        p.last_status()
    return torch.cat(parts).cpu().numpy().astype(np.float64).reshape(nz, ny, nx)


@pytest.mark.parametrize("N,dtype,P", [(64, "f32", 2), (64, "f32", 4), (48, "f64", 3), (24, "f32", 2),
                                       (256, "f32", 4), (32, "f64", 2)])
def test_cube_slabs(torch_cuda, plan_cache, N, dtype, P):
    from paper_1612_01799_gb300 import Plan
    L = 10.0
    tol = 1e-12 if dtype == "f64" else 1e-6
    rho = D.config_aniso4(N=N, seed=600 + N).gaussians.sample(N, L)
    uo = osolver.solve(rho, L, tol, plan=plan_cache(N, L, tol))
    plans = [Plan(N, L, tol, dtype) for _ in range(P)]
    try:
        u = emulated(torch_cuda, plans, rho)
        whole = plans[0].solve(torch_cuda.from_numpy(rho.astype(plans[0].np_dtype)).cuda()).cpu().numpy()
    finally:
        for p in plans:
            p.close()
    assert rel_l2(u, uo) <= TOL[dtype]
    assert np.abs(u - uo).max() <= 50 * TOL[dtype] * np.abs(uo).max()
    assert rel_l2(u, whole) <= TOL[dtype]


def test_box_slabs_fp64_arithmetics(torch_cuda):
    from paper_1612_01799_gb300 import Plan
    n, lo, hi = (16, 24, 32), (-2.0, -4.0, -6.0), (2.0, 4.0, 6.0)
    op = obox.make_box_plan(n, lo, hi, 1e-12)
    rho = np.random.default_rng(8).uniform(-1, 1, (n[2], n[1], n[0]))
    uo = obox.solve_box(rho, op)
    for ar in ("df", "f64"):
        plans = [Plan(n, (2.0, 4.0, 6.0), 1e-12, "f64") for _ in range(3)]
        try:
            for p in plans:
                p.arith = ar
            u = emulated(torch_cuda, plans, rho)
        finally:
            for p in plans:
                p.close()
        assert rel_l2(u, uo) <= TOL["f64"], ar


def test_slab_arguments(torch_cuda):
    import ctypes
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    with Plan(16, 4.0, 1e-6, "f32") as p:
        t = torch_cuda.zeros(16 ** 3, device="cuda")
        ptr = ctypes.c_void_p(t.data_ptr())
        assert lib.poisson_slab_forward(p.handle, ptr, 10, 7, None) == -1     # past n_z
        assert lib.poisson_slab_forward(p.handle, None, 0, 4, None) == -1
        assert lib.poisson_slab_z(p.handle, 30, 3, None) == -1               # past 2 n_y
        assert lib.poisson_slab_inverse(p.handle, ptr, -1, 2, None) == -1
        assert lib.poisson_plan_spectrum(p.handle, 2, ctypes.byref(ctypes.c_void_p()), None, None) == -1
