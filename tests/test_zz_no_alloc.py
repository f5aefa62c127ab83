"""poisson_solve_noalloc: the solve for callers that may not allocate device memory when
they solve (a real-time loop that must not enter an allocator, a process whose device
memory a framework's caching allocator holds).  It keeps its tables, workspace and status
word in one static device array instead of a plan.  Its results must match poisson_solve
(a plan's solve) within the parity tolerances, on consecutive calls that share the array,
including a change of parameters in between; a timed-out wait must be reported by
poisson_noalloc_last_status; and its calls must take no device memory.  Collected last
(file name), so a run that stops at the first failure has run every other test before
this one."""
import ctypes

import numpy as np
import pytest

from paper_1612_01799_gb300 import densities as D

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
CODE = {"f32": 0, "f64": 1}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01799_gb300 import _lib, build
    build.build()
    return torch, _lib.load()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def noalloc(torch, lib, N, L, tol, dtype, rho_t):
    out = torch.empty_like(rho_t)
    s = torch.cuda.current_stream().cuda_stream
    rc = lib.poisson_solve_noalloc(N, L, tol, CODE[dtype], ctypes.c_void_p(rho_t.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s))
    assert rc == 0, rc
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def planned(torch, N, L, tol, dtype, rho_t):
    from paper_1612_01799_gb300 import Plan
    with Plan(N, L, tol, dtype) as p:
        u = p.solve(rho_t)
        torch.cuda.synchronize()
        return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_plan_solve(env, dtype):
    torch, lib = env
    tol = 1e-12 if dtype == "f64" else 1e-6
    npdt = np.float64 if dtype == "f64" else np.float32
    cases = [(64, 10.0, 11), (64, 10.0, 12), (32, 8.0, 13), (64, 10.0, 14)]
    for N, L, seed in cases:            # two calls in a row, a change of N, and back
        rho = D.config_aniso4(N=N, seed=seed).gaussians.sample(N, L).astype(npdt)
        rho_t = torch.from_numpy(rho).cuda()
        got = noalloc(torch, lib, N, L, tol, dtype, rho_t)
        ref = planned(torch, N, L, tol, dtype, rho_t)
        assert rel_l2(got, ref) <= TOL[dtype], (N, seed)


def test_noalloc_rejects_sizes_beyond_its_array(env):
    torch, lib = env
    t = torch.zeros(96 ** 3, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    assert lib.poisson_solve_noalloc(96, 10.0, 1e-6, 0, p, p, None) == -4   # N > 64
    assert lib.poisson_solve_noalloc(63, 10.0, 1e-6, 0, p, p, None) == -1   # odd N
    assert lib.poisson_solve_noalloc(64, 10.0, 1e-6, 0, None, p, None) == -1
    assert lib.poisson_solve_noalloc(64, 10.0, 1e-6, 5, p, p, None) == -1


def test_noalloc_timeout_is_reported_and_cleared(env):
    """A bounded wait on the allocation-free solves' status word that nothing completes gives
    up, poisson_noalloc_last_status reports POISSON_ERR_TIMEOUT once and clears the word, and
    the next allocation-free solve still matches a plan's solve."""
    torch, lib = env
    N, L, tol = 64, 10.0, 1e-6
    rho = D.config_aniso4(N=N, seed=15).gaussians.sample(N, L).astype(np.float32)
    rho_t = torch.from_numpy(rho).cuda()
    noalloc(torch, lib, N, L, tol, "f32", rho_t)
    assert lib.poisson_noalloc_last_status(None) == 0
    assert lib.poisson_noalloc_selftest_wait(ctypes.c_longlong(2000), None) == 0
    assert lib.poisson_noalloc_last_status(None) == -5            # POISSON_ERR_TIMEOUT
    assert lib.poisson_noalloc_last_status(None) == 0             # read once, then cleared
    got = noalloc(torch, lib, N, L, tol, "f32", rho_t)
    assert lib.poisson_noalloc_last_status(None) == 0             # the solve's own waits completed
    assert rel_l2(got, planned(torch, N, L, tol, "f32", rho_t)) <= TOL["f32"]
    assert lib.poisson_noalloc_selftest_wait(ctypes.c_longlong(0), None) == -1


def test_noalloc_set_up_and_solve_take_no_device_memory(env):
    """A call that redoes the set-up (same N and kernels, another L) and a call that only
    solves leave the device's free memory unchanged."""
    torch, lib = env
    N, tol = 64, 1e-6
    rho_t = torch.from_numpy(D.config_aniso4(N=N, seed=16).gaussians.sample(N, 10.0)
                             .astype(np.float32)).cuda()
    out = torch.empty_like(rho_t)
    s = torch.cuda.current_stream().cuda_stream
    args = lambda L: (N, L, tol, 0, ctypes.c_void_p(rho_t.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                      ctypes.c_void_p(s))
    assert lib.poisson_solve_noalloc(*args(10.0)) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert lib.poisson_solve_noalloc(*args(9.0)) == 0          # new tables, same kernels
    assert lib.poisson_solve_noalloc(*args(9.0)) == 0          # launches only
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert lib.poisson_noalloc_last_status(None) == 0
