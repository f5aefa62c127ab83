"""Failure detection on the GPU without a fault: a device-side wait of the kind the TMA
passes use, on an mbarrier that nothing completes, runs out of its poll budget, records the
timeout in the plan's status word and returns; the host reads POISSON_ERR_TIMEOUT, the word
clears, and the same plan and context keep solving correctly."""
import ctypes

import numpy as np
import pytest

from oracle import solver as osolver
from paper_1612_01799_gb300 import densities as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01799_gb300 import build
    build.build()
    return torch


def test_timed_out_wait_is_reported_and_cleared(torch_cuda, plan_cache):
    torch = torch_cuda
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    N, L = 16, 4.0
    with Plan(N, L, 1e-6, "f32") as p:
        assert lib.poisson_last_status(p.handle, None) == 0
        assert lib.poisson_selftest_wait(p.handle, ctypes.c_longlong(2000), None) == 0
        assert lib.poisson_last_status(p.handle, None) == -5      # POISSON_ERR_TIMEOUT
        assert lib.poisson_last_status(p.handle, None) == 0       # read once, then cleared
        rho = D.config_aniso4(N=N, seed=7).gaussians.sample(N, L)
        u = p.solve(torch.from_numpy(rho.astype(np.float32)).cuda()).cpu().numpy()
        p.last_status()                                           # the solve's own waits completed
    uo = osolver.solve(rho, L, 1e-6, plan=plan_cache(N, L, 1e-6))
    assert np.linalg.norm(u - uo) / np.linalg.norm(uo) <= 1e-5


def test_selftest_arguments(torch_cuda):
    from paper_1612_01799_gb300 import Plan, _lib
    lib = _lib.load()
    with Plan(16, 4.0, 1e-6, "f32") as p:
        assert lib.poisson_selftest_wait(p.handle, ctypes.c_longlong(0), None) == -1
        assert lib.poisson_selftest_wait(p.handle, ctypes.c_longlong(1 << 25), None) == -1
    assert lib.poisson_selftest_wait(None, ctypes.c_longlong(10), None) == -1
