"""The plan's per-axis table A_j(k), built on the device at plan creation, against the host
rule it follows (the library's csrc/setup.cpp, compiled here with g++ through the test
shim): the same composite Gauss-Legendre rule and closed form, the cosines by rotation
from panel to panel (re-seeded every 16 panels) instead of a cos per node."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1612_01799_gb300", "csrc")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01799_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("shim") / "host_setup.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-I", CSRC,
                    os.path.join(CSRC, "setup.cpp"), os.path.join(HERE, "native", "host_setup_shim.cpp"),
                    "-o", out], check=True)
    lib = ctypes.CDLL(out)
    P = ctypes.POINTER(ctypes.c_double)
    lib.shim_host_tables.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int), P, P, P, P]
    return lib


@pytest.mark.parametrize("N,L,tol", [(160, 10.0, 1e-9), (512, 6.0, 1e-6), (512, 10.0, 1e-12), (1024, 10.0, 1e-12)])
def test_device_axis_table_matches_host_rule(torch_cuda, shim, N, L, tol):
    from paper_1612_01799_gb300 import Plan
    cap = 1000
    n = ctypes.c_int()
    tau, w = np.zeros(cap), np.zeros(cap)
    A = np.zeros(cap * (N + 1))
    sc = np.zeros(6)
    P = ctypes.POINTER(ctypes.c_double)
    assert shim.shim_host_tables(N, L, tol, cap, ctypes.byref(n), tau.ctypes.data_as(P), w.ctypes.data_as(P),
                                 A.ctypes.data_as(P), sc.ctypes.data_as(P)) == 0
    S = n.value
    A = A[:S * (N + 1)].reshape(S, N + 1)
    with Plan(N, L, tol, "f32") as p:
        tp, wp = p.gauss_sum()
        Ad = p.axis_table()
    assert len(tp) == S and np.array_equal(tp, tau[:S]) and np.array_equal(wp, w[:S])
    assert Ad.shape == A.shape
    assert np.max(np.abs(Ad - A)) <= 1e-13
    big = tau[:S] >= 3.0  # closed form on both sides
    assert np.max(np.abs(Ad[big] - A[big]) / np.maximum(np.abs(A[big]), 1e-300)) <= 1e-13
