"""The library's host-side setup (csrc/setup.cpp, built here with g++ through a test shim)
against the oracle: same Gaussian sum, per-axis factors to 1e-13, near-zone constants,
and exact twiddles.  No GPU needed."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1612_01799_gb300", "csrc")


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
    lib.shim_twiddles.argtypes = [ctypes.c_int, P]
    lib.shim_box_scalars.argtypes = [ctypes.POINTER(ctypes.c_int), P, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int), P, P, P]
    return lib


def host_tables(lib, N, L, tol):
    cap = 1000
    n = ctypes.c_int()
    tau, w = np.zeros(cap), np.zeros(cap)
    A = np.zeros(cap * (N + 1))
    sc = np.zeros(6)
    P = ctypes.POINTER(ctypes.c_double)
    rc = lib.shim_host_tables(N, L, tol, cap, ctypes.byref(n), tau.ctypes.data_as(P),
                              w.ctypes.data_as(P), A.ctypes.data_as(P), sc.ctypes.data_as(P))
    assert rc == 0
    k = n.value
    return tau[:k], w[:k], A[:k * (N + 1)].reshape(k, N + 1), sc


@pytest.mark.parametrize("N,L,tol", [(32, 8.0, 1e-12), (64, 10.0, 1e-6), (256, 10.0, 1e-12),
                                     (512, 6.0, 1e-6), (96, 16.0, 1e-9)])
def test_host_tables_match_oracle(shim, plan_cache, N, L, tol):
    tau, w, A, sc = host_tables(shim, N, L, tol)
    po = plan_cache(N, L, tol)
    assert len(tau) == len(po.gs.tau)
    assert sc[0] == pytest.approx(po.delta, rel=1e-15)
    assert sc[1] == po.eps
    assert np.max(np.abs(tau / po.gs.tau - 1)) <= 1e-14
    assert np.max(np.abs(w / po.gs.w - 1)) <= 1e-14
    assert np.max(np.abs(A - po.A)) <= 1e-13
    assert sc[2] == pytest.approx(po.C0, rel=1e-12)
    assert sc[3] == pytest.approx(po.C2, rel=1e-10)


def test_twiddles_exact(shim):
    for n in (8, 96, 512, 2048):
        out = np.zeros(2 * n)
        shim.shim_twiddles(n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        z = out[0::2] + 1j * out[1::2]
        import mpmath as mp
        mp.mp.dps = 30
        for e in (1, n // 8 + 1, n // 3, n - 1):
            ref = complex(mp.exp(-2j * mp.pi * e / n))
            assert abs(z[e] - ref) <= 1.2e-16
        # numpy evaluates 2 pi e / n in double: its own error reaches ~1e-15
        assert np.max(np.abs(z - np.exp(-2j * np.pi * np.arange(n) / n))) <= 4e-15


@pytest.mark.parametrize("N,L3,tol", [(32, (2.5, 2.75, 3.0), 1e-12), (64, (2.0, 4.0, 6.0), 1e-6),
                                      (48, (4.0, 4.0, 4.0), 1e-10), ((162, 162, 162), (2.0, 4.0, 6.0), 1e-12),
                                      ((16, 64, 12), (2.0, 4.0, 6.0), 1e-10), ((100, 40, 24), (1.0, 3.0, 3.0), 1e-6)])
def test_box_scalars_match_oracle(shim, N, L3, tol):
    """Box plans (Sec. 2 standardised form, n_q points on axis q): lambda, l_q, delta (the
    Sec. 3 heuristic's minimum over the axes), the Gaussian sum on [delta, 2 |l|] and the
    near-zone constants against the oracle's box plan."""
    from oracle import box
    P = ctypes.POINTER(ctypes.c_double)
    cap = 1000
    n = ctypes.c_int()
    tau, w, out = np.zeros(cap), np.zeros(cap), np.zeros(9)
    L = np.array(L3, dtype=np.float64)
    n3 = np.array(N if np.ndim(N) else (N, N, N), dtype=np.int32)
    assert shim.shim_box_scalars(n3.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), L.ctypes.data_as(P), tol, cap,
                                 ctypes.byref(n), tau.ctypes.data_as(P), w.ctypes.data_as(P),
                                 out.ctypes.data_as(P)) == 0
    k = n.value
    po = box.make_box_plan(tuple(int(v) for v in n3), [-v for v in L3], list(L3), tol)
    assert out[0] == po.lam and tuple(out[1:4]) == pytest.approx(po.l, rel=1e-15)
    assert out[4] == pytest.approx(po.delta, rel=1e-15) and out[5] == po.eps
    assert k == len(po.gs.tau)
    assert np.max(np.abs(tau[:k] / po.gs.tau - 1)) <= 1e-14
    assert np.max(np.abs(w[:k] / po.gs.w - 1)) <= 1e-14
    assert out[6] == pytest.approx(po.C0, rel=1e-12)
    assert out[7] == pytest.approx(po.C2, rel=1e-10)
    assert out[8] == pytest.approx(po.gs.r_max, rel=1e-15)
