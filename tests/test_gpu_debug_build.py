"""The debug build (libgspoisson_debug.so: the same sources with GSP_DEBUG, every shared
access of the pass kernels' access helpers and the runtime-length forms' computed indices
bounds-checked, a failed check skipping the access and setting a device-wide flag word).
A child process with POISSON_DEBUG=1 runs solves in every kernel family (compiled warp
and block forms at several sizes, the N = 512 warp forms, the double-float FP64 plan,
runtime-length sizes and a box with a different count per axis, a batched and a checked
solve); no check may fail (flags 0) and each potential must equal the release library's
within rounding.  The build's self-test shows the checks firing: its two out-of-range
predicates (evaluated without an access) set both flag bits."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, shape, dtype, (z, y, x) forms or None for the plan's own choice)
CASES = [
    ("warp64", 64, "f32", (2, 1, 1)),
    ("warp192", 192, "f32", (2, 1, 1)),
    ("warp256", 256, "f32", (2, 1, 1)),
    ("warp512", 512, "f32", (2, 1, 1)),
    ("block32", 32, "f32", (0, 0, 0)),
    ("df48", 48, "f64", None),
    ("any24", 24, "f32", None),
    ("anybox", (20, 24, 30), "f64", None),
]

CHILD = r'''
import json, os, sys
import numpy as np, torch
sys.path.insert(0, os.environ["GSP_ROOT"])
from paper_1612_01799_gb300 import Plan, solve_batched, _lib
from paper_1612_01799_gb300 import densities as D
cases = json.loads(os.environ["GSP_CASES"])
out_dir = os.environ["GSP_OUT"]
import ctypes
lib = _lib.load()
assert os.path.basename(lib._name) == "libgspoisson_debug.so", lib._name
def flags():
    f = ctypes.c_uint(0)
    rc = lib.poisson_debug_flags(ctypes.byref(f), None)
    assert rc == 0, rc
    return f.value
report = {}
assert flags() == 0
# the checks fire: the self-test's two failing predicates set both bits, and reading clears them
assert lib.poisson_debug_selftest(None) == 0
report["selftest"] = flags()
report["cleared"] = flags()
for name, shape, dtype, forms in cases:
    n = shape if isinstance(shape, int) else tuple(shape)
    N = n if isinstance(n, int) else n[0]
    rho = np.load(os.path.join(out_dir, name + "_rho.npy"))
    with Plan(n, 6.0, 1e-6 if dtype == "f32" else 1e-12, dtype) as p:
        if forms:
            p.z_form, p.y_form, p.x_form = forms
        t = torch.from_numpy(rho).cuda()
        u = p.solve(t)
        if name == "warp192":  # the batched driver and the checked (spectral-tail) variant
            u2 = torch.empty_like(t)
            solve_batched([p, p], [t, t], [u2, torch.empty_like(t)])
            eta, u3 = ctypes.c_double(), torch.empty_like(t)
            rc = lib.poisson_solve_checked(p.handle, ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(u3.data_ptr()),
                                           ctypes.byref(eta), None)
            assert rc == 0, rc
        torch.cuda.synchronize()
        np.save(os.path.join(out_dir, name + "_dbg.npy"), u.cpu().numpy())
    report[name] = flags()
print(json.dumps(report))
'''


@pytest.mark.gpu
def test_debug_build_checks_pass_and_results_match(tmp_path):
    torch = pytest.importorskip("torch")
    from paper_1612_01799_gb300 import Plan, build
    from paper_1612_01799_gb300 import densities as D
    build.build(debug=True)
    release = {}
    for name, shape, dtype, forms in CASES:
        n = shape if isinstance(shape, int) else tuple(shape)
        N = n if isinstance(n, int) else n[0]
        rho = D.config_aniso4(N=N, seed=21).gaussians.sample(n if isinstance(n, tuple) else N, 6.0) \
            if isinstance(n, int) else None
        if rho is None:
            rng = np.random.default_rng(21)
            rho = rng.standard_normal(n[::-1]).astype(np.float64)
        rho = np.ascontiguousarray(rho.astype(np.float32 if dtype == "f32" else np.float64))
        np.save(tmp_path / (name + "_rho.npy"), rho)
        with Plan(n, 6.0, 1e-6 if dtype == "f32" else 1e-12, dtype) as p:
            if forms:
                p.z_form, p.y_form, p.x_form = forms
            release[name] = p.solve(torch.from_numpy(rho).cuda()).cpu().numpy()
    env = dict(os.environ, POISSON_DEBUG="1", GSP_ROOT=ROOT, GSP_OUT=str(tmp_path), GSP_CASES=json.dumps(CASES))
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    report = json.loads(r.stdout.strip().splitlines()[-1])
    assert report.pop("selftest") == 3 and report.pop("cleared") == 0, report
    assert report == {name: 0 for name, *_ in CASES}, report
    for name, shape, dtype, forms in CASES:
        dbg = np.load(tmp_path / (name + "_dbg.npy"))
        ref = release[name]
        tol = 1e-6 if dtype == "f32" else 1e-13
        assert np.abs(dbg - ref).max() <= tol * np.abs(ref).max(), name
