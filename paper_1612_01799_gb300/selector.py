"""Learned grid selection: train and use the network that picks N for a density.

Every computation runs in the library's kernels (density sampling, solves, the spectral
tail check, exact potentials, errors, features, MLP forward/backward/Adam); this module
only orders the calls and keeps the bookkeeping.

Pipeline for a density:
  1. sample it on the 32^3 grid and compute 64 radial power-spectrum features;
  2. the network predicts log10 of the relative L2 error of an FP32 solve at each
     candidate N; take the smallest N whose prediction is below log10(tol) - margin;
  3. solve at N with the a-posteriori check: eta (the outer-shell energy fraction of the
     padded spectrum) mapped to an error estimate by a monotone calibration fitted on the
     training data; if the estimate exceeds tol, move to the next candidate and solve again.

The plain method (start at the smallest candidate and refine with the same check) is the
fallback, and the yardstick for what the network saves.
"""
import ctypes
import json
import math
import time

import numpy as np

from . import _lib
from . import densities as D

CANDIDATES = (32, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512)
NPTS = 1024          # grid points per (density, N) where the error is measured
BOX = 16.0           # selector workload box [-16, 16]^3
FEATURES = 64


def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def gaussian_params(g):
    """(ng, 7) records (cx, cy, cz, sx, sy, sz, q) of a GaussianSum, FP64, C order."""
    rec = np.concatenate([g.centres, g.sigmas, g.charges[:, None]], axis=1)
    return np.ascontiguousarray(rec, dtype=np.float64)


class Workspace:
    """Device buffers and plans reused across densities."""

    def __init__(self, candidates=CANDIDATES, tol_plan=1e-6, dtype="f32"):
        from .api import Plan
        torch = _torch()
        self.lib = _lib.load()
        self.candidates = tuple(candidates)
        self.dtype = dtype
        self.plans = {N: Plan(N, BOX, tol_plan, dtype) for N in self.candidates}
        tdt = torch.float32 if dtype == "f32" else torch.float64
        nmax = max(self.candidates)
        self.rho = torch.empty(nmax ** 3, dtype=tdt, device="cuda")
        self.u = torch.empty(nmax ** 3, dtype=tdt, device="cuda")
        self.idx = torch.empty(NPTS * 3, dtype=torch.int32, device="cuda")
        self.ref = torch.empty(NPTS, dtype=torch.float64, device="cuda")
        self.s32 = torch.empty(32 ** 3, dtype=torch.float32, device="cuda")
        self.bplans = {}

    def batch_plan(self, N):
        """A plan of N whose workspace holds several densities (made on first use; about
        10 GB of workspace per size at most)."""
        from .api import Plan
        if N not in self.bplans:
            per = 40 * N ** 3 * (4 if self.dtype == "f32" else 8) // 4   # bytes of workspace per density
            mb = int(max(1, min(16, (10 << 30) // per)))
            self.bplans[N] = Plan(N, BOX, self.plans[N].tol, self.dtype, max_batch=mb)
        return self.bplans[N]

    def close(self):
        for p in list(self.plans.values()) + list(self.bplans.values()):
            p.close()

    def sample(self, params, N, out, dtype_code):
        P = params.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _lib.check(self.lib.poisson_sample_gaussians(N, BOX, params.shape[0], P, dtype_code, _ptr(out), _stream()),
                   "poisson_sample_gaussians")

    def solve_error(self, params, N, seed):
        """FP relative L2 error (against the exact potential at NPTS seeded grid points) and
        the spectral-tail indicator eta of one checked solve at N."""
        torch = _torch()
        code = 0 if self.dtype == "f32" else 1
        n3 = N ** 3
        rho, u = self.rho[:n3], self.u[:n3]
        self.sample(params, N, rho, code)
        eta = ctypes.c_double()
        plan = self.plans[N]
        _lib.check(self.lib.poisson_solve_checked(plan.handle, _ptr(rho), _ptr(u), ctypes.byref(eta), _stream()),
                   "poisson_solve_checked")
        err = self.error_at_points(params, N, u, seed)
        return err, eta.value

    def error_at_points(self, params, N, u, seed):
        torch = _torch()
        rng = np.random.default_rng([seed, N])
        pts = rng.integers(0, N, size=(NPTS, 3)).astype(np.int32)
        self.idx.copy_(torch.from_numpy(pts.ravel()))
        P = params.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _lib.check(self.lib.poisson_gaussian_potential(N, BOX, params.shape[0], P, NPTS, _ptr(self.idx),
                                                       _ptr(self.ref), _stream()), "poisson_gaussian_potential")
        e = ctypes.c_double()
        code = 0 if u.dtype == torch.float32 else 1
        _lib.check(self.lib.poisson_compare_points(_ptr(u), code, N, NPTS, _ptr(self.idx), _ptr(self.ref),
                                                   ctypes.byref(e), _stream()), "poisson_compare_points")
        return e.value

    def features(self, params_list):
        """count x 64 features of the densities' 32^3 samples (device tensor)."""
        torch = _torch()
        n = len(params_list)
        s = torch.empty(n * 32 ** 3, dtype=torch.float32, device="cuda")
        for i, p in enumerate(params_list):
            self.sample(p, 32, s[i * 32 ** 3:(i + 1) * 32 ** 3], 0)
        f = torch.empty(n * FEATURES, dtype=torch.float32, device="cuda")
        _lib.check(self.lib.poisson_features32(_ptr(s), n, _ptr(f), _stream()), "poisson_features32")
        return f.view(n, FEATURES), s


def density(i, seed=5):
    return D.config_selector(i, seed=seed, N=64).gaussians


def make_dataset(indices, ws, log_floor=-9.0):
    """Features, log10 errors and log10 eta over the candidate grids for densities `indices`."""
    params = [gaussian_params(density(i)) for i in indices]
    feats, _ = ws.features(params)
    K = len(ws.candidates)
    lerr = np.zeros((len(indices), K))
    leta = np.zeros((len(indices), K))
    for a, (i, p) in enumerate(zip(indices, params)):
        for k, N in enumerate(ws.candidates):
            err, eta = ws.solve_error(p, N, seed=1000 + i)
            lerr[a, k] = max(math.log10(max(err, 1e-300)), log_floor)
            leta[a, k] = math.log10(max(eta, 1e-300))
    return feats.cpu().numpy(), lerr, leta


class Network:
    """MLP parameters on the device plus the kernels' training loop."""

    def __init__(self, K, seed=0):
        torch = _torch()
        self.lib = _lib.load()
        self.K = K
        self.n = self.lib.poisson_mlp_nparams(K)
        rng = np.random.default_rng(seed)
        parts = []
        for fan_in, fan_out in ((64, 64), (64, 64), (64, 64), (64, K)):
            lim = math.sqrt(6.0 / (fan_in + fan_out))
            parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
            parts.append(np.zeros(fan_out))
        p = np.concatenate(parts).astype(np.float32)
        assert p.size == self.n
        self.params = torch.from_numpy(p).cuda()
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.mean = torch.zeros(FEATURES, device="cuda")
        self.std = torch.ones(FEATURES, device="cuda")

    def forward(self, x, acts=None):
        torch = _torch()
        y = torch.empty(x.shape[0] * self.K, dtype=torch.float32, device="cuda")
        _lib.check(self.lib.poisson_mlp_forward(_ptr(self.params), self.K, _ptr(x), x.shape[0], _ptr(y),
                                                _ptr(acts) if acts is not None else None, _stream()),
                   "poisson_mlp_forward")
        return y.view(x.shape[0], self.K)

    def gradient(self, x, t):
        """Loss and parameter gradient (into self.grad) for inputs x and targets t."""
        torch = _torch()
        B = x.shape[0]
        acts = torch.empty(B * 3 * 64, dtype=torch.float32, device="cuda")
        y = self.forward(x, acts)
        dy = torch.empty_like(y)
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        _lib.check(self.lib.poisson_mlp_loss(_ptr(y), _ptr(t), y.numel(), _ptr(dy), _ptr(loss), _stream()),
                   "poisson_mlp_loss")
        _lib.check(self.lib.poisson_mlp_backward(_ptr(self.params), self.K, _ptr(x), _ptr(acts), B, _ptr(dy),
                                                 _ptr(self.grad), _stream()), "poisson_mlp_backward")
        return loss

    def train(self, x, t, epochs=3000, lr=2e-3):
        """Full-batch Adam on standardised inputs.  Returns the loss before the first step
        and every 500 steps after it (and at the last step)."""
        losses = []
        for step in range(1, epochs + 1):
            loss = self.gradient(x, t)
            _lib.check(self.lib.poisson_mlp_adam(_ptr(self.params), _ptr(self.grad), _ptr(self.m), _ptr(self.v),
                                                 self.n, ctypes.c_float(lr), ctypes.c_float(0.9),
                                                 ctypes.c_float(0.999), ctypes.c_float(1e-8), step, _stream()),
                       "poisson_mlp_adam")
            if step == 1 or step % 500 == 0 or step == epochs:
                losses.append(float(loss.item()))
        return losses


def calibrate(leta, lerr, quantile=0.98, width=0.25, min_count=4):
    """Monotone map from log10(eta) to a log10 error bound, as a step function.

    The training pairs are binned by log10(eta) (bins `width` wide); each bin's bound is the
    `quantile` of its log10 errors (its maximum when it holds fewer than `min_count` pairs),
    and a running maximum from small to large eta makes the map non-decreasing.  A straight
    line would not do: the error stops falling at the FP32 round-off floor while eta keeps
    falling, which flattens a fitted slope until no eta passes the check.
    Returns {"x0": left edge of bin 0, "width": bin width, "bound": [log10 bound per bin]}."""
    x, y = np.ravel(leta), np.ravel(lerr)
    keep = np.isfinite(x) & np.isfinite(y) & (x > -29)
    x, y = x[keep], y[keep]
    if x.size == 0:
        raise ValueError("calibrate: no finite (eta, error) pairs")
    x0 = math.floor(x.min() / width) * width
    nb = int(math.floor((x.max() - x0) / width)) + 1
    b = np.minimum(((x - x0) / width).astype(int), nb - 1)
    bound, run = [], -math.inf
    for i in range(nb):
        yi = y[b == i]
        if yi.size:
            q = float(np.quantile(yi, quantile)) if yi.size >= min_count else float(yi.max())
            run = max(run, q)
        bound.append(run)
    return {"x0": float(x0), "width": float(width), "bound": bound}


def calibrated_bound(cal, eta):
    """log10 error bound for eta under a calibration from `calibrate` (+inf beyond the
    largest eta seen in training, the bin-0 bound below the smallest)."""
    x = math.log10(max(eta, 1e-300))
    i = int(math.floor((x - cal["x0"]) / cal["width"]))
    if i >= len(cal["bound"]):
        return math.inf
    return cal["bound"][max(i, 0)]


def eta_threshold(cal, tol):
    """Largest eta (a bin's upper edge) that the check accepts at tol, or 0 if none."""
    ok = [i for i, b in enumerate(cal["bound"]) if b <= math.log10(tol)]
    return 10.0 ** (cal["x0"] + (ok[-1] + 1) * cal["width"]) if ok else 0.0


def save(path, net, candidates, margin, cal):
    torch = _torch()
    with open(path, "wb") as f:
        f.write(b"GSPSEL01")
        f.write(np.int32(len(candidates)).tobytes())
        f.write(np.asarray(candidates, np.int32).tobytes())
        f.write(np.float32(margin).tobytes())
        f.write(net.mean.cpu().numpy().astype(np.float32).tobytes())
        f.write(net.std.cpu().numpy().astype(np.float32).tobytes())
        f.write(net.params.cpu().numpy().astype(np.float32).tobytes())
    with open(path + ".json", "w") as f:
        json.dump({"candidates": list(candidates), "margin": margin, "calibration": cal}, f)


class Selector:
    """A trained selector loaded through the C-ABI."""

    def __init__(self, path, capacity=512):
        self.lib = _lib.load()
        self.h = ctypes.c_void_p()
        _lib.check(self.lib.poisson_selector_load(ctypes.byref(self.h), path.encode(), capacity),
                   "poisson_selector_load")
        with open(path + ".json") as f:
            meta = json.load(f)
        self.candidates = tuple(meta["candidates"])
        self.cal = meta["calibration"]

    def select(self, samples32, count, tol):
        N = (ctypes.c_int * count)()
        pred = (ctypes.c_float * (count * len(self.candidates)))()
        _lib.check(self.lib.poisson_select_n(self.h, _ptr(samples32), count, tol, N, pred, _stream()),
                   "poisson_select_n")
        return list(N), np.frombuffer(pred, dtype=np.float32).reshape(count, -1)

    def check(self, eta, tol):
        """The a-posteriori acceptance test: calibrated error bound of eta within tol."""
        return calibrated_bound(self.cal, eta) <= math.log10(tol)

    def close(self):
        if self.h.value:
            self.lib.poisson_selector_destroy(self.h)
            self.h = ctypes.c_void_p()


def fit(train_indices, ws, path, epochs=3000, lr=2e-3, margin=0.3, seed=0):
    """Generate the training data with the method itself, train the network on the GPU,
    fit the check's calibration and write the selector file."""
    torch = _torch()
    feats, lerr, leta = make_dataset(train_indices, ws)
    mean = feats.mean(0)
    std = np.maximum(feats.std(0), 1e-3)
    K = len(ws.candidates)
    net = Network(K, seed=seed)
    net.mean.copy_(torch.from_numpy(mean.astype(np.float32)))
    net.std.copy_(torch.from_numpy(std.astype(np.float32)))
    x = torch.from_numpy(((feats - mean) / std).astype(np.float32)).cuda().contiguous()
    t = torch.from_numpy(lerr.astype(np.float32)).cuda().contiguous()
    losses = net.train(x, t, epochs=epochs, lr=lr)
    cal = calibrate(leta, lerr)
    save(path, net, ws.candidates, margin, cal)
    return {"losses": losses, "calibration": cal, "train_densities": len(train_indices),
            "label_mean_log10_err": float(lerr.mean())}


def _solve_until_checked(ws, sel, params, start_k, tol):
    """Solve at candidates from index start_k up until the calibrated check passes.
    Returns (N, index of N, number of solves)."""
    k = start_k
    while True:
        N = ws.candidates[k]
        n3 = N ** 3
        ws.sample(params, N, ws.rho[:n3], 0 if ws.dtype == "f32" else 1)
        eta = ctypes.c_double()
        _lib.check(ws.lib.poisson_solve_checked(ws.plans[N].handle, _ptr(ws.rho[:n3]), _ptr(ws.u[:n3]),
                                                ctypes.byref(eta), _stream()), "poisson_solve_checked")
        if sel.check(eta.value, tol) or k == len(ws.candidates) - 1:
            return N, k, k - start_k + 1
        k += 1


def solve_batched_until_checked(ws, sel, params, start_ks, tol):
    """The same refinement for many densities at once: the densities at the same candidate
    solve together (poisson_solve_checked_batched, up to the plan's max_batch per call), and
    those whose check fails move on together.  Returns one (N, index, solves) per density."""
    torch = _torch()
    code = 0 if ws.dtype == "f32" else 1
    tdt = torch.float32 if ws.dtype == "f32" else torch.float64
    last = len(ws.candidates) - 1
    pending = dict(enumerate(start_ks))
    solves = [0] * len(params)
    out = [None] * len(params)
    while pending:
        groups = {}
        for i, k in pending.items():
            groups.setdefault(k, []).append(i)
        pending = {}
        for k in sorted(groups):
            N = ws.candidates[k]
            plan = ws.batch_plan(N)
            members = groups[k]
            for c0 in range(0, len(members), plan.max_batch):
                chunk = members[c0:c0 + plan.max_batch]
                n = len(chunk)
                rho = torch.empty((n, N ** 3), dtype=tdt, device="cuda")
                u = torch.empty_like(rho)
                for j, i in enumerate(chunk):
                    ws.sample(params[i], N, rho[j], code)
                rp = (ctypes.c_void_p * n)(*[rho[j].data_ptr() for j in range(n)])
                up = (ctypes.c_void_p * n)(*[u[j].data_ptr() for j in range(n)])
                eta = (ctypes.c_double * n)()
                _lib.check(ws.lib.poisson_solve_checked_batched(plan.handle, n, rp, up, eta, _stream()),
                           "poisson_solve_checked_batched")
                for j, i in enumerate(chunk):
                    solves[i] += 1
                    if sel.check(eta[j], tol) or k == last:
                        out[i] = (N, k, solves[i])
                    else:
                        pending[i] = k + 1
    return out


def gain_test(test_indices, ws, sel, tol=1e-6, start_N=64, fixed_N=512):
    """Cost and accuracy of three ways to meet `tol` on the test densities:
    (i) a fixed N = fixed_N FP64 solve of every density, (ii) the plain method: start at
    start_N and refine with the a-posteriori check, (iii) the network's N, refined with the
    same check.  (ii) and (iii) solve the densities at the same N together (batched checked
    solves), so their difference is the network's; both in FP32."""
    torch = _torch()
    from .api import Plan
    params = [gaussian_params(density(i)) for i in test_indices]
    res = {}
    # Batched plans and their workspaces exist before the timed runs.
    for N in ws.candidates:
        ws.batch_plan(N)
    # (iii) network + check
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, s32 = ws.features(params)
    Ns, _ = sel.select(s32, len(params), tol)
    chosen3 = solve_batched_until_checked(ws, sel, params, [ws.candidates.index(n) for n in Ns], tol)
    torch.cuda.synchronize()
    t3 = time.perf_counter() - t0
    # (ii) plain method + check
    t0 = time.perf_counter()
    chosen2 = solve_batched_until_checked(ws, sel, params, [ws.candidates.index(start_N)] * len(params), tol)
    torch.cuda.synchronize()
    t2 = time.perf_counter() - t0
    # accuracy of the grids each strategy ended on (untimed)
    def errors(chosen):
        out = []
        for i, p, (N, _, _) in zip(test_indices, params, chosen):
            out.append(ws.solve_error(p, N, seed=5000 + i)[0])
        return np.array(out)
    e3, e2 = errors(chosen3), errors(chosen2)
    # (i) fixed N, FP64 plan (its timed arithmetic), every test density: timed, then its errors
    with Plan(fixed_N, BOX, 1e-12, "f64") as p64:
        rho = torch.empty(fixed_N ** 3, dtype=torch.float64, device="cuda")
        u = torch.empty_like(rho)
        ws.sample(params[0], fixed_N, rho, 1)
        p64.solve(rho, u)                      # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for pr in params:
            ws.sample(pr, fixed_N, rho, 1)
            p64.solve(rho, u)
        torch.cuda.synchronize()
        t1 = time.perf_counter() - t0
        e1 = np.array([ws.error_at_points(pr, fixed_N, (ws.sample(pr, fixed_N, rho, 1), p64.solve(rho, u))[1],
                                          seed=5000 + i)
                       for i, pr in zip(test_indices, params)])
        arith = p64.arith

    def summary(t, e, chosen):
        d = {"seconds": t, "met_tol": float(np.mean(e <= tol)), "median_err": float(np.median(e)),
             "max_err": float(np.max(e))}
        if chosen is not None:
            d["mean_N"] = float(np.mean([c[0] for c in chosen]))
            d["solves_per_density"] = float(np.mean([c[2] for c in chosen]))
        return d
    res["fixed_N%d_f64" % fixed_N] = summary(t1, e1, None)
    res["fixed_N%d_f64" % fixed_N]["timed_densities"] = len(params)
    res["fixed_N%d_f64" % fixed_N]["arith"] = arith
    res["plain_adaptive_from_N%d_f32_batched" % start_N] = summary(t2, e2, chosen2)
    res["network_plus_check_f32_batched"] = summary(t3, e3, chosen3)
    res["network_first_guess_kept"] = float(np.mean([c[0] == n for c, n in zip(chosen3, Ns)]))
    res["speedup_vs_fixed"] = t1 / t3
    res["speedup_vs_plain"] = t2 / t3
    res["densities"] = len(params)
    res["tol"] = tol
    return res
