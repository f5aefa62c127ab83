#!/usr/bin/env python
"""Throughput of the free-space Poisson solve: grid points per second per solve (N^3 / solve
time) on the 4-anisotropic-Gaussian workload (box [-10, 10]^3, N = 256, padded 512^3),
FP32 split-precision path, with the FP64 path, the rel-L2 and rel-l-infinity error of both
against the FP64 oracle, the per-pass HBM roofline, an end-to-end figure through the C-ABI
on host buffers, and the FP64 CPU oracle as a reported baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one solve (all five passes).  Inputs are resident in HBM before the timed
region; L2 (129 MB) is flushed by a 512 MB write between steps; each step is timed with
CUDA events on the launching stream.  With --gpus N > 1 (torchrun, one rank per GPU)
every rank solves its own density and rank 0 prints the aggregate (weak scaling; no
data-path collective, the solves are independent).  --impl reference times the oracle
(plain FP64 CPU implementation of the same discretisation) on the host cores.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT, L_BOX, TOL32, TOL64 = 256, 10.0, 1e-6, 1e-12
METRIC = "grid pts/s per solve (N^3/s) FP32 vs FP64 at stated rel-L2 err; % HBM roofline"
UNIT = "pts/s"
PASSES = ["x_forward", "y_forward", "z_fwd_symbol_inv", "y_inverse", "x_inverse"]
Z_FORMS = ["direct", "split", "warp"]
Y_FORMS = ["block", "warp"]
XY_FORMS = ["separate", "fused"]
# arithmetic of a plan: FP32; FP64 on the FP64 pipe; double-float (FP32 pairs, 48-bit significand)
ARITH_NAMES = {"f32": "fp32", "f64": "fp64", "df": "double-float (FP32 pairs, 48-bit significand)"}
Z_KERNELS = ["k_z_symbol", "k_z_split", "k_z_warp"]
# forms of the x and y passes: "block" (tiles staged in shared memory, columns or rows spread
# over a block) and "warp" (one warp or half-warp per column or row pair)
KERNEL_NAMES = ["k_x_forward", "k_col<fwd>", "k_z_symbol", "k_col<inv>", "k_x_inverse"]

# DRAM bytes per launch of the dominant kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by the hash of the kernel sources it was taken on; a
# source change makes the figure stale and it is reported as null.
NCU_TRAFFIC = {("6acf6ecbe1e2131e", "k_z_warp", 256): 358141440 + 236751872,
               ("6acf6ecbe1e2131e", "k_z_w512", 512): 3114766848 + 2138680576}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("fft_core.cuh", "passes.cuh", "passes_tma.cuh", "passes_zwarp.cuh", "passes_xy.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_1612_01799_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# Algorithmic bytes per grid point of each pass in FP32 (the per-unit figures of the five-pass
# design with the middle pass fused and the zero halves pruned, (N+1) taken as N): x forward
# reads rho (4) and writes the Hermitian half spectrum (8); y forward reads it (8) and writes
# the y-padded spectrum (16); the fused z pass reads and writes that (16 + 16); the inverse
# passes mirror the forward ones.  FP64 doubles every figure.  The z pass's symbol octant is
# this implementation's choice, not algorithmic traffic, and is reported on its own.
BYTES_PER_POINT_F32 = [12, 24, 32, 24, 12]


def pass_bytes(N, s):
    """Algorithmic DRAM bytes of each pass of one solve, s = bytes per real value."""
    return [b * (s // 4) * N ** 3 for b in BYTES_PER_POINT_F32]


def symbol_bytes(N, s):
    """Bytes of the symbol octant the z pass reads (N+1)^3 reals: implementation traffic."""
    return (N + 1) ** 3 * s


def pass_table(N, s, per_pass, xyform, names):
    """(pass, kernel, ms, algorithmic bytes) of the launches of one solve.  With the fused
    x-y form the forward x and y passes are one kernel (rho in, y-padded spectrum out: the x
    spectrum stays in L2) and so are the inverse y and x passes; their times sit in entries 0
    and 3."""
    b = pass_bytes(N, s)
    if not xyform:
        return [(PASSES[i], names[i], per_pass[i], b[i]) for i in range(5)]
    w1 = 8 * (s // 4) * N ** 3     # one write or one read of the x spectrum
    return [("xy_forward", "k_xy_fwd", per_pass[0], b[0] + b[1] - 2 * w1),
            (PASSES[2], names[2], per_pass[2], b[2]),
            ("yx_inverse", "k_yx_inv", per_pass[3], b[3] + b[4] - 2 * w1)]


def errors(u, ref):
    """rel-L2 and rel-l-infinity (the paper's E, Sec. 5) of u against ref, FP64."""
    import numpy as np
    u = np.asarray(u, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = u - ref
    return {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
            "rel_linf": float(np.abs(d).max() / np.abs(ref).max())}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(rank):
    """Seed of the density a rank solves: every rank its own density of the same family
    (independent solves, weak scaling; no data crosses ranks)."""
    return 2 + rank


def max_over_ranks(torch, value, device):
    """The largest of the ranks' values (every rank gets it): the job's time is its
    slowest rank's.  A single process returns its own value."""
    if not torch.distributed.is_available() or not torch.distributed.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, N, seconds):
    """Whole-job grid points per second: every rank solved N^3 points in `seconds`."""
    return world * N ** 3 / seconds


def oracle_reference(rho, N, L, tol):
    """The oracle as it stands on the host cores: setup untimed (as for the GPU plan), then one
    full FP64 solve of the workload, timed.  Returns (potential, pts/s, cores, seconds)."""
    from oracle import fft, gtensor, solver as osolver
    plan = gtensor.make_plan(N, L, tol)
    G = gtensor.symbol(plan)
    t0 = time.perf_counter()
    u = osolver.solve(rho, L, tol, plan=plan, G=G)
    dt = time.perf_counter() - t0
    return u, N ** 3 / dt, fft.threads(), dt


def oracle_lines(rho, N, L, tol, lines):
    """Sampled output lines u[z, y, :] of the oracle's real-space evaluation of the same
    discrete convolution (for grids whose FFT oracle would hold 17 GB)."""
    from oracle import direct, gtensor
    return direct.sample_lines(rho, gtensor.make_plan(N, L, tol), lines)


# Output lines (z, y) of the N = 512 accuracy sample: both tile edges of the column passes,
# the box faces and the interior, 8 distinct z planes.
LINES_512 = [(0, 0), (0, 511), (7, 8), (7, 300), (64, 63), (64, 64), (255, 256), (255, 100),
             (256, 255), (256, 17), (300, 1), (300, 400), (448, 447), (448, 0), (511, 511), (511, 256)]


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import fft, gtensor, solver as osolver
    from paper_1612_01799_gb300 import densities as D
    N = args.N
    w = D.config_aniso4(N=N)
    rho = w.sample()
    plan = gtensor.make_plan(N, w.L, TOL32)
    G = gtensor.symbol(plan)
    for _ in range(args.warmup):
        osolver.solve(rho, w.L, TOL32, plan=plan, G=G)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        osolver.solve(rho, w.L, TOL32, plan=plan, G=G)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = N ** 3 / (ms / 1e3)
    cores = fft.threads()
    sample = ("one full FP64 oracle solve per step of the N=%d workload (the oracle's own FFT of the "
              "padded %d^3 grid, symbol product, inverse FFT, crop); setup untimed" % (N, 2 * N))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(N, "f32"),  # the FP32 arm's workload and tolerance
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(N, dtype):
    return {"workload": "aniso4_N%d: 4 anisotropic normalised Gaussians (seed 2), box [-10,10]^3, "
                        "N=%d per axis, padded %d^3" % (N, N, 2 * N),
            "N": N, "L": L_BOX, "tol": TOL32 if dtype == "f32" else TOL64, "dtype": dtype,
            "l2": "flushed between steps (512 MB write)", "parallelism": "independent solves per GPU"}


def time_solves(torch, plan, rho_t, out_t, steps, warmup, flush, hold_s=0.0):
    """Per-step device times (ms) of whole solves and per-pass times, L2 flushed before
    every solve.  A step is one replay of a CUDA graph holding one poisson_solve (its five
    kernels, no host launches inside the timed span), timed with CUDA events on the
    replaying stream.  Each step is followed by one poisson_solve_timed (events between the
    passes) for the per-pass breakdown and the roofline's kernel times.  Untimed warm-up: at
    least `warmup` solves, continued for hold_s seconds so that the clock sampler records
    the GPU under this load right up to the timed steps."""
    cur = torch.cuda.current_stream()
    s = torch.cuda.Stream()
    s.wait_stream(cur)
    with torch.cuda.stream(s):
        plan.solve(rho_t, out=out_t, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.solve(rho_t, out=out_t, stream=s)
    t0, i = time.perf_counter(), 0
    while i < warmup or time.perf_counter() - t0 < hold_s:
        flush.zero_()
        g.replay()
        flush.zero_()
        plan.solve_timed(rho_t, out_t)
        i += 1
    torch.cuda.synchronize()
    totals, passes = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        g.replay()
        e1.record(cur)
        flush.zero_()
        ms = plan.solve_timed(rho_t, out_t)  # events on the launching stream, synchronised
        totals.append(e0.elapsed_time(e1))
        passes.append(ms)
    del g
    return totals, passes


def run_batched(torch, dev, steps, warmup, seed=4):
    """64 independent densities of uneven N (64..192), FP32: the batched call captured once in
    a CUDA graph; one step = one graph replay = 64 solves.  Inputs (0.74 GB) exceed L2."""
    import numpy as np
    from paper_1612_01799_gb300 import Plan, solve_batched
    from paper_1612_01799_gb300 import densities as D
    work = D.config_batch(count=64, seed=seed)
    counts = {}
    for w in work:
        counts[w.N] = counts.get(w.N, 0) + 1
    plans = {N: Plan(N, L_BOX, TOL32, "f32", max_batch=c) for N, c in counts.items()}
    rhos = [torch.from_numpy(w.gaussians.sample(w.N, w.L).astype(np.float32)).to(dev) for w in work]
    outs = [torch.empty_like(r) for r in rhos]
    pl = [plans[w.N] for w in work]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        solve_batched(pl, rhos, outs, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        solve_batched(pl, rhos, outs, stream=s)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    cur = torch.cuda.current_stream()
    ev[0].record(cur)
    for _ in range(steps):
        g.replay()
    ev[1].record(cur)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / steps
    for p in plans.values():
        p.last_status()
        p.close()
    pts = sum(w.N ** 3 for w in work)
    return {"value": pts / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "densities": len(work), "points_per_step": pts,
            "sizes": {str(k): v for k, v in sorted(counts.items())},
            "launch": "one CUDA graph replay per step: grouped launches per size (5 per size), "
                      "sizes concurrent on forked streams",
            "workload": "config_batch: 64 densities, N uniform over {64,96,128,160,192}, 1-6 "
                        "anisotropic Gaussians each (seed 4), box [-10,10]^3, FP32"}


def run_large(torch, dev, flush, steps, warmup, peak, N=512):
    """Config 3, the large single solve (padded 1024^3), FP32 with FP64 beside it: per-pass
    times against the HBM roofline.  Reported next to the headline, not as it."""
    import numpy as np
    from paper_1612_01799_gb300 import Plan
    from paper_1612_01799_gb300 import densities as D
    wl = D.config_bump8(N=N)
    sample = wl.sample()

    def one(dtype, tol, nsteps):
        rho = torch.from_numpy(sample.astype(np.float32 if dtype == "f32" else np.float64)).to(dev)
        with Plan(N, wl.L, tol, dtype) as plan:
            out = torch.empty_like(rho)
            totals, passes = time_solves(torch, plan, rho, out, nsteps, warmup, flush)
            plan.last_status()
            forms = {"z": Z_FORMS[plan.z_form], "y": Y_FORMS[plan.y_form], "x": Y_FORMS[plan.x_form],
                     "xy": XY_FORMS[plan.xy_form], "arith": ARITH_NAMES[plan.arith]}
            xyform = plan.xy_form
            u = out.view(N, N, N)
            got = np.stack([u[z, y, :].cpu().numpy() for z, y in LINES_512])
        err = errors(got, oracle_lines(sample, N, wl.L, tol, LINES_512))
        err["vs"] = ("FP64 oracle (real-space evaluation of the same discrete convolution) on %d "
                     "output lines of %d points" % (len(LINES_512), N))
        ms = statistics.mean(totals)
        per = [statistics.mean(p[i] for p in passes) for i in range(5)]
        rows = pass_table(N, 4 if dtype == "f32" else 8, per, xyform, [None] * 5)
        return {"value": N ** 3 / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": nsteps, "dtype": dtype,
                "passes": [{"pass": n, "ms": t, "GB_s": b / (t * 1e-3) / 1e9,
                            "frac": b / (t * 1e-3) / 1e9 / peak} for n, _, t, b in rows],
                "forms": forms, "accuracy": err}

    r = one("f32", TOL32, steps)
    r["f64"] = one("f64", TOL64, 3)
    r["workload"] = ("config_large: (1-r^2/16)^4 on r<4 plus 8 Gaussians (widths U[0.3,1], seed 3), box "
                     "[-6,6]^3, N=512 per axis, padded 1024^3, FP32 (FP64 beside it), L2 flushed between steps")
    return r


def run_selector(n_train=384, n_test=128, epochs=3000):
    """Config 5: train the grid selector on densities 0..n_train-1 (labels from the method's
    own FP32 solves against exact potentials), then the gain test on the next n_test:
    fixed N=512 FP64 vs the plain adaptive method vs network + a-posteriori check."""
    import tempfile as _tf
    from paper_1612_01799_gb300 import selector as S
    ws = S.Workspace()
    try:
        t0 = time.perf_counter()
        path = os.path.join(_tf.mkdtemp(), "selector.bin")
        info = S.fit(list(range(n_train)), ws, path, epochs=epochs)
        t_fit = time.perf_counter() - t0
        sel = S.Selector(path, capacity=n_test)
        res = S.gain_test(list(range(n_train, n_train + n_test)), ws, sel, tol=1e-6)
        sel.close()
    finally:
        ws.close()
    res["train"] = {"densities": n_train, "epochs": epochs, "final_loss": info["losses"][-1],
                    "seconds_labels_and_training": t_fit,
                    "check_accepts_eta_below": S.eta_threshold(info["calibration"], 1e-6)}
    res["workload"] = ("config_selector: densities of 1-8 Gaussians, widths log-uniform [0.2, 2], "
                       "charges U[-1,1], centres U[-2,2]^3 (seed 5), box [-16,16]^3, tol 1e-6 rel-L2")
    return res


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    from paper_1612_01799_gb300 import Plan, build
    from paper_1612_01799_gb300 import densities as D
    build.build()
    N = args.N
    dev = torch.device("cuda", torch.cuda.current_device())
    # Each rank solves its own density of the same family (weak scaling).
    wl = D.config_aniso4(N=N, seed=rank_seed(rank))
    rho64 = wl.sample()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    results = {}
    for dtype in ("f32", "f64"):
        tol = TOL32 if dtype == "f32" else TOL64
        plan = Plan(N, L_BOX, tol, dtype)
        if dtype == "f32" and args.z_form is not None:
            plan.z_form = Z_FORMS.index(args.z_form)
        if dtype == "f32" and args.y_form is not None:
            plan.y_form = Y_FORMS.index(args.y_form)
        if dtype == "f32" and args.x_form is not None:
            plan.x_form = Y_FORMS.index(args.x_form)
        if dtype == "f32" and args.xy_form is not None:
            plan.xy_form = XY_FORMS.index(args.xy_form)
        rho_t = torch.from_numpy(rho64.astype(plan.np_dtype)).to(dev)
        out_t = torch.empty_like(rho_t)
        steps = args.steps if dtype == "f32" else max(3, args.steps // 4)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev.index) if dtype == "f32" else None
        if sampler:
            sampler.__enter__()
        totals, passes = time_solves(torch, plan, rho_t, out_t, steps, args.warmup, flush,
                                     hold_s=1.0 if sampler else 0.0)
        if sampler:
            sampler.__exit__(None, None, None)
        torch.cuda.synchronize()
        ms = max_over_ranks(torch, statistics.mean(totals), dev)
        per_pass = [statistics.mean(p[i] for p in passes) for i in range(5)]
        results[dtype] = {"ms": ms, "per_pass": per_pass, "steps": steps, "z_form": plan.z_form, "y_form": plan.y_form, "x_form": plan.x_form,
                          "xy_form": plan.xy_form, "arith": plan.arith,
                          "clocks": sampler.summary() if sampler else None, "plan": plan,
                          "rho": rho_t, "out": out_t}

    # End to end through the C-ABI on pinned host buffers (H2D + solve + D2H each step).
    p32 = results["f32"]["plan"]
    host_in = torch.from_numpy(rho64.astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    for _ in range(max(1, args.warmup)):
        p32.solve_host(host_in, host_out)
    t0 = time.perf_counter()
    e2e_steps = args.steps
    for _ in range(e2e_steps):
        p32.solve_host(host_in, host_out)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(torch, e2e_s, dev)

    if rank == 0:
        peak, peak_kind = load_peaks()
        r32 = results["f32"]
        names = list(KERNEL_NAMES)
        names[2] = Z_KERNELS[r32["z_form"]]
        if r32["z_form"] == 2 and N == 512:
            names[2] = "k_z_w512"
        if r32["y_form"] == 1:
            names[1], names[3] = ("k_y_w512<fwd>", "k_y_w512<inv>") if N == 512 else ("k_y_warp<fwd>", "k_y_warp<inv>")
        if r32["x_form"] == 1:
            names[0], names[4] = "k_x_warp_fwd", "k_x_warp_inv"
        if results["f32"]["plan"]._lib.poisson_supported_n(N) == 2:   # the runtime-length forms
            names = ["k_any_x_fwd", "k_any_col<fwd>", "k_any_z", "k_any_col<inv>", "k_any_x_inv"]
        rows32 = pass_table(N, 4, r32["per_pass"], r32["xy_form"], names)
        gbs = [b / (t * 1e-3) / 1e9 for _, _, t, b in rows32]
        dom = max(range(len(rows32)), key=lambda i: rows32[i][2])
        src_hash = kernel_source_hash()
        traffic = NCU_TRAFFIC.get((src_hash, rows32[dom][1], N))
        r64 = results["f64"]
        rows64 = pass_table(N, 8, r64["per_pass"], r64["xy_form"], [None] * 5)
        gbs64 = [b / (t * 1e-3) / 1e9 for _, _, t, b in rows64]
        # Accuracy of the timed outputs against the FP64 oracle on the whole grid; the oracle's
        # solve with the FP32 plan's tolerance is also the CPU baseline (timed, setup untimed).
        acc, cpu = {}, None
        if not args.no_accuracy and world == 1:
            for dtype, tol in (("f32", TOL32), ("f64", TOL64)):
                ref, v, cores, dt = oracle_reference(rho64, N, L_BOX, tol)
                acc[dtype] = errors(results[dtype]["out"].cpu().numpy(), ref)
                acc[dtype]["vs"] = "FP64 oracle, whole %d^3 grid, plan tolerance %g" % (N, tol)
                if dtype == "f32":
                    cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": "1 full FP64 oracle solve of the same N=%d workload (its own "
                                     "FFT of the padded %d^3 grid, symbol product, inverse, crop; "
                                     "setup untimed), %.1f s" % (N, 2 * N, dt)}
                del ref
        line = {
            "metric": METRIC, "value": aggregate_rate(world, N, r32["ms"] * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": r32["steps"], "warmup": args.warmup, "ms_per_step": r32["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(N, "f32"),
            "accuracy": acc.get("f32"),
            "roofline": {"bound": "hbm", "achieved": gbs[dom], "peak": peak, "unit": "GB/s",
                         "frac": gbs[dom] / peak, "traffic": traffic,
                         "kernel": rows32[dom][1], "algorithmic_bytes": rows32[dom][3],
                         "bytes_per_point": rows32[dom][3] / N ** 3,
                         "symbol_bytes": symbol_bytes(N, 4) if rows32[dom][0] == PASSES[2] else 0,
                         "peak_source": peak_kind},
            "passes": [{"pass": n, "kernel": k, "ms": t, "GB_s": gbs[i], "frac": gbs[i] / peak}
                       for i, (n, k, t, _) in enumerate(rows32)],
            "f64": {"value": aggregate_rate(world, N, r64["ms"] * 1e-3), "ms_per_step": r64["ms"],
                    "steps": r64["steps"], "accuracy": acc.get("f64"), "arith": ARITH_NAMES[r64["arith"]],
                    "passes": [{"pass": n, "ms": t, "GB_s": gbs64[i], "frac": gbs64[i] / peak}
                               for i, (n, _, t, _) in enumerate(rows64)]},
            "e2e": {"value": aggregate_rate(world, N, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": N ** 3 * 4, "d2h_bytes_per_step": N ** 3 * 4},
            "gpu_launches": len(rows32) * r32["steps"],
            "step": "one replay of a CUDA graph holding one poisson_solve (its kernels, nothing else), "
                    "CUDA events around it on the replaying stream; per-pass times from a "
                    "poisson_solve_timed after each step (events between the passes)",
            "tuning": {"z_pass_f32": Z_FORMS[r32["z_form"]],
                       "z_pass_f64": Z_FORMS[results["f64"]["z_form"]],
                       "y_passes_f32": Y_FORMS[r32["y_form"]], "y_passes_f64": Y_FORMS[results["f64"]["y_form"]],
                       "x_passes_f32": Y_FORMS[r32["x_form"]], "x_passes_f64": Y_FORMS[results["f64"]["x_form"]],
                       "xy_passes_f32": XY_FORMS[r32["xy_form"]],
                       "how": ("pinned by --z-form/--y-form/--x-form/--xy-form"
                               if args.z_form or args.y_form or args.x_form or args.xy_form else
                               "timed at plan creation, cached per (device, N, dtype)")},
            "clocks": r32["clocks"],
        }
        if not args.no_large and world == 1:
            line["large"] = run_large(torch, dev, flush, max(3, args.steps // 2), args.warmup, peak)
        if not args.no_batched:
            line["batched"] = run_batched(torch, dev, max(3, args.steps // 2), args.warmup)
        if not args.no_selector and world == 1:
            line["selector"] = run_selector()
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    for r in results.values():
        r["plan"].close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_slab(args):
    """One solve split over the ranks as z slabs and ky lines (two all-to-all exchanges of
    the y-spectrum; strong scaling: the same N^3 solve on every N).  Rank 0 checks its own
    planes against the oracle and prints the line."""
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    from paper_1612_01799_gb300 import Plan, build, slab
    from paper_1612_01799_gb300 import densities as D
    build.build()
    N = args.N
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = D.config_aniso4(N=N)
    rho64 = wl.sample()
    z0, z1 = slab.bounds(N, world, rank)
    plan = Plan(N, L_BOX, TOL32, "f32")
    stages = slab.PlanStages(torch, plan)
    rho_slab = torch.from_numpy(np.ascontiguousarray(rho64[z0:z1]).astype(np.float32)).to(dev).reshape(-1)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        return slab.slab_solve(torch, stages, rho_slab, (N, N, N), rank, world)

    for _ in range(args.warmup):
        u = step()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        u = step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = max_over_ranks(torch, statistics.mean(times), dev)
    plan.last_status()
    if rank == 0:
        ref, _, _, _ = oracle_reference(rho64, N, L_BOX, TOL32) if not args.no_accuracy else (None, 0, 0, 0)
        acc = None
        if ref is not None:
            acc = errors(u.cpu().numpy().reshape(z1 - z0, N, N), ref[z0:z1])
            acc["vs"] = "FP64 oracle, rank 0's planes %d..%d of the %d^3 grid" % (z0, z1 - 1, N)
        line = {"metric": METRIC, "value": N ** 3 / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(workload_config(N, "f32"), parallelism="one solve over %d ranks: z slabs for the x "
                               "and y passes, ky lines for the z pass, two all-to-all exchanges" % world),
                "accuracy": acc, "gpu_launches": 5 * args.steps,
                "step": "forward x and y on the rank's planes, exchange, z pass on its lines, exchange, "
                        "inverse y and x; CUDA events on the rank's stream, max over ranks"}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--N", type=int, default=N_DEFAULT)
    ap.add_argument("--slab", action="store_true",
                    help="one solve split over the ranks (slab decomposition) instead of one solve per rank")
    ap.add_argument("--no-accuracy", "--no-cpu-baseline", dest="no_accuracy", action="store_true",
                    help="skip the oracle solves (accuracy figures and the CPU baseline); "
                         "--no-cpu-baseline is its older name")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the N=512 single-solve section")
    ap.add_argument("--no-selector", action="store_true")
    ap.add_argument("--z-form", choices=Z_FORMS, default=None,
                    help="pin the FP32 z-pass form (default: the plan's timed choice); for profiling")
    ap.add_argument("--y-form", choices=Y_FORMS, default=None,
                    help="pin the FP32 y-pass form (default: the plan's timed choice); for profiling")
    ap.add_argument("--x-form", choices=Y_FORMS, default=None,
                    help="pin the FP32 x-pass form (default: the plan's timed choice); for profiling")
    ap.add_argument("--xy-form", choices=XY_FORMS, default=None,
                    help="pin the FP32 x-y form, separate passes or fused (default: the plan's timed choice)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.slab:
        return run_slab(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
