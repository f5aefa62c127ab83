"""Batched solves: entries sharing a plan run as grouped launches (one per pass), groups of
different sizes run concurrently on forked streams; results must equal the single solves
bit for bit, also when the batched call is captured in a CUDA graph and replayed."""
import numpy as np
import pytest

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


def _inputs(torch, spec, dtype=np.float32):
    out = []
    for i, (N, seed) in enumerate(spec):
        rho = D.config_aniso4(N=N, seed=seed).gaussians.sample(N, 10.0).astype(dtype)
        out.append(torch.from_numpy(rho).cuda())
    return out


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batched_equals_single(torch_cuda, dtype):
    from paper_1612_01799_gb300 import Plan, solve_batched
    torch = torch_cuda
    npdt = np.float32 if dtype == "f32" else np.float64
    tol = 1e-6 if dtype == "f32" else 1e-12
    spec = [(64, 1), (96, 2), (64, 3), (64, 4), (96, 5), (64, 6), (64, 7), (32, 8)]
    rhos = _inputs(torch, spec, npdt)
    p64 = Plan(64, 10.0, tol, dtype, max_batch=4)      # 5 entries: a group of 4, then 1
    p96 = Plan(96, 10.0, tol, dtype, max_batch=2)
    p32 = Plan(32, 10.0, tol, dtype)
    plans = [{64: p64, 96: p96, 32: p32}[N] for N, _ in spec]
    outs = [torch.empty_like(r) for r in rhos]
    solve_batched(plans, rhos, outs)
    torch.cuda.synchronize()
    for p, r, o in zip(plans, rhos, outs):
        single = p.solve(r)
        torch.cuda.synchronize()
        assert torch.equal(single, o)
    for p in (p64, p96, p32):
        p.last_status()
        p.close()


def test_batched_graph_capture(torch_cuda):
    """The batched call captured once in a CUDA graph and replayed on new inputs."""
    from paper_1612_01799_gb300 import Plan, solve_batched
    torch = torch_cuda
    spec = [(64, 11), (128, 12), (64, 13), (160, 14), (128, 15)]
    rhos = _inputs(torch, spec)
    plans_by_n = {64: Plan(64, 10.0, 1e-6, "f32", max_batch=2), 128: Plan(128, 10.0, 1e-6, "f32", max_batch=2),
                  160: Plan(160, 10.0, 1e-6, "f32")}
    plans = [plans_by_n[N] for N, _ in spec]
    outs = [torch.empty_like(r) for r in rhos]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        solve_batched(plans, rhos, outs, stream=s)          # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        solve_batched(plans, rhos, outs, stream=s)
    new = _inputs(torch, [(N, seed + 100) for N, seed in spec])
    for r, n in zip(rhos, new):
        r.copy_(n)
    g.replay()
    torch.cuda.synchronize()
    for p, r, o in zip(plans, rhos, outs):
        assert torch.equal(p.solve(r), o)
    for p in plans_by_n.values():
        p.close()


@pytest.mark.parametrize("xyform", [0, 1])
def test_graph_capture_warp_forms(torch_cuda, xyform):
    """A batched solve at N = 256 in the warp forms of all passes (persistent kernels with
    TMA copies and mbarriers), separate or with the fused x-y passes (whose counters must
    be back at zero for every replay), captured in a CUDA graph and replayed twice on new
    inputs: equal to the direct solves bit for bit."""
    from paper_1612_01799_gb300 import Plan, solve_batched
    torch = torch_cuda
    spec = [(256, 21), (256, 22)]
    rhos = _inputs(torch, spec)
    with Plan(256, 10.0, 1e-6, "f32", max_batch=2) as p:
        p.z_form, p.y_form, p.x_form, p.xy_form = 2, 1, 1, xyform
        outs = [torch.empty_like(r) for r in rhos]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            solve_batched([p, p], rhos, outs, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            solve_batched([p, p], rhos, outs, stream=s)
        for seeds in ((31, 32), (41, 42)):
            for r, n in zip(rhos, _inputs(torch, [(256, seeds[0]), (256, seeds[1])])):
                r.copy_(n)
            g.replay()
            torch.cuda.synchronize()
            for r, o in zip(rhos, outs):
                assert torch.equal(p.solve(r), o)
        p.last_status()
