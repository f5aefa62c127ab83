"""Host logic of the multi-GPU path on CPU: two gloo ranks, as torchrun would start them.
Each rank solves its own density (no data crosses ranks), the job's time is the slowest
rank's, and the whole-job rate counts every rank's points; under N > 1 the oracle arm runs
on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    from paper_1612_01799_gb300 import densities as D
    dist.init_process_group("gloo", init_method="env://")
    w, r, _ = bench.dist_env()
    rho = D.config_aniso4(N=16, seed=bench.rank_seed(r)).gaussians.sample(16, 10.0)
    # every rank's density, gathered only to check they differ
    mine = torch.from_numpy(rho.ravel()[:64].copy())
    allr = [torch.empty_like(mine) for _ in range(w)]
    dist.all_gather(allr, mine)
    t = bench.max_over_ranks(torch, 1.0 + 2.0 * r, torch.device("cpu"))
    rate = bench.aggregate_rate(w, 16, t)
    with open(out % r, "w") as f:
        json.dump({"world": w, "rank": r, "max_t": t, "rate": rate,
                   "distinct": bool(not torch.equal(allr[0], allr[1]))}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / "rank%d.json")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(out % r)) for r in range(2)]
    for r, d in enumerate(res):
        assert d["world"] == 2 and d["rank"] == r
        assert d["max_t"] == 3.0                       # the slowest rank's time, on every rank
        assert d["rate"] == pytest.approx(2 * 16 ** 3 / 3.0)
        assert d["distinct"]                           # each rank solves its own density


def test_single_process_defaults(monkeypatch):
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(torch, 2.5, torch.device("cpu")) == 2.5
    assert bench.rank_seed(0) != bench.rank_seed(1)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--N", "16"], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""                      # rank 1: no work, no line
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--N", "16"], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    sys.path.insert(0, ROOT)
    import bench
    # the same workload, metric and direction as the CUDA arm's line
    assert line["config"] == bench.workload_config(16, "f32")
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"]
