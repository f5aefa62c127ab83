"""The slab decomposition of one solve on CPU: gloo ranks (world size 2 and 4, as torchrun
would start them) run the library's driver (paper_1612_01799_gb300.slab: block bounds, the
two all-to-all exchanges of the spectrum) with the stages restated on the CPU from the
oracle's steps (its own FFT along x and y on the rank's planes, along z with the padded
symbol on its lines), and the gathered potential must equal the single-rank oracle solve
element by element.  A planted mistake in the exchange (the rank's own block skipped) must
break it."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleStages:
    """The three stages of a slab rank on the CPU, in FP64, from the oracle's steps (Sec. 2:
    zero padding to 2 n_q per axis, unnormalised forward transforms, the padded symbol, the
    1 / (2 n_q)-normalised inverses, lambda^2, crop).  Spectrum buffers [z][ky][kx <= nx]
    complex, shown to the exchange as float64 [z][ky][2 (nx + 1)]."""

    def __init__(self, torch, N, L, tol):
        from oracle import gtensor
        self.torch, self.N = torch, N
        self.plan = gtensor.make_plan(N, L, tol)
        self.G = gtensor.symbol(self.plan)                 # [kz][ky][kx], padded (2N)^3
        self.buf = [torch.zeros((N, 2 * N, N + 1, 2), dtype=torch.float64) for _ in range(2)]

    def _c(self, which):
        return self.buf[which].numpy().view(np.complex128)[..., 0]

    def spectrum(self, which):
        return self.buf[which].view(self.N, 2 * self.N, 2 * (self.N + 1))

    def forward(self, rho_slab, z0, nz):
        from oracle import fft
        N = self.N
        a = np.zeros((nz, 2 * N, 2 * N), np.complex128)
        a[:, :N, :N] = rho_slab.numpy().reshape(nz, N, N)
        fft.transform_axis(a, 2, -1)
        fft.transform_axis(a, 1, -1)
        self._c(0)[z0:z0 + nz] = a[:, :, :N + 1]

    def z(self, ky0, nky):
        from oracle import fft
        N = self.N
        a = np.zeros((2 * N, nky, N + 1), np.complex128)
        a[:N] = self._c(0)[:, ky0:ky0 + nky]
        fft.transform_axis(a, 0, -1)
        a *= self.G[:, ky0:ky0 + nky, :N + 1]
        fft.transform_axis(a, 0, +1)
        self._c(1)[:, ky0:ky0 + nky] = a[:N] / (2 * N)

    def inverse(self, z0, nz):
        from oracle import fft
        N = self.N
        a = np.ascontiguousarray(self._c(1)[z0:z0 + nz])   # [z][ky][kx <= N]
        fft.transform_axis(a, 1, +1)
        half = a[:, :N, :] / (2 * N)
        full = np.zeros((nz, N, 2 * N), np.complex128)     # the Hermitian spectrum along x
        full[:, :, :N + 1] = half
        full[:, :, N + 1:] = np.conj(half[:, :, 1:N][:, :, ::-1])
        fft.transform_axis(full, 2, +1)
        u = self.plan.lam ** 2 * full.real[:, :, :N] / (2 * N)
        return self.torch.from_numpy(np.ascontiguousarray(u).ravel())


def _rank_main(rank, world, port, out, N, plant):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ["ORACLE_THREADS"] = "1"
    import torch
    import torch.distributed as dist
    from paper_1612_01799_gb300 import densities as D, slab
    from test_slab_host import OracleStages
    dist.init_process_group("gloo", init_method="env://")
    L, tol = 8.0, 1e-10
    rho = D.config_aniso4(N=N, seed=9).gaussians.sample(N, L)
    z0, z1 = slab.bounds(N, world, rank)
    stages = OracleStages(torch, N, L, tol)
    if plant:
        real = slab.exchange

        def skip_own(torch_, send, recv, group=None):
            saved = [r.clone() for r in recv]
            real(torch_, send, recv, group)
            recv[rank].copy_(torch_.zeros_like(saved[rank]))
        slab.exchange = skip_own
    u = slab.slab_solve(torch, stages, torch.from_numpy(rho[z0:z1].ravel().copy()), (N, N, N), rank, world)
    np.save(out % rank, u.numpy().reshape(z1 - z0, N, N))
    dist.barrier()
    dist.destroy_process_group()


def run_world(tmp_path, world, N, plant=False):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    out = str(tmp_path / ("u_%d_%d_%%d.npy" % (world, N)))
    mp.start_processes(_rank_main, args=(world, _free_port(), out, N, plant), nprocs=world, start_method="spawn",
                       join=True)
    return np.concatenate([np.load(out % r) for r in range(world)])


def oracle_solve(N):
    from oracle import solver
    from paper_1612_01799_gb300 import densities as D
    L, tol = 8.0, 1e-10
    rho = D.config_aniso4(N=N, seed=9).gaussians.sample(N, L)
    return solver.solve(rho, L, tol)


def test_bounds_cover_every_item_once():
    sys.path.insert(0, ROOT)
    from paper_1612_01799_gb300 import slab
    for n in (8, 13, 64, 100):
        for P in (1, 2, 3, 4, 7):
            b = [slab.bounds(n, P, r) for r in range(P)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(P - 1))
            assert max(h - l for l, h in b) - min(h - l for l, h in b) <= 1


@pytest.mark.parametrize("world,N", [(2, 32), (4, 32), (2, 16), (4, 12)])
def test_gloo_ranks_equal_single_rank_oracle(tmp_path, world, N):
    u = run_world(tmp_path, world, N)
    ref = oracle_solve(N)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= 1e-13
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_planted_exchange_mistake_is_caught(tmp_path):
    u = run_world(tmp_path, 2, 16, plant=True)
    ref = oracle_solve(16)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) > 1e-3
