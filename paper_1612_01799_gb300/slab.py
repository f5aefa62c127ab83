"""Slab decomposition of one solve over the ranks of a torch.distributed group.

The x and y passes of the method's five (Sec. 2: the zero-padded transforms along each axis)
work plane by plane in z, and the fused z pass (forward transform, product with the symbol,
inverse) works line by line in (kx, ky).  So a solve splits over P ranks:

* rank r owns density planes [z0_r, z1_r) and y-spectrum lines [ky0_r, ky1_r) (balanced
  block bounds, ``bounds``);
* it runs the x and y forward passes of its planes (``poisson_slab_forward``);
* one all-to-all gives it every plane of its lines (``exchange`` on the spectrum buffer);
* it runs the z pass of its lines (``poisson_slab_z``);
* the reverse all-to-all gives it every line of its planes;
* it runs the y and x inverse passes of its planes (``poisson_slab_inverse``).

The exchanges are the only data-path collectives (``torch.distributed.all_to_all_single``,
NCCL between GPUs).  The stage functions come from an object with ``forward``, ``z``,
``inverse`` and ``spectrum``; ``PlanStages`` binds them to a plan's C-ABI calls.  Argument
marshalling only: every transform runs in the library's kernels.
"""
import ctypes

from . import _lib


def bounds(n, parts, r):
    """[lo, hi) of block r when n items are split into `parts` balanced blocks."""
    return n * r // parts, n * (r + 1) // parts


def exchange(torch, send_blocks, recv_blocks, group=None):
    """All-to-all among the group's ranks: send_blocks[s] goes to rank s and recv_blocks[s]
    is filled with what rank s sent here (views into the caller's buffers, any strides)."""
    dev = send_blocks[0].device
    send = torch.cat([b.reshape(-1) for b in send_blocks])
    rsz = [b.numel() for b in recv_blocks]
    recv = torch.empty(sum(rsz), dtype=send.dtype, device=dev)
    torch.distributed.all_to_all_single(recv, send, output_split_sizes=rsz,
                                        input_split_sizes=[b.numel() for b in send_blocks], group=group)
    o = 0
    for b, n in zip(recv_blocks, rsz):
        b.copy_(recv[o:o + n].view(b.shape))
        o += n


def slab_solve(torch, stages, rho_slab, n3, rank, world, group=None):
    """This rank's planes of the potential: stages.forward on its density planes, the
    exchange, stages.z on its lines, the reverse exchange, stages.inverse on its planes."""
    nx, ny, nz = n3
    if world > nz or world > 2 * ny:
        raise ValueError("more ranks than planes or lines")
    zb = [bounds(nz, world, s) for s in range(world)]
    kb = [bounds(2 * ny, world, s) for s in range(world)]
    (z0, z1), (k0, k1) = zb[rank], kb[rank]
    stages.forward(rho_slab, z0, z1 - z0)
    if world > 1:                                           # one rank owns every block
        w = stages.spectrum(0)                              # [z][ky][row]
        exchange(torch, [w[z0:z1, a:b] for a, b in kb], [w[a:b, k0:k1] for a, b in zb], group)
    stages.z(k0, k1 - k0)
    if world > 1:
        w = stages.spectrum(1)
        exchange(torch, [w[a:b, k0:k1] for a, b in zb], [w[z0:z1, a:b] for a, b in kb], group)
    return stages.inverse(z0, z1 - z0)


class _DeviceArray:
    """A device buffer the library owns, shown to torch through the CUDA array interface."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class PlanStages:
    """The slab stages of one plan (its first density) on the current stream."""

    def __init__(self, torch, plan):
        self.torch, self.plan, self.lib = torch, plan, _lib.load()
        self.nx, self.ny, self.nz = plan.n

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def forward(self, rho_slab, z0, nz):
        _lib.check(self.lib.poisson_slab_forward(self.plan.handle, ctypes.c_void_p(rho_slab.data_ptr()), z0, nz,
                                                 self._stream()), "poisson_slab_forward")

    def z(self, ky0, nky):
        _lib.check(self.lib.poisson_slab_z(self.plan.handle, ky0, nky, self._stream()), "poisson_slab_z")

    def inverse(self, z0, nz):
        u = self.torch.empty(nz * self.ny * self.nx, dtype=self.plan.torch_dtype, device="cuda")
        _lib.check(self.lib.poisson_slab_inverse(self.plan.handle, ctypes.c_void_p(u.data_ptr()), z0, nz,
                                                 self._stream()), "poisson_slab_inverse")
        return u

    def spectrum(self, which):
        """The plan's spectrum buffer `which` as a tensor [z][ky][row], row the floats (FP32,
        double-float) or doubles (FP64) of one ky row."""
        ptr, plane, row = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_size_t()
        _lib.check(self.lib.poisson_plan_spectrum(self.plan.handle, which, ctypes.byref(ptr), ctypes.byref(plane),
                                                  ctypes.byref(row)), "poisson_plan_spectrum")
        wide = self.plan.dtype == "f64" and self.plan.arith == "f64"
        size = 8 if wide else 4
        arr = _DeviceArray(ptr.value, (self.nz, 2 * self.ny, row.value // size), "<f8" if wide else "<f4")
        return self.torch.as_tensor(arr, device="cuda")
