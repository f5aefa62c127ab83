"""Python front of the C-ABI.  Argument marshalling only: every step of a solve runs in
the CUDA kernels of libgspoisson.so.  torch supplies device memory and streams."""
import ctypes

import numpy as np

from . import _lib

DTYPES = {"f32": _lib.F32, "f64": _lib.F64}


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def supported_n(N):
    """True if plans with N points per axis can be made (compiled or runtime-length forms)."""
    return bool(_lib.load().poisson_supported_n(int(N)))


class Plan:
    """A solve plan for the cube [-L, L]^3, or with L = (Lx, Ly, Lz) the box
    [-Lx, Lx] x [-Ly, Ly] x [-Lz, Lz], with N cell-centred points per axis, or with
    N = (nx, ny, nz) a box with n_q points on axis q (setup phase: Gaussian sum, G-tensor
    factors, near-zone constants, symbol table).  Arrays hold nz x ny x nx values, x
    fastest."""

    def __init__(self, N, L, tol, dtype="f32", max_batch=1):
        if dtype not in DTYPES:
            raise ValueError("dtype must be 'f32' or 'f64'")
        self.n = tuple(int(v) for v in N) if np.ndim(N) else (int(N),) * 3
        if len(self.n) != 3:
            raise ValueError("N is one count or three (nx, ny, nz)")
        self.N, self.tol, self.dtype = self.n[0], float(tol), dtype
        self.npoints = self.n[0] * self.n[1] * self.n[2]
        self.max_batch = int(max_batch)
        self._lib = _lib.load()
        self._h = ctypes.c_void_p()
        if np.ndim(N) and not np.ndim(L):
            L = (float(L),) * 3
        if np.ndim(L):
            self.box = tuple(float(v) for v in L)
            if len(self.box) != 3 or self.max_batch != 1:
                raise ValueError("a box takes three half-lengths and one density per solve")
            self.L = max(self.box)
            _lib.check(self._lib.poisson_plan_create_box_n(ctypes.byref(self._h), *self.n, *self.box, self.tol,
                                                           DTYPES[dtype]), "poisson_plan_create_box_n")
        else:
            self.box = None
            self.L = float(L)
            _lib.check(self._lib.poisson_plan_create_batched(ctypes.byref(self._h), self.N, self.L,
                                                             self.tol, DTYPES[dtype], self.max_batch),
                       "poisson_plan_create_batched")

    @property
    def handle(self):
        return self._h

    @property
    def torch_dtype(self):
        torch = _torch()
        return torch.float32 if self.dtype == "f32" else torch.float64

    @property
    def np_dtype(self):
        return np.float32 if self.dtype == "f32" else np.float64

    def _check_tensor(self, t, name):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
        if t.dtype != self.torch_dtype or t.numel() != self.npoints or not t.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor of nx ny nz = %d values"
                             % (name, self.torch_dtype, self.npoints))

    def solve(self, rho, out=None, stream=None):
        """u = U * rho on the device; rho, out: contiguous CUDA tensors of nx ny nz values."""
        self._check_tensor(rho, "rho")
        if out is None:
            out = _torch().empty_like(rho)
        self._check_tensor(out, "out")
        _lib.check(self._lib.poisson_solve(self._h, ctypes.c_void_p(rho.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
                   "poisson_solve")
        return out

    def solve_host(self, rho, out=None, stream=None):
        """The same solve on host memory (numpy array or CPU tensor; pinned is fastest)."""
        torch = _torch()
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho, dtype=self.np_dtype)
            if rho.size != self.npoints:
                raise ValueError("rho must hold nx ny nz values")
            if out is None:
                out = np.empty_like(rho)
            pin, pout = rho.ctypes.data, out.ctypes.data
        else:
            if rho.is_cuda or rho.dtype != self.torch_dtype or rho.numel() != self.npoints:
                raise ValueError("rho must be a CPU tensor of nx ny nz values of the plan's dtype")
            rho = rho.contiguous()
            if out is None:
                out = torch.empty_like(rho)
            pin, pout = rho.data_ptr(), out.data_ptr()
        _lib.check(self._lib.poisson_solve_host(self._h, ctypes.c_void_p(pin), ctypes.c_void_p(pout),
                                                _stream_handle(stream)), "poisson_solve_host")
        return out

    def solve_timed(self, rho, out, stream=None):
        """Solve and return the five per-pass device times (ms) from CUDA events."""
        self._check_tensor(rho, "rho")
        self._check_tensor(out, "out")
        ms = (ctypes.c_float * 5)()
        _lib.check(self._lib.poisson_solve_timed(self._h, ctypes.c_void_p(rho.data_ptr()),
                                                 ctypes.c_void_p(out.data_ptr()),
                                                 _stream_handle(stream), ms), "poisson_solve_timed")
        return list(ms)

    def last_status(self, stream=None):
        """Synchronise the stream and raise if a bounded device wait of a solve gave up."""
        _lib.check(self._lib.poisson_last_status(self._h, _stream_handle(stream)), "poisson_last_status")

    def info(self):
        d, e, c0, c2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int()
        ws, tb = ctypes.c_size_t(), ctypes.c_size_t()
        _lib.check(self._lib.poisson_plan_info(self._h, ctypes.byref(d), ctypes.byref(e), ctypes.byref(n),
                                               ctypes.byref(c0), ctypes.byref(c2), ctypes.byref(ws),
                                               ctypes.byref(tb)), "poisson_plan_info")
        return {"delta": d.value, "eps": e.value, "n_terms": n.value, "C0": c0.value, "C2": c2.value,
                "ws_bytes": ws.value, "table_bytes": tb.value}

    @property
    def z_form(self):
        """Form of the fused z pass in use (chosen by timing at plan creation): 0 length-2N
        transforms, 1 even/odd length-N split, 2 one warp per column pair."""
        v = ctypes.c_int()
        _lib.check(self._lib.poisson_plan_get_knob(self._h, _lib.KNOB_Z_FORM, ctypes.byref(v)),
                   "poisson_plan_get_knob")
        return v.value

    @z_form.setter
    def z_form(self, value):
        _lib.check(self._lib.poisson_plan_set_knob(self._h, _lib.KNOB_Z_FORM, int(value)), "poisson_plan_set_knob")

    @property
    def y_form(self):
        """Form of the y passes in use (chosen by timing at plan creation): 0 a column pair
        spread over a block, 1 one warp per column pair."""
        v = ctypes.c_int()
        _lib.check(self._lib.poisson_plan_get_knob(self._h, _lib.KNOB_Y_FORM, ctypes.byref(v)),
                   "poisson_plan_get_knob")
        return v.value

    @y_form.setter
    def y_form(self, value):
        _lib.check(self._lib.poisson_plan_set_knob(self._h, _lib.KNOB_Y_FORM, int(value)), "poisson_plan_set_knob")

    @property
    def x_form(self):
        """Form of the x passes in use (chosen by timing at plan creation): 0 a tile of rows
        staged in shared memory, 1 one half-warp per pair of rows."""
        v = ctypes.c_int()
        _lib.check(self._lib.poisson_plan_get_knob(self._h, _lib.KNOB_X_FORM, ctypes.byref(v)),
                   "poisson_plan_get_knob")
        return v.value

    @x_form.setter
    def x_form(self, value):
        _lib.check(self._lib.poisson_plan_set_knob(self._h, _lib.KNOB_X_FORM, int(value)), "poisson_plan_set_knob")

    @property
    def xy_form(self):
        """Whether the x and y passes run separately (0) or fused (1: one kernel per
        direction, the x spectrum handed over through an L2-resident ring of planes)."""
        v = ctypes.c_int()
        _lib.check(self._lib.poisson_plan_get_knob(self._h, _lib.KNOB_XY_FORM, ctypes.byref(v)),
                   "poisson_plan_get_knob")
        return v.value

    @xy_form.setter
    def xy_form(self, value):
        _lib.check(self._lib.poisson_plan_set_knob(self._h, _lib.KNOB_XY_FORM, int(value)), "poisson_plan_set_knob")

    @property
    def arith(self):
        """Arithmetic of the solve: "f32" for an FP32 plan; for an FP64 plan "f64" (the FP64
        pipe) or "df" (double-float: pairs of FP32 numbers on the FP32 pipe, 48-bit
        significand), chosen by timing at plan creation."""
        if self.dtype == "f32":
            return "f32"
        v = ctypes.c_int()
        _lib.check(self._lib.poisson_plan_get_knob(self._h, _lib.KNOB_ARITH, ctypes.byref(v)),
                   "poisson_plan_get_knob")
        return ("f64", "df")[v.value]

    @arith.setter
    def arith(self, value):
        code = {"f64": 0, "df": 1}.get(value)
        if code is None or self.dtype != "f64":
            raise ValueError("arith of an FP64 plan is 'f64' or 'df'")
        _lib.check(self._lib.poisson_plan_set_knob(self._h, _lib.KNOB_ARITH, code), "poisson_plan_set_knob")

    @property
    def correction(self):
        """Where the near-field correction enters: "fused" (C0 - C2 |kappa|^2 at every
        padded frequency) or "literal" (C0 rho + C2 Laplace(rho) of the N-periodic series,
        the paper's unpadded transform pair, placed at the all-even padded frequencies)."""
        v = ctypes.c_int()
        _lib.check(self._lib.poisson_plan_get_knob(self._h, _lib.KNOB_CORRECTION, ctypes.byref(v)),
                   "poisson_plan_get_knob")
        return ("fused", "literal")[v.value]

    @correction.setter
    def correction(self, value):
        code = {"fused": 0, "literal": 1}.get(value)
        if code is None:
            raise ValueError("correction must be 'fused' or 'literal'")
        _lib.check(self._lib.poisson_plan_set_knob(self._h, _lib.KNOB_CORRECTION, code), "poisson_plan_set_knob")

    def gauss_sum(self):
        n = self.info()["n_terms"]
        tau, w = np.empty(n), np.empty(n)
        _lib.check(self._lib.poisson_plan_gauss_sum(
            self._h, tau.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n), "poisson_plan_gauss_sum")
        return tau, w

    def axis_table(self):
        n = self.info()["n_terms"]
        a = np.empty((n, self.N + 1))
        _lib.check(self._lib.poisson_plan_axis_table(
            self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size), "poisson_plan_axis_table")
        return a

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.poisson_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_batched(plans, rhos, outs, stream=None):
    """Independent solves (uneven N allowed) through poisson_solve_batched.  Entries that
    share a plan are solved together (up to the plan's max_batch per launch sequence)."""
    n = len(plans)
    if not (len(rhos) == len(outs) == n):
        raise ValueError("plans, rhos and outs must have the same length")
    for p, r, o in zip(plans, rhos, outs):
        p._check_tensor(r, "rho")
        p._check_tensor(o, "out")
    H = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    R = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhos])
    O = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    lib = _lib.load()
    _lib.check(lib.poisson_solve_batched(n, H, R, O, _stream_handle(stream)), "poisson_solve_batched")
    return outs
