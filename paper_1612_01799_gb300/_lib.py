"""ctypes binding of libgspoisson.so: signatures of include/poisson.h, nothing more.

With POISSON_DEBUG=1 in the environment the binding loads the debug build instead
(libgspoisson_debug.so: the same sources with bounds checks, built by
build.build(debug=True))."""
import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgspoisson.so")
DEBUG_LIB_PATH = os.path.join(PKG, "libgspoisson_debug.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "poisson.h")

F32, F64 = 0, 1
OK = 0
ERRORS = {-1: "POISSON_ERR_ARG", -2: "POISSON_ERR_ALLOC", -3: "POISSON_ERR_CUDA",
          -4: "POISSON_ERR_UNSUPPORTED", -5: "POISSON_ERR_TIMEOUT", -6: "POISSON_ERR_NUMERIC"}

_lock = threading.Lock()
_lib = None

c_int, c_double, c_size_t, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
P = ctypes.POINTER

SIGNATURES = {
    "poisson_plan_create": (c_int, [P(c_void_p), c_int, c_double, c_double, c_int]),
    "poisson_plan_create_batched": (c_int, [P(c_void_p), c_int, c_double, c_double, c_int, c_int]),
    "poisson_plan_create_box": (c_int, [P(c_void_p), c_int, c_double, c_double, c_double, c_double, c_int]),
    "poisson_plan_create_box_n": (c_int, [P(c_void_p), c_int, c_int, c_int, c_double, c_double, c_double, c_double,
                                          c_int]),
    "poisson_plan_destroy": (c_int, [c_void_p]),
    "poisson_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "poisson_solve_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "poisson_solve_batched": (c_int, [c_int, P(c_void_p), P(c_void_p), P(c_void_p), c_void_p]),
    "poisson_solve_timed": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, P(ctypes.c_float)]),
    "poisson_last_status": (c_int, [c_void_p, c_void_p]),
    "poisson_selftest_wait": (c_int, [c_void_p, ctypes.c_longlong, c_void_p]),
    "poisson_solve_checked": (c_int, [c_void_p, c_void_p, c_void_p, P(c_double), c_void_p]),
    "poisson_solve_checked_batched": (c_int, [c_void_p, c_int, P(c_void_p), P(c_void_p), P(c_double), c_void_p]),
    "poisson_compare": (c_int, [c_void_p, c_int, c_void_p, c_int, c_size_t, P(c_double), P(c_double), c_void_p]),
    "poisson_plan_info": (c_int, [c_void_p, P(c_double), P(c_double), P(c_int), P(c_double),
                                  P(c_double), P(c_size_t), P(c_size_t)]),
    "poisson_plan_get_knob": (c_int, [c_void_p, c_int, P(c_int)]),
    "poisson_plan_set_knob": (c_int, [c_void_p, c_int, c_int]),
    "poisson_plan_gauss_sum": (c_int, [c_void_p, P(c_double), P(c_double), c_int]),
    "poisson_plan_axis_table": (c_int, [c_void_p, P(c_double), c_size_t]),
    "poisson_supported_n": (c_int, [c_int]),
    "poisson_strerror": (ctypes.c_char_p, [c_int]),
    "poisson_last_cuda_error": (ctypes.c_char_p, []),
    "poisson_solve_noalloc": (c_int, [c_int, c_double, c_double, c_int, c_void_p, c_void_p, c_void_p]),
    "poisson_noalloc_last_status": (c_int, [c_void_p]),
    "poisson_slab_forward": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "poisson_slab_z": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "poisson_slab_inverse": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "poisson_plan_spectrum": (c_int, [c_void_p, c_int, P(c_void_p), P(ctypes.c_size_t), P(ctypes.c_size_t)]),
    "poisson_noalloc_selftest_wait": (c_int, [ctypes.c_longlong, c_void_p]),
    "poisson_debug_flags": (c_int, [P(ctypes.c_uint), c_void_p]),
    "poisson_debug_selftest": (c_int, [c_void_p]),
    "poisson_sample_gaussians": (c_int, [c_int, c_double, c_int, P(c_double), c_int, c_void_p, c_void_p]),
    "poisson_gaussian_potential": (c_int, [c_int, c_double, c_int, P(c_double), c_int, c_void_p, c_void_p,
                                           c_void_p]),
    "poisson_compare_points": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, P(c_double),
                                       c_void_p]),
    "poisson_features32": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "poisson_mlp_nparams": (c_int, [c_int]),
    "poisson_mlp_forward": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "poisson_mlp_loss": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "poisson_mlp_backward": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "poisson_mlp_adam": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_float, c_int, c_void_p]),
    "poisson_selector_load": (c_int, [P(c_void_p), ctypes.c_char_p, c_int]),
    "poisson_selector_destroy": (c_int, [c_void_p]),
    "poisson_select_n": (c_int, [c_void_p, c_void_p, c_int, c_double, P(c_int), P(ctypes.c_float), c_void_p]),
}


class PoissonError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, ERRORS.get(code, "unknown"), code))


KNOB_Z_FORM = 0
KNOB_Y_FORM = 1
KNOB_X_FORM = 2
KNOB_XY_FORM = 3
KNOB_CORRECTION = 4
KNOB_ARITH = 5


def debug_requested():
    return os.environ.get("POISSON_DEBUG", "") == "1"


def load():
    """Load the in-tree library (its debug build with POISSON_DEBUG=1).  There is no
    fallback: without it nothing can run."""
    global _lib
    with _lock:
        if _lib is None:
            path = DEBUG_LIB_PATH if debug_requested() else LIB_PATH
            if not os.path.exists(path):
                raise ImportError("%s is not built; run paper_1612_01799_gb300.build.build(%s) first"
                                  % (path, "debug=True" if debug_requested() else ""))
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def check(rc, what):
    if rc != OK:
        detail = ""
        if _lib is not None and rc in (-2, -3):
            detail = " [%s]" % _lib.poisson_last_cuda_error().decode()
        raise PoissonError(rc, what + detail)
