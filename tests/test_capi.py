"""The C-ABI library: it builds, loads, exports every function include/poisson.h declares,
and rejects bad arguments on the host before any device work.  No GPU needed."""
import ctypes
import re

import pytest

from paper_1612_01799_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    with open(_lib.HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(poisson_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(_lib.SIGNATURES)


def test_knob_codes_match_the_header():
    with open(_lib.HEADER) as f:
        defs = dict(re.findall(r"#define POISSON_(KNOB_[A-Z_]+)\s+(\d+)", f.read()))
    assert defs, "no knob codes in the header"
    for name, code in defs.items():
        assert getattr(_lib, name) == int(code), name


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def five_smooth_even(n):
    if n < 4 or n > 1024 or n % 2:
        return False
    for f in (2, 3, 5):
        while n % f == 0:
            n //= f
    return n == 1


def test_supported_sizes(lib):
    """1: compiled-length forms; 2: runtime-length forms (every other even N in 4..1024
    with no prime factor above 5, i.e. 2N factors into 2, 3 and 5); 0: unsupported."""
    compiled = (4, 8, 16, 32, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 1024)
    for n in compiled:
        assert lib.poisson_supported_n(n) == 1
    for n in range(-4, 1100):
        if n not in compiled:
            assert lib.poisson_supported_n(n) == (2 if five_smooth_even(n) else 0), n
    assert sum(lib.poisson_supported_n(n) == 2 for n in range(1100)) == 51


def test_error_strings(lib):
    assert lib.poisson_strerror(0) == b"ok"
    assert lib.poisson_strerror(-1) == b"invalid argument"
    assert lib.poisson_strerror(-99) == b"unknown error"


def test_plan_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p(1234)
    assert lib.poisson_plan_create(None, 32, 8.0, 1e-12, 1) == -1
    assert lib.poisson_plan_create(ctypes.byref(h), 33, 8.0, 1e-12, 1) == -1     # odd N
    assert h.value is None                                                        # cleared
    assert lib.poisson_plan_create(ctypes.byref(h), 2, 8.0, 1e-12, 1) == -1
    assert lib.poisson_plan_create(ctypes.byref(h), 32, 8.0, 1e-12, 7) == -1     # dtype
    assert lib.poisson_plan_create(ctypes.byref(h), 14, 8.0, 1e-12, 0) == -4     # prime factor 7
    assert lib.poisson_plan_create(ctypes.byref(h), 1030, 8.0, 1e-12, 0) == -1   # above 1024
    assert lib.poisson_plan_create(ctypes.byref(h), 32, -1.0, 1e-12, 0) == -1    # L <= 0
    assert lib.poisson_plan_create(ctypes.byref(h), 32, float("nan"), 1e-12, 0) == -1
    assert lib.poisson_plan_create(ctypes.byref(h), 32, 8.0, 0.0, 0) == -1       # tol <= 0
    assert lib.poisson_plan_create(ctypes.byref(h), 4, 1000.0, 1e-6, 0) == -1    # delta >= 1


def test_box_plan_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p(1234)
    assert lib.poisson_plan_create_box(None, 32, 1.0, 2.0, 3.0, 1e-12, 1) == -1
    assert lib.poisson_plan_create_box(ctypes.byref(h), 33, 1.0, 2.0, 3.0, 1e-12, 1) == -1   # odd N
    assert h.value is None
    assert lib.poisson_plan_create_box(ctypes.byref(h), 44, 1.0, 2.0, 3.0, 1e-12, 0) == -4   # prime factor 11
    assert lib.poisson_plan_create_box(ctypes.byref(h), 32, 1.0, -2.0, 3.0, 1e-12, 0) == -1  # L_q <= 0
    assert lib.poisson_plan_create_box(ctypes.byref(h), 32, 1.0, float("inf"), 3.0, 1e-12, 0) == -1
    assert lib.poisson_plan_create_box(ctypes.byref(h), 32, 1.0, 2.0, 3.0, 0.0, 0) == -1     # tol <= 0
    # Sec. 3 side condition: delta (at least 1e-3) must lie below the flattest l_q = 1e-4
    assert lib.poisson_plan_create_box(ctypes.byref(h), 4, 0.001, 10.0, 10.0, 1e-6, 0) == -1


def test_box_n_plan_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p(1234)
    f = lib.poisson_plan_create_box_n
    assert f(None, 16, 24, 32, 1.0, 2.0, 3.0, 1e-12, 1) == -1
    assert f(ctypes.byref(h), 16, 25, 32, 1.0, 2.0, 3.0, 1e-12, 1) == -1    # odd n_y
    assert h.value is None
    assert f(ctypes.byref(h), 16, 24, 2, 1.0, 2.0, 3.0, 1e-12, 1) == -1     # n_z < 4
    assert f(ctypes.byref(h), 16, 24, 2048, 1.0, 2.0, 3.0, 1e-12, 1) == -1  # n_z > 1024
    assert f(ctypes.byref(h), 16, 28, 32, 1.0, 2.0, 3.0, 1e-12, 1) == -4    # prime factor 7
    assert f(ctypes.byref(h), 16, 24, 32, 1.0, 0.0, 3.0, 1e-12, 1) == -1    # L_y <= 0
    assert f(ctypes.byref(h), 16, 24, 32, 1.0, 2.0, 3.0, 1e-12, 3) == -1    # dtype
    assert f(ctypes.byref(h), 16, 24, 32, 1.0, 2.0, 3.0, -1.0, 0) == -1     # tol <= 0


def test_null_plan_calls_are_errors(lib):
    assert lib.poisson_plan_destroy(None) == 0
    assert lib.poisson_solve(None, None, None, None) == -1
    assert lib.poisson_solve_host(None, None, None, None) == -1
    assert lib.poisson_solve_timed(None, None, None, None, None) == -1
    assert lib.poisson_plan_info(None, None, None, None, None, None, None, None) == -1
    assert lib.poisson_solve_batched(0, None, None, None, None) == 0
    assert lib.poisson_solve_batched(-1, None, None, None, None) == -1
    assert lib.poisson_solve_batched(2, None, None, None, None) == -1


def test_product_path_has_no_fallback(monkeypatch, tmp_path):
    """Without the shared library the solver raises instead of computing anything."""
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()


def test_release_build_has_no_debug_flags(lib):
    """The bounds-check word exists only in the debug build: the release library answers
    POISSON_ERR_UNSUPPORTED with the flags zeroed, and a null pointer is an argument error
    (no device work in either case)."""
    flags = ctypes.c_uint(7)
    assert lib.poisson_debug_flags(ctypes.byref(flags), None) == -4
    assert flags.value == 0
    assert lib.poisson_debug_flags(None, None) == -1
    assert lib.poisson_debug_selftest(None) == -4


def test_debug_build_is_selected_by_the_environment(monkeypatch):
    """POISSON_DEBUG=1 points the binding at libgspoisson_debug.so (and nothing else)."""
    monkeypatch.setenv("POISSON_DEBUG", "1")
    assert _lib.debug_requested()
    monkeypatch.setenv("POISSON_DEBUG", "0")
    assert not _lib.debug_requested()
