"""The C-ABI library loads, exports every symbol include/se2.h declares, and
rejects bad arguments on the host before touching a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_05149_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(se2_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"se2_plan_create", "se2_coeffs", "se2_convolve", "se2_convolve_chain"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_version_and_error_text(lib):
    lib.se2_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.se2_version()
    lib.se2_last_error.restype = ctypes.c_char_p
    assert lib.se2_last_error() is not None


@pytest.mark.parametrize("N,M,B,prec,status", [
    (7, 16, 1, 1, 2),     # N not a power of two -> UNSUPPORTED
    (1024, 16, 1, 1, 2),  # N too large
    (32, 3, 1, 1, 2),     # M not a power of two
    (32, 256, 1, 1, 2),   # M too large
    (32, 16, 0, 1, 1),    # batch < 1 -> INVALID_ARG
    (32, 16, 1, 9, 2),    # unknown precision -> UNSUPPORTED
])
def test_plan_create_rejects_bad_sizes_on_host(lib, N, M, B, prec, status):
    h = ctypes.c_void_p(1)
    lib.se2_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_uint, ctypes.c_int]
    assert lib.se2_plan_create(ctypes.byref(h), N, M, B, prec, 0, 0) == status
    assert not h.value  # NULL on failure


def test_null_plan_and_null_pointers_rejected(lib):
    vp = ctypes.c_void_p
    lib.se2_convolve.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp, vp]
    lib.se2_coeffs.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp]
    assert lib.se2_convolve(None, None, 1, None, None, None, None) == 1
    assert lib.se2_coeffs(None, None, 1, None, None, None) == 1
    assert lib.se2_plan_create(None, 32, 16, 1, 1, 0, 0) == 1
    lib.se2_plan_destroy.argtypes = [vp]
    assert lib.se2_plan_destroy(None) == 0


def test_samplers_reject_null_plan_on_host(lib):
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.se2_sample_se2_gaussian.argtypes = [vp, dp, dp, ctypes.c_int, vp, vp]
    lib.se2_sample_deformed_gaussian.argtypes = [vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, vp]
    beta = (ctypes.c_double * 3)(0, 0, 0)
    S = (ctypes.c_double * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    H = (ctypes.c_double * 4)(1, 0, 0, 1)
    assert lib.se2_sample_se2_gaussian(None, beta, S, 1, None, None) == 1
    assert lib.se2_sample_deformed_gaussian(None, H, 0.0, 0.1, 1, None, None) == 1


@pytest.mark.parametrize("L,N,status", [
    ((8, 9, 9), (8, 9, 9), 2),       # even sampling size -> UNSUPPORTED
    ((9, 9, 257), (9, 9, 257), 2),   # above the largest sampling size
    ((9, 9, 9), (9, 8, 9), 1),       # N < L -> INVALID_ARG
    ((9, 9, 9), (9, 9, 2000), 1),    # N too large
])
def test_grid_plan_rejects_bad_sizes_on_host(lib, L, N, status):
    h = ctypes.c_void_p(1)
    i3 = ctypes.c_int * 3
    lib.se2_grid_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                         ctypes.c_int]
    assert lib.se2_grid_plan_create(ctypes.byref(h), i3(*L), i3(*N), 1, 1, 0, 0) == status
    assert not h.value


@pytest.mark.parametrize("eps,grad,kinf,c,want", [
    (0.5, 1.0, 0, 0.0, 64),        # 32 * 1 / 0.5
    (3.0, 1.0, 0, 0.0, 11),        # ceil(10.67)
    (3.0, 1.0, 40, 0.0, 40),       # ||k||_inf dominates
    (1.0, 0.0, 0, 0.0, 1),         # K in N
    (0.5, 1.0, 0, 36.0, 72),       # the proof's constant
])
def test_accuracy_order_algorithm1_on_host(lib, eps, grad, kinf, c, want):
    lib.se2_accuracy_order.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_longlong)]
    K = ctypes.c_longlong(-1)
    assert lib.se2_accuracy_order(eps, grad, kinf, c, ctypes.byref(K)) == 0
    assert K.value == want


@pytest.mark.parametrize("eps,grad,kinf", [(0.0, 1.0, 0), (-1.0, 1.0, 0), (1.0, -1.0, 0), (1.0, 1.0, -2),
                                           (float("nan"), 1.0, 0), (1.0, float("inf"), 0)])
def test_accuracy_order_rejects_bad_input(lib, eps, grad, kinf):
    lib.se2_accuracy_order.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_longlong)]
    K = ctypes.c_longlong(-1)
    assert lib.se2_accuracy_order(eps, grad, kinf, 0.0, ctypes.byref(K)) == 1


def test_unknown_plan_flag_rejected_on_host(lib):
    h = ctypes.c_void_p(1)
    lib.se2_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_uint, ctypes.c_int]
    assert lib.se2_plan_create(ctypes.byref(h), 32, 16, 1, 1, 0x80, 0) == 1
    assert not h.value


def test_allocation_accounting_entry_points(lib):
    """se2_debug_alloc_stats / se2_debug_fail_alloc work without a device:
    the counts are consistent (both 0 where nothing has been allocated in this
    process; GPU tests earlier in the same process may have allocated), bad
    arguments are rejected, and arming or disarming the failure injection
    succeeds."""
    ll = ctypes.c_longlong
    lib.se2_debug_alloc_stats.argtypes = [ctypes.POINTER(ll), ctypes.POINTER(ll)]
    lib.se2_debug_fail_alloc.argtypes = [ll]
    live, total = ll(-1), ll(-1)
    assert lib.se2_debug_alloc_stats(ctypes.byref(live), ctypes.byref(total)) == 0
    assert 0 <= live.value <= total.value
    assert lib.se2_debug_alloc_stats(None, ctypes.byref(total)) == 1
    assert lib.se2_debug_fail_alloc(-1) == 1
    assert lib.se2_debug_fail_alloc(3) == 0
    assert lib.se2_debug_fail_alloc(0) == 0
