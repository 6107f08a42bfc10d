"""ctypes binding of oracle/direct.c (brute-force routes of the FP64 oracle).

TEST INFRASTRUCTURE ONLY (see oracle/se2_oracle.py).  `build()` compiles the
C file with gcc into oracle/lib/; `__graft_entry__.build()` calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "lib", "libse2_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        lib.se2_direct_conv.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp]
        lib.se2_direct_conv_shift.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        lib.se2_direct_conv_points.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, lp, ctypes.c_long, dp]
        lib.se2_group_quadrature.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                             ctypes.c_int, dp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def direct_conv(F: np.ndarray, P: np.ndarray, origin_zero: bool = False) -> np.ndarray:
    """out[n] = (1/|L|) sum_m F[m] P[n - m + (0, c, c)] (even N), c = N/2 on
    Omega_L and c = 0 for grids sampled at x_i = i/N."""
    lib = _load()
    M, N, N2 = F.shape
    assert N == N2 and N % 2 == 0 and P.shape == F.shape
    F = np.ascontiguousarray(F, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    out = np.empty_like(F)
    lib.se2_direct_conv_shift(_ptr(F), _ptr(P), N, M, 0 if origin_zero else N // 2, _ptr(out))
    return out


def direct_conv_points(F: np.ndarray, P: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """The direct sum at the given flat output indices only."""
    lib = _load()
    M, N, _ = F.shape
    F = np.ascontiguousarray(F, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    out = np.empty(pts.size, dtype=np.float64)
    lib.se2_direct_conv_points(_ptr(F), _ptr(P), N, M,
                               pts.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), pts.size, _ptr(out))
    return out


def group_quadrature(F: np.ndarray, kind: int, params, images: int = 2) -> np.ndarray:
    """Rectangle rule of the SE(2) convolution with the full group law."""
    lib = _load()
    M, N, _ = F.shape
    F = np.ascontiguousarray(F, dtype=np.float64)
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    out = np.empty_like(F)
    lib.se2_group_quadrature(_ptr(F), N, M, kind, _ptr(p), images, _ptr(out))
    return out
