"""Batched execution of many independent SE(2) convolutions of uneven sizes,
on the library's batch plan (se2_batch_plan_*).

The C runtime groups the problems into size classes (equal grid N x N x M),
gives each class its own plan, runs the classes on one or more stream lanes
forked from the caller's (one `se2_batch_convolve_separable` call,
capturable in a CUDA graph) and tunes, per class, the schedule of its
launches (pipeline depth and group size of the FP32 fast path, or the
persistent dataflow kernel) by timing the candidates on the class's own
data, then the number of lanes for the whole batch (`se2_batch_tune`).  Each
problem carries a chain of separable radial kernels (Gaussian x wrapped
normal), whose product is kept in factored form (three 1-D tables per
problem).  This module only holds the packed tensors and marshals calls.
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import _check, _ptr, _stream, load_library

_CACHE_ENV = "SE2_AUTOTUNE_CACHE"


def _default_cache() -> str:
    return os.environ.get(_CACHE_ENV, os.path.join(os.path.expanduser("~"), ".cache", "se2_autotune.json"))


class _Shape(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int)]


def _bind(lib):
    if getattr(lib, "_se2_batch_bound", False):
        return lib
    vp, ip = ctypes.c_void_p, ctypes.c_int
    ll = ctypes.POINTER(ctypes.c_longlong)
    lib.se2_batch_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Shape), ip, ip, ctypes.c_uint, ip]
    lib.se2_batch_plan_destroy.argtypes = [vp]
    lib.se2_batch_plan_layout.argtypes = [vp, ctypes.POINTER(ip), ll, ll, ll, ll]
    lib.se2_batch_separable_tables.argtypes = [vp, vp, vp, ip, vp, vp]
    lib.se2_batch_convolve_separable.argtypes = [vp, vp, vp, vp, vp]
    lib.se2_batch_tune.argtypes = [vp, vp, vp, vp, ip, vp]
    lib.se2_batch_plan_config.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(_Shape), ctypes.POINTER(ip),
                                          ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip),
                                          ctypes.POINTER(ctypes.c_double)]
    lib.se2_batch_plan_lanes.argtypes = [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_double)]
    lib.se2_batch_plan_one_launch.argtypes = [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_double)]
    lib.se2_batch_plan_status.argtypes = [vp, vp]
    lib.se2_debug_batch_wait_timeout.argtypes = [vp, vp, vp, vp, vp]
    lib.se2_batch_plan_launches.argtypes = [vp]
    lib.se2_batch_plan_launches.restype = ctypes.c_ulonglong
    for name in ("se2_batch_plan_create", "se2_batch_plan_destroy", "se2_batch_plan_layout", "se2_batch_separable_tables",
                 "se2_batch_convolve_separable", "se2_batch_tune", "se2_batch_plan_config", "se2_batch_plan_lanes",
                 "se2_batch_plan_one_launch", "se2_batch_plan_status", "se2_debug_batch_wait_timeout"):
        getattr(lib, name).restype = ctypes.c_int
    lib._se2_batch_bound = True
    return lib


class BatchRunner:
    """Packed inputs/outputs/tables of a fixed set of problem shapes over one
    batch plan.  Usage: fill `f_of(i)` and `set_chain(...)`, then `run()` (or
    `capture()` once and `replay()`)."""

    def __init__(self, shapes: Sequence[Tuple[int, int]], device: int = 0, autotune: bool = True,
                 cache_path: Optional[str] = None, kmax: int = 16):
        self.lib = _bind(load_library())
        self.device = device
        self.dev = torch.device("cuda", device)
        self.shapes = [(int(N), int(M)) for N, M in shapes]
        self.kmax = kmax
        n = len(self.shapes)
        arr = (_Shape * n)(*[_Shape(N, M) for N, M in self.shapes])
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.dev):
            _check(self.lib.se2_batch_plan_create(ctypes.byref(self._h), arr, n, 1, 0, device))
        pos = (ctypes.c_int * n)()
        goff = (ctypes.c_longlong * n)()
        toff = (ctypes.c_longlong * n)()
        gtot, ttot = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self.lib.se2_batch_plan_layout(self._h, pos, goff, toff, ctypes.byref(gtot), ctypes.byref(ttot)))
        self.pos, self.goff, self.toff = list(pos), list(goff), list(toff)
        self.f_packed = torch.zeros(int(gtot.value), dtype=torch.float32, device=self.dev)
        self.out_packed = torch.empty_like(self.f_packed)
        self.tab_packed = torch.empty(int(ttot.value), dtype=torch.complex64, device=self.dev)
        self.params = torch.zeros((n, kmax, 3), dtype=torch.float64, device=self.dev)
        self.params[:, :, 0] = 0.02
        self.params[:, :, 1] = 0.3
        self.k = torch.ones(n, dtype=torch.int32, device=self.dev)
        self.classes: Dict[Tuple[int, int], List[int]] = {}
        for i, s in enumerate(self.shapes):
            self.classes.setdefault(s, []).append(i)
        self.order = [c for c, *_ in self._config()]   # the plan's class order (largest work first)
        # per-class views of the packed output (classes are contiguous blocks)
        self.out = {}
        for c in self.order:
            first = min(self.goff[i] for i in self.classes[c])
            size = c[0] * c[0] * c[1] * len(self.classes[c])
            self.out[c] = self.out_packed[first:first + size]
        self.cache_path = cache_path or _default_cache()
        self.config: Dict[Tuple[int, int], Tuple[str, int]] = {}
        self._autotune = autotune
        self._tuned = False
        self._tables = False
        self.graph = None
        self._graph_launches = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.se2_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs ---------------------------------------------------------------
    def _view(self, t: torch.Tensor, i: int) -> torch.Tensor:
        N, M = self.shapes[i]
        return t[self.goff[i]:self.goff[i] + N * N * M].view(M, N, N)

    def f_of(self, i: int) -> torch.Tensor:
        return self._view(self.f_packed, i)

    def out_of(self, i: int) -> torch.Tensor:
        return self._view(self.out_packed, i)

    def set_chain(self, i: int, kernels: Sequence[Tuple[float, float, float]]):
        """Kernel chain of problem i: a list of (sigma, sigma_theta, nu)."""
        if not 1 <= len(kernels) <= self.kmax:
            raise ValueError(f"chain length must be in [1, {self.kmax}]")
        p = torch.zeros((self.kmax, 3), dtype=torch.float64)
        for j, kp in enumerate(kernels):
            p[j] = torch.tensor([float(v) for v in kp], dtype=torch.float64)
        self.params[self.pos[i]] = p.to(self.dev)
        self.k[self.pos[i]] = len(kernels)

    def build_tables(self):
        """Factored chain coefficients for every problem (se2_batch_separable_tables)."""
        _check(self.lib.se2_batch_separable_tables(self._h, _ptr(self.params), _ptr(self.k), self.kmax,
                                                   _ptr(self.tab_packed), _stream(self.dev)))
        self._tables = True

    # -- tuning -----------------------------------------------------------------
    def _config(self):
        nc = ctypes.c_int()
        _check(self.lib.se2_batch_plan_config(self._h, ctypes.byref(nc), None, None, None, None, None, None))
        m = nc.value
        shp = (_Shape * m)()
        cnt, dep, grp, per = ((ctypes.c_int * m)() for _ in range(4))
        ms = (ctypes.c_double * m)()
        _check(self.lib.se2_batch_plan_config(self._h, ctypes.byref(nc), shp, cnt, dep, grp, per, ms))
        return [((shp[j].N, shp[j].M), cnt[j], dep[j], grp[j], per[j], ms[j]) for j in range(m)]

    def tune(self, reps: int = 3):
        """se2_batch_tune on the current data; the choices per class are also
        written to a JSON record keyed by GPU name, size, class population."""
        if not self._tables:
            self.build_tables()
        _check(self.lib.se2_batch_tune(self._h, _ptr(self.f_packed), _ptr(self.tab_packed), _ptr(self.out_packed),
                                       int(reps), _stream(self.dev)))
        self._tuned = True
        gpu = torch.cuda.get_device_name(self.dev)
        record = {}
        for c, n, depth, group, pers, ms in self._config():
            path = "persistent" if pers else ("pipelined" if depth > 1 else "three")
            self.config[c] = (path, group)
            record[f"{gpu}|N={c[0]}|M={c[1]}|n={n}|f32"] = [path, depth, group, ms]
        lanes, _, lane_ms = self.lanes()
        one, one_ms = self.one_launch()
        record[f"{gpu}|batch|classes={len(self.order)}|n={len(self.shapes)}|f32"] = \
            ["one launch" if one else "lanes", lanes, lane_ms, one_ms]
        try:
            os.makedirs(os.path.dirname(self.cache_path) or ".", exist_ok=True)
            old = {}
            if os.path.exists(self.cache_path):
                with open(self.cache_path) as fh:
                    old = json.load(fh)
            old.update(record)
            with open(self.cache_path, "w") as fh:
                json.dump(old, fh, indent=1, sort_keys=True)
        except Exception:
            pass

    def lanes(self, n: Optional[int] = None):
        """Set the number of stream lanes (n >= 1) or leave it (None); returns
        (lanes in force, lane of each class in plan order, {L: tuned
        whole-batch ms on L lanes})."""
        m = len(self.order)
        cur = ctypes.c_int()
        lane = (ctypes.c_int * m)()
        ms = (ctypes.c_double * m)()
        _check(self.lib.se2_batch_plan_lanes(self._h, int(n) if n else 0, ctypes.byref(cur), lane, ms))
        return cur.value, list(lane), {L + 1: ms[L] for L in range(m) if ms[L] > 0}

    def one_launch(self, enable: Optional[bool] = None):
        """Enable (True) or disable (False) the one-launch kernel for the whole
        batch, or leave it (None); returns (in force, tuner's ms for it)."""
        cur = ctypes.c_int()
        ms = ctypes.c_double()
        mode = -1 if enable is None else int(bool(enable))
        with torch.cuda.device(self.dev):
            _check(self.lib.se2_batch_plan_one_launch(self._h, mode, ctypes.byref(cur), ctypes.byref(ms)))
        if enable is not None:
            self.graph = None          # a captured graph holds the other schedule
        return bool(cur.value), ms.value

    def status(self):
        """se2_batch_plan_status on the current stream (raises on a timed-out wait)."""
        _check(self.lib.se2_batch_plan_status(self._h, _stream(self.dev)))

    # -- execution --------------------------------------------------------------
    def run(self):
        """Every problem, classes concurrently, on the current stream."""
        if not self._tables:
            self.build_tables()
        if self._autotune and not self._tuned:
            self.tune()
        _check(self.lib.se2_batch_convolve_separable(self._h, _ptr(self.f_packed), _ptr(self.tab_packed),
                                                     _ptr(self.out_packed), _stream(self.dev)))

    def launches(self) -> int:
        return int(self.lib.se2_batch_plan_launches(self._h))

    def capture(self):
        """Record run() into a CUDA graph (tables and tuning done first)."""
        if not self._tables:
            self.build_tables()
        if self._autotune and not self._tuned:
            self.tune()
        self.run()                                   # warm-up outside capture
        torch.cuda.synchronize(self.dev)
        g = torch.cuda.CUDAGraph()
        before = self.launches()
        with torch.cuda.graph(g):
            self.run()
        self._graph_launches = self.launches() - before
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def launches_per_run(self) -> int:
        """Kernel launches of one run(), counted by the plan while the graph was
        captured, or over one eager run()."""
        if self._graph_launches is not None:
            return self._graph_launches
        before = self.launches()
        self.run()
        return self.launches() - before

    def points(self) -> int:
        return sum(N * N * M * len(v) for (N, M), v in self.classes.items())
