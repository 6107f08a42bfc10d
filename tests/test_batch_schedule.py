"""The one-launch batch kernel's work list, built on the host by the library
(se2_debug_batch_work_list), checked without a GPU:

* every unit of every problem appears exactly once;
* every dependency points to an earlier place in the list (unit B of a
  problem after all its units A, C after all its B, A of problem p after
  all units C of problem p - D whose ring slot it reuses), which is what
  makes the in-order claiming deadlock-free;
* a discrete-event run of `grid` blocks claiming units in list order (each
  waiting for its dependency, one unit claimed ahead) finishes every unit.
"""
import ctypes
import heapq

import pytest

from paper_2504_05149_gb300 import load_library


class _Shape(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int)]


def _work_list(classes, grid):
    lib = load_library()
    f = lib.se2_debug_batch_work_list
    f.argtypes = [ctypes.POINTER(_Shape), ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                  ctypes.POINTER(ctypes.c_int)]
    f.restype = ctypes.c_int
    n = len(classes)
    shp = (_Shape * n)(*[_Shape(N, M) for N, M, _ in classes])
    cnt = (ctypes.c_int * n)(*[c for _, _, c in classes])
    total = ctypes.c_longlong(0)
    assert f(shp, cnt, n, grid, None, ctypes.byref(total), None, None) == 0
    units = (ctypes.c_uint * total.value)()
    slots = (ctypes.c_int * n)()
    lag = (ctypes.c_int * n)()
    assert f(shp, cnt, n, grid, units, ctypes.byref(total), slots, lag) == 0
    codes = [(u >> 28, (u >> 26) & 3, (u >> 16) & 0x3FF, u & 0xFFFF) for u in units]
    return codes, list(slots), list(lag)


def _yr(N, M):
    teams = 256 // (1 if N < 32 else (16 if N >= 128 else 8))
    return max(1, min(8, teams * 4 // M))


def _expected_units(N, M):
    nA = N // _yr(N, M)
    lines = 256 // (16 if N >= 128 else 8)
    nB = (M * (N // 4 + 1) + lines - 1) // lines
    return nA, nB, nA


# the batching workload's classes, largest work first, with their counts
C4 = [(256, 64, 332), (256, 32, 371), (128, 64, 364), (256, 16, 353), (128, 32, 334), (64, 64, 362),
      (128, 16, 357), (64, 32, 345), (32, 64, 337), (64, 16, 332), (32, 32, 308), (32, 16, 301)]


def _check_order(classes, codes, slots):
    pos_max = {}
    pos_min = {}
    seen = set()
    for i, key in enumerate(codes):
        assert key not in seen, key
        seen.add(key)
        c, s, u, p = key
        k = (c, s, p)
        pos_max[k] = i
        pos_min.setdefault(k, i)
    for c, (N, M, n) in enumerate(classes):
        nA, nB, nC = _expected_units(N, M)
        for p in range(n):
            for s, nu in enumerate((nA, nB, nC)):
                for u in range(nu):
                    assert (c, s, u, p) in seen, (c, s, u, p)
            assert pos_min[(c, 1, p)] > pos_max[(c, 0, p)]
            assert pos_min[(c, 2, p)] > pos_max[(c, 1, p)]
            if p >= slots[c]:
                assert pos_min[(c, 0, p)] > pos_max[(c, 2, p - slots[c])]
    assert len(seen) == sum(n * sum(_expected_units(N, M)) for N, M, n in classes)


def test_work_list_of_the_batching_classes_is_complete_and_ordered():
    codes, slots, lag = _work_list(C4, 304)
    _check_order(C4, codes, slots)
    for (N, M, n), D, L in zip(C4, slots, lag):
        assert L >= 1 and D == min(3 * L + 1, n)
    # the largest class keeps a ring of 4 problems (about 76 MB, inside L2)
    assert slots[0] == 4


@pytest.mark.parametrize("grid", [1, 7, 304])
def test_small_batches_and_grids(grid):
    classes = [(256, 16, 3), (64, 64, 1), (32, 16, 9)]
    codes, slots, _ = _work_list(classes, grid)
    _check_order(classes, codes, slots)


def test_unsupported_class_is_refused():
    lib = load_library()
    f = lib.se2_debug_batch_work_list
    f.argtypes = [ctypes.POINTER(_Shape), ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                  ctypes.POINTER(ctypes.c_int)]
    n = ctypes.c_longlong(0)
    for N, M, cnt in ((512, 64, 1), (256, 128, 1), (256, 8, 1), (64, 16, 70000)):
        shp = (_Shape * 1)(_Shape(N, M))
        c = (ctypes.c_int * 1)(cnt)
        assert f(shp, c, 1, 304, None, ctypes.byref(n), None, None) == 2   # SE2_ERR_UNSUPPORTED


def _simulate(classes, codes, slots, grid, dur):
    """Blocks claim units in list order (one ahead); a claimed unit starts
    when its dependency count is met; returns the finish time (None on a
    stall with work left)."""
    nunits = {}
    for c, (N, M, n) in enumerate(classes):
        nunits[c] = _expected_units(N, M)
    done = {}
    waiting = {}           # dependency key -> list of (block, unit index)
    nxt = 0
    events = []            # (time, block, unit index)
    t = 0.0

    def dep_of(key):
        c, s, _, p = key
        if s == 1:
            return (c, 0, p), nunits[c][0]
        if s == 2:
            return (c, 1, p), nunits[c][1]
        if p >= slots[c]:
            return (c, 2, p - slots[c]), nunits[c][2]
        return None, 0

    def try_start(b, i, now):
        dk, target = dep_of(codes[i])
        if dk is not None and done.get(dk, 0) < target:
            waiting.setdefault(dk, []).append((b, i, target))
            return
        heapq.heappush(events, (now + dur(codes[i]), b, i))

    for b in range(min(grid, len(codes))):
        try_start(b, nxt, 0.0)
        nxt += 1
    finished = 0
    while events:
        t, b, i = heapq.heappop(events)
        c, s, _, p = codes[i]
        k = (c, s, p)
        done[k] = done.get(k, 0) + 1
        finished += 1
        if k in waiting:
            still = []
            for (bb, ii, target) in waiting.pop(k):
                if done[k] >= target:
                    heapq.heappush(events, (t + dur(codes[ii]), bb, ii))
                else:
                    still.append((bb, ii, target))
            if still:
                waiting[k] = still
        if nxt < len(codes):
            try_start(b, nxt, t)
            nxt += 1
    return t if finished == len(codes) else None


@pytest.mark.parametrize("grid", [3, 40])
def test_in_order_claiming_finishes_every_unit(grid):
    classes = [(256, 32, 6), (128, 16, 9), (64, 64, 5), (32, 16, 12)]
    codes, slots, _ = _work_list(classes, grid)
    # unit durations proportional to the points a unit covers, B a little longer
    def dur(key):
        c, s, _, _ = key
        N, M, _ = classes[c]
        nA, nB, nC = _expected_units(N, M)
        return N * N * M / (nB if s == 1 else nA) * (1.2 if s == 1 else 1.0)
    assert _simulate(classes, codes, slots, grid, dur) is not None
