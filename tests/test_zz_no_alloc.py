"""se2_convolve_noalloc -- the allocation-free entry point -- against the
plan-based se2_convolve, through the C ABI, on two calls in a row.

The entry point exists for callers that are not allowed to allocate device
memory (a plan allocates its scratch with cudaMalloc); it works in a fixed
device array inside the library instead.  This file is named so that pytest
collects it last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    lib = m.load_library()
    vp = ctypes.c_void_p
    lib.se2_convolve_noalloc.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    lib.se2_convolve_noalloc.restype = ctypes.c_int
    return m


def _noalloc(se2, f, C, out, N, M, B):
    lib = se2.load_library()
    st = lib.se2_convolve_noalloc(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), N, M, B,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.se2_last_error().decode()


@pytest.mark.parametrize("N,M,B", [(256, 64, 5), (32, 16, 3), (512, 8, 2)])
def test_noalloc_matches_plan_path_on_two_calls(se2, N, M, B):
    rng = np.random.default_rng(N + 7 * M)
    plan = se2.Plan(N, M, batch=B)
    outs = []
    for call in range(2):
        f = torch.from_numpy(rng.standard_normal((B, M, N, N)).astype(np.float32)).cuda()
        P = torch.from_numpy(rng.random((B, M, N, N)).astype(np.float32)).cuda()
        C, _ = se2.coeffs(plan, P)
        want = se2.convolve(plan, f, C)
        got = torch.full_like(f, float("nan"))
        _noalloc(se2, f, C, got, N, M, B)
        torch.cuda.synchronize()
        w = want.double().cpu().numpy()
        g = got.double().cpu().numpy()
        assert np.isfinite(g).all()
        assert np.max(np.abs(g - w)) / np.max(np.abs(w)) < 1e-5
        outs.append(g)
    assert not np.allclose(outs[0], outs[1])   # the second call really recomputed


def test_noalloc_rejects_too_large_and_bad_arguments(se2):
    lib = se2.load_library()
    f = torch.zeros(16, device="cuda")
    # N = 512, M = 128 needs more scratch than the fixed array holds
    st = lib.se2_convolve_noalloc(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                  ctypes.c_void_p(f.data_ptr() + 8), 512, 128, 1, None)
    assert st == 2 and b"scratch" in lib.se2_last_error()
    assert lib.se2_convolve_noalloc(None, None, None, 32, 16, 1, None) == 1
    assert lib.se2_convolve_noalloc(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                    ctypes.c_void_p(f.data_ptr() + 8), 48, 16, 1, None) == 2
