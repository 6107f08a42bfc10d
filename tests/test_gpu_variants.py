"""The opt-in FP32 variants give the default path's results bit for bit.

* SE2_FAST2=1: units A and C with bulk row copies and the real-FFT split in
  registers (N = 256 or 64).
* SE2_FLOW=1: the whole batch as one persistent dataflow launch (N = 256).
* SE2_L2_DISCARD=1: unit C drops the scratch rows it has consumed from L2;
  the scratch slots are rewritten before any later read, so repeated calls,
  the pipelined schedule and the chain outputs are unchanged.

Both perform the same floating-point operations in the same order as the
default units, so the outputs are identical; the default path itself is
checked against the FP64 oracle in test_gpu_parity.py.  One case per variant
is also checked against the oracle directly.  Pointers that are not 16-byte
aligned fall back to the default units.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import se2_oracle as O  # noqa: E402


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    return m


def _inputs(N, M, B, k, seed):
    Fs = [synth.sample_bumps(N, M, synth.make_problem(seed, b, N, M, n_bumps=6).bumps).astype(np.float32)
          for b in range(B)]
    kps = [synth.KernelParams(0.02 + 0.007 * i, 0.2 + 0.05 * i, 0.1 * i) for i in range(k)]
    Ps = [np.stack([synth.sample_kernel(N, M, kp) for _ in range(B)]).astype(np.float32) for kp in kps]
    return np.stack(Fs), Ps


def _convolve(se2, env, F, Ps, normalize, offset=False):
    old = {key: os.environ.get(key) for key in env}
    os.environ.update(env)
    try:
        B, M, N, _ = F.shape
        plan = se2.Plan(N, M, batch=B)
    finally:
        for key, v in old.items():
            if v is None:
                os.environ.pop(key, None)
            else:
                os.environ[key] = v
    if offset:   # f and out 4 bytes past a 16-byte boundary
        big = torch.empty(F.size + 1, device="cuda")
        f = big[1:].view(F.shape)
        f.copy_(torch.from_numpy(F))
        ob = torch.empty(F.size + 1, device="cuda")
        out = ob[1:].view(F.shape)
    else:
        f = torch.from_numpy(F).cuda()
        out = torch.empty_like(f)
    Cs, Ls = [], []
    for P in Ps:
        C, ls = se2.coeffs(plan, torch.from_numpy(P).cuda(), normalize=normalize)
        Cs.append(C)
        Ls.append(ls)
    se2.convolve_chain(plan, f, Cs, Ls if normalize else None, out=out)
    plan.status()
    torch.cuda.synchronize()
    return out.cpu().numpy(), plan


@pytest.mark.parametrize("N,M,B,k,normalize", [(256, 64, 3, 1, False), (256, 32, 2, 3, True), (64, 32, 5, 2, False),
                                               (64, 16, 1, 1, True)])
def test_bulk_copy_units_match_default(se2, N, M, B, k, normalize):
    F, Ps = _inputs(N, M, B, k, 31)
    ref, _ = _convolve(se2, {}, F, Ps, normalize)
    got, _ = _convolve(se2, {"SE2_FAST2": "1"}, F, Ps, normalize)
    assert np.array_equal(got, ref)
    mis, _ = _convolve(se2, {"SE2_FAST2": "1"}, F, Ps, normalize, offset=True)
    assert np.array_equal(mis, ref)


@pytest.mark.parametrize("M,B,k,normalize", [(64, 1, 1, False), (64, 6, 1, False), (32, 9, 2, True), (16, 5, 3, False)])
def test_dataflow_kernel_matches_default(se2, M, B, k, normalize):
    N = 256
    F, Ps = _inputs(N, M, B, k, 32)
    ref, _ = _convolve(se2, {}, F, Ps, normalize)
    got, plan = _convolve(se2, {"SE2_FLOW": "1"}, F, Ps, normalize)
    assert np.array_equal(got, ref)


def test_dataflow_kernel_is_one_launch_and_timed(se2):
    N, M, B = 256, 32, 7
    F, Ps = _inputs(N, M, B, 1, 33)
    old = os.environ.get("SE2_FLOW")
    os.environ["SE2_FLOW"] = "1"
    try:
        plan = se2.Plan(N, M, batch=B)
    finally:
        if old is None:
            os.environ.pop("SE2_FLOW")
        else:
            os.environ["SE2_FLOW"] = old
    f = torch.from_numpy(F).cuda()
    C, _ = se2.coeffs(plan, torch.from_numpy(Ps[0]).cuda())
    plan.timing(True)
    n0 = plan.launches()
    se2.convolve(plan, f, C)
    torch.cuda.synchronize()
    stats = plan.timing_read()
    plan.timing(False)
    assert plan.launches() - n0 == 1
    assert stats[3][1] == 1 and stats[3][0] > 0 and sum(c for _, c in stats[:3]) == 0


def test_dataflow_kernel_against_oracle(se2):
    """Two problems at 256^2 x 16 with a 2-kernel chain, against the FP64 oracle."""
    N, M, B = 256, 16, 2
    F, Ps = _inputs(N, M, B, 2, 34)
    got, _ = _convolve(se2, {"SE2_FLOW": "1"}, F, Ps, False)
    for b in range(B):
        want = O.convolve_chain(F[b].astype(np.float64), [P[b].astype(np.float64) for P in Ps])
        err = np.max(np.abs(got[b] - want)) / np.max(np.abs(want))
        assert err < 1e-5, err


@pytest.mark.parametrize("N,M,B,k,normalize", [(256, 64, 6, 1, False), (256, 32, 5, 3, True), (64, 32, 9, 2, False)])
def test_l2_discard_matches_default(se2, N, M, B, k, normalize):
    F, Ps = _inputs(N, M, B, k, 35)
    ref, _ = _convolve(se2, {}, F, Ps, normalize)
    for _ in range(2):   # the second call reuses scratch slots whose lines were discarded
        got, _ = _convolve(se2, {"SE2_L2_DISCARD": "1"}, F, Ps, normalize)
        assert np.array_equal(got, ref)


def test_l2_discard_chain_all_and_backward(se2):
    """Every chain prefix (unit C after each running product) and the input
    gradient (unit C after the adjoint lines) with discarding on."""
    N, M, B, k = 64, 16, 3, 3
    F, Ps = _inputs(N, M, B, k, 36)
    outs = {}
    for env in ({}, {"SE2_L2_DISCARD": "1"}):
        old = {key: os.environ.get(key) for key in env}
        os.environ.update(env)
        try:
            plan = se2.Plan(N, M, batch=B)
        finally:
            for key, v in old.items():
                if v is None:
                    os.environ.pop(key, None)
                else:
                    os.environ[key] = v
        f = torch.from_numpy(F).cuda()
        Cs = [se2.coeffs(plan, torch.from_numpy(P).cuda())[0] for P in Ps]
        allp = se2.convolve_chain_all(plan, f, Cs)
        g = torch.from_numpy(F[::-1].copy()).cuda()
        gf, _ = se2.backward(plan, g, Cs[0])
        plan.status()
        torch.cuda.synchronize()
        outs[bool(env)] = (allp.cpu().numpy(), gf.cpu().numpy())
    assert np.array_equal(outs[True][0], outs[False][0])
    assert np.array_equal(outs[True][1], outs[False][1])
