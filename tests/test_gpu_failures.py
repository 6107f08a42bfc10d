"""Failure paths made on the host or by bounded device checks, none of which
faults the GPU:

* an injected device-allocation failure at every allocation of plan creation
  returns SE2_ERR_OOM and leaks nothing (se2_debug_fail_alloc /
  se2_debug_alloc_stats);
* SE2_CHECK_FINITE reports a NaN or infinity in an output as SE2_ERR_NUMERIC
  at se2_plan_status, which then clears; finite outputs and plans without the
  flag report SE2_OK.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OOM, NUMERIC = 3, 6


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    return m


@pytest.mark.parametrize("make", [
    lambda se2: se2.Plan(64, 16, batch=3, flags=se2.HOST_STAGING | se2.CHECK_FINITE),
    lambda se2: se2.Plan(256, 64, batch=2, precision="split_bf16"),
    lambda se2: se2.Plan(32, 8, batch=2, precision="f64", flags=se2.MASS_RENORM),
    lambda se2: se2.GridPlan((9, 11, 13), (12, 14, 16), batch=2),
])
def test_injected_allocation_failure_returns_oom_without_leaks(se2, make):
    live0, total0 = se2.alloc_stats()
    plan = make(se2)                       # count the allocations of one creation
    live1, total1 = se2.alloc_stats()
    n_alloc = total1 - total0
    assert n_alloc >= 2 and live1 - live0 == n_alloc
    plan.close()
    assert se2.alloc_stats()[0] == live0
    for n in range(1, n_alloc + 1):
        se2.fail_alloc(n)
        try:
            with pytest.raises(se2.SE2Error) as ei:
                make(se2)
            assert ei.value.status == OOM
        finally:
            se2.fail_alloc(0)
        assert se2.alloc_stats()[0] == live0, f"allocation {n} failing leaked memory"
    plan = make(se2)                       # creation works again afterwards
    plan.close()


def _grid(B, M, N, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.rand((B, M, N, N), generator=g).cuda()


def test_check_finite_flags_nan_and_inf_outputs(se2):
    N, M, B = 64, 16, 3
    plan = se2.Plan(N, M, batch=B, flags=se2.CHECK_FINITE)
    C, _ = se2.coeffs(plan, _grid(B, M, N, 1))
    f = _grid(B, M, N, 2)
    se2.convolve(plan, f, C)
    plan.status()                          # finite: no error
    bad = f.clone()
    bad[1, 3, 5, 7] = float("nan")
    se2.convolve(plan, bad, C)
    with pytest.raises(se2.SE2Error) as ei:
        plan.status()
    assert ei.value.status == NUMERIC
    plan.status()                          # the error word was cleared
    bad[1, 3, 5, 7] = float("inf")
    se2.convolve_chain_all(plan, bad, [C, C])
    with pytest.raises(se2.SE2Error) as ei:
        plan.status()
    assert ei.value.status == NUMERIC
    # without the flag nothing is checked
    plain = se2.Plan(N, M, batch=B)
    out = se2.convolve(plain, bad, C)
    plain.status()
    assert not torch.isfinite(out).all()


def test_check_finite_on_the_adjoint_and_separable_paths(se2):
    N, M, B = 32, 8, 2
    plan = se2.Plan(N, M, batch=B, flags=se2.CHECK_FINITE)
    params = torch.tensor([[[0.03, 0.3, 0.0]]] * B, dtype=torch.float64, device="cuda")
    k = torch.ones(B, dtype=torch.int32, device="cuda")
    tab = se2.separable_tables(plan, params, k)
    f = _grid(B, M, N, 3)
    f[0, 0, 0, 0] = float("nan")
    se2.convolve_separable(plan, f, tab)
    with pytest.raises(se2.SE2Error) as ei:
        plan.status()
    assert ei.value.status == NUMERIC
