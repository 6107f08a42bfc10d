"""se2_grid_ffc_at: one finite Fourier coefficient f^[k; L] (Eq. FkLv) read
from grid coefficients on the device, against the oracle's FFC of the same
samples (FP64 plan), for k in every sign pattern."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import se2_upsample as U  # noqa: E402


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    return m


@pytest.mark.parametrize("k", [(0, 0, 0), (1, -2, 3), (-3, 2, -1), (4, 5, -6), (-4, -5, 6), (0, -5, 6), (-1, 0, 0)])
def test_ffc_at_reads_eq_fklv(se2, k):
    L = (9, 11, 13)
    rng = np.random.default_rng(3)
    P = rng.standard_normal((2,) + L[::-1])
    plan = se2.GridPlan(L, batch=2, precision="f64")
    C = se2.grid_coeffs(plan, torch.from_numpy(P).cuda())
    k1, k2, k3 = k
    for index in range(2):
        got = se2.ffc_at(plan, C, k, index=index)
        full = U.ffc_odd(P[index])
        want = full[k3 % L[2], k2 % L[1], k1 % L[0]]
        assert abs(got - want) < 1e-13 * np.max(np.abs(full))


def test_ffc_at_rejects_out_of_range(se2):
    plan = se2.GridPlan((5, 5, 5), batch=1, precision="f64")
    C = se2.grid_coeffs(plan, torch.zeros((1, 5, 5, 5), dtype=torch.float64, device="cuda"))
    for k in [(3, 0, 0), (0, -3, 0), (0, 0, 3)]:
        with pytest.raises(se2.SE2Error):
            se2.ffc_at(plan, C, k)
    with pytest.raises(se2.SE2Error):
        se2.ffc_at(plan, C, (0, 0, 0), index=1)
