"""Host-side logic of the binding that needs no GPU: reading finite Fourier
coefficients out of a half spectrum (Eq. FkLv), checked against the oracle."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2504_05149_gb300 as se2  # noqa: E402
from oracle import se2_upsample as U  # noqa: E402


@pytest.mark.parametrize("k", [(0, 0, 0), (1, -2, 3), (-3, 2, -1), (4, 5, -6), (-4, -5, 6), (0, -5, 6)])
def test_ffc_at_reads_eq_fklv(k):
    L = (9, 11, 13)
    rng = np.random.default_rng(3)
    P = rng.standard_normal(L[::-1])
    # the half spectrum the grid plans produce: C = DFT(P) / |L|, x bins 0..Kx
    C = torch.from_numpy((np.fft.fftn(P) / P.size)[..., : (L[0] - 1) // 2 + 1][None].copy())
    plan = types.SimpleNamespace(Lx=L[0], Ly=L[1], Lr=L[2])
    got = se2.ffc_at(plan, C, k)
    full = U.ffc_odd(P)
    k1, k2, k3 = k
    want = full[k3 % L[2], k2 % L[1], k1 % L[0]]
    assert abs(got - want) < 1e-13 * np.max(np.abs(full))


def test_ffc_at_rejects_out_of_range():
    plan = types.SimpleNamespace(Lx=5, Ly=5, Lr=5)
    C = torch.zeros((1, 5, 5, 3), dtype=torch.complex128)
    with pytest.raises(ValueError):
        se2.ffc_at(plan, C, (3, 0, 0))
