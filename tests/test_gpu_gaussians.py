"""The analytic SE(2) inputs on the GPU (se2_sample_se2_gaussian,
se2_sample_deformed_gaussian) against the FP64 oracle, and the paper's chain
experiments with the matrix-log Gaussian kernel (Section 6.3: a triple
convolution f * rho^(3), and every V_p, p = 1..6, by Algorithm 6) at
power-of-two grids.  Errors are normwise: max|gpu - oracle| / max|oracle|."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import se2_gaussians as G  # noqa: E402
from oracle import se2_oracle as O  # noqa: E402

TOL = {"f32": 1e-5, "f64": 1e-10}
SAMPLE_TOL = {"f32": 1e-6, "f64": 1e-13}


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


SIGMA_GEN = [[0.02, 0.004, 0.001], [0.004, 0.03, -0.002], [0.001, -0.002, 0.5]]
SE2_CASES = [
    # (N, M, beta, Sigma or sigma2, images, origin_zero)
    (64, 32, (0.0, 0.0, math.pi / 4), 0.005, 1, False),        # Eq. gbS0, shifted pi/4
    (32, 16, (0.1, -0.2, 0.3), SIGMA_GEN, 1, False),           # general mean and covariance
    (32, 64, (0.05, 0.0, 2.0), SIGMA_GEN, 0, True),            # no images, origin-zero grid
    (16, 8, (0.0, 0.0, math.pi / 7), 0.0029, 2, False),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", range(len(SE2_CASES)))
def test_se2_gaussian_sampler(se2, prec, case):
    N, M, beta, S, images, oz = SE2_CASES[case]
    plan = se2.Plan(N, M, batch=1, precision=prec, flags=se2.GRID_ORIGIN_ZERO if oz else 0)
    if isinstance(S, float):
        got = se2.sample_se2_gaussian(plan, beta, sigma2=S, images=images)
        Sig = S * np.eye(3)
    else:
        got = se2.sample_se2_gaussian(plan, beta, Sigma=S, images=images)
        Sig = np.array(S)
    want = G.se2_gaussian(N, M, beta, Sig, images=images, origin_zero=oz)
    got = got[0].double().cpu().numpy()
    assert _rel(got, want) < SAMPLE_TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("oz", [False, True])
def test_deformed_gaussian_sampler(se2, prec, oz):
    N, M = 64, 32
    H = [[40.0, 6.0], [4.0, 120.0]]   # only the symmetric part enters
    plan = se2.Plan(N, M, batch=1, precision=prec, flags=se2.GRID_ORIGIN_ZERO if oz else 0)
    got = se2.sample_deformed_gaussian(plan, H, math.pi / 4, 0.0125, images=1)[0].double().cpu().numpy()
    want = G.deformed_gaussian(N, M, np.array(H), math.pi / 4, 0.0125, images=1, origin_zero=oz)
    assert _rel(got, want) < SAMPLE_TOL[prec]


def _inputs(se2, plan, H, s, nu, sigma2):
    f = se2.sample_deformed_gaussian(plan, H, nu, s, images=1)
    rho = se2.sample_se2_gaussian(plan, (0.0, 0.0, nu), sigma2=sigma2, images=1)
    N, M = plan.N, plan.M
    F = G.deformed_gaussian(N, M, np.array(H), nu, s, images=1)
    P = G.se2_gaussian_kernel(N, M, sigma2, nu, images=1)
    return f, rho, F, P


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_triple_convolution_with_gbs0_kernel(se2, prec):
    """f * rho^(3) with f = f_H^{nu,s}, H = diag(0.025, 0.0025)^-1, s = 0.0125,
    nu = pi/4 and rho of Eq. gbS0 with sigma^2 = 0.005 shifted by pi/4, as in
    the paper's triple-convolution experiment, on a 64 x 64 x 128 grid; the
    oracle raises rho's coefficients to the third power (Eq. MatSqKfgG)."""
    N, M = 64, 128
    plan = se2.Plan(N, M, batch=1, precision=prec)
    H = [[1 / 0.025, 0.0], [0.0, 1 / 0.0025]]
    f, rho, F, P = _inputs(se2, plan, H, 0.0125, math.pi / 4, 0.005)
    C, ls = se2.coeffs(plan, rho, normalize=(prec == "f32"))
    out = se2.convolve_chain(plan, f, [C, C, C], None if ls is None else [ls, ls, ls])
    got = out[0].double().cpu().numpy()
    want = O.convolve_power(F, P, 3)
    assert _rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_all_six_powers_with_gbs0_kernel(se2, prec):
    """V_p = f * rho^(p), p = 1..6, from one forward transform (Algorithm 6)
    with f = f_H^{nu,s}, H = diag(0.0143, 0.0014)^-1, s = 0.0071, nu = pi/7 and
    rho of Eq. gbS0 with sigma^2 = 0.0029 shifted by pi/7, on 64 x 64 x 64."""
    N, M = 64, 64
    plan = se2.Plan(N, M, batch=1, precision=prec)
    H = [[1 / 0.0143, 0.0], [0.0, 1 / 0.0014]]
    f, rho, F, P = _inputs(se2, plan, H, 0.0071, math.pi / 7, 0.0029)
    C, ls = se2.coeffs(plan, rho, normalize=(prec == "f32"))
    out = se2.convolve_chain_all(plan, f, [C] * 6, None if ls is None else [ls] * 6)
    out = out[:, 0].double().cpu().numpy()
    want = O.convolve_all(F, [P] * 6)
    for p in range(6):
        assert _rel(out[p], want[p]) < TOL[prec], p


def test_sampler_invalid_arguments(se2):
    plan = se2.Plan(32, 16, batch=1)
    with pytest.raises(se2.SE2Error):
        se2.sample_se2_gaussian(plan, (0, 0, 0), Sigma=[[1, 0, 0], [0, -1, 0], [0, 0, 1]])   # not positive definite
    with pytest.raises(se2.SE2Error):
        se2.sample_se2_gaussian(plan, (0, 0, 0), Sigma=[[1, 0.5, 0], [0, 1, 0], [0, 0, 1]])  # not symmetric
    with pytest.raises(se2.SE2Error):
        se2.sample_se2_gaussian(plan, (0, 0, 0), sigma2=0.01, images=9)
    with pytest.raises(se2.SE2Error):
        se2.sample_deformed_gaussian(plan, [[1, 0], [0, -2]], 0.0, 0.1)
    with pytest.raises(se2.SE2Error):
        se2.sample_deformed_gaussian(plan, [[1, 0], [0, 2]], 0.0, 0.0)
    with pytest.raises(ValueError):
        se2.sample_se2_gaussian(plan, (0, 0), sigma2=0.01)
