"""Odd sampling grids L = 2K+1 with output on an N-grid >= L
(se2_grid_plan_*, Eqs. Qf, W, MatSKfgonG) against the FP64 oracle's series
definition.  Errors are normwise: max|gpu - oracle| / max|oracle|."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import se2_gaussians as G  # noqa: E402
from oracle import se2_upsample as U  # noqa: E402

TOL = {"f32": 1e-5, "f64": 1e-10}
NP = {"f32": np.float32, "f64": np.float64}


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


def _axes(L):
    Lx, Ly, Lr = L
    return (-0.5 + np.arange(Lx) / Lx, -0.5 + np.arange(Ly) / Ly, 2 * np.pi * np.arange(Lr) / Lr)


def deformed(L, H, nu, s):
    """f_H^{nu,s} (Eq. fHsnu) on the anisotropic grid Omega_L, [Lr][Ly][Lx]."""
    x, y, t = _axes(L)
    Y, X = np.meshgrid(y, x, indexing="ij")
    sp = np.exp(-(H[0][0] * X * X + (H[0][1] + H[1][0]) * X * Y + H[1][1] * Y * Y))
    return np.exp(-((t - nu) ** 2) / s)[:, None, None] * sp[None]


def se2_gauss(L, sigma2, nu):
    """rho of Eq. gbS0 shifted by nu, one lattice image, [Lr][Ly][Lx]."""
    x, y, t = _axes(L)
    T, Y, X = np.meshgrid(t, y, x, indexing="ij")
    return G.se2_gaussian_at(X, Y, T, (0.0, 0.0, nu), sigma2 * np.eye(3))


def _dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a.astype(NP[prec]))).cuda()


def _round(a, prec):
    return a.astype(NP[prec]).astype(np.float64)


CASES = [
    # (L = (Lx, Ly, Lr), N = (Nx, Ny, Nr), k, B)
    ((31, 33, 61), (36, 38, 76), 1, 1),     # the paper's single-convolution experiment shape
    ((7, 5, 9), (7, 5, 9), 2, 2),           # N = L, odd
    ((15, 17, 21), (32, 32, 32), 3, 3),     # upsampled chain
    ((9, 11, 13), (20, 21, 22), 0, 2),      # S_K[f] itself (no kernel)
    ((1, 3, 5), (4, 3, 8), 1, 1),           # K = 0 along x
    ((41, 43, 151), (41, 43, 151), 3, 1),   # the triple-convolution shape, N = L
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_grid_chain_matches_series(se2, prec, case):
    L, N, k, B = CASES[case]
    plan = se2.GridPlan(L, N, batch=B, precision=prec)
    Fs = [_round(deformed(L, [[1 / 0.03, 0.002], [0.002, 1 / 0.01]], math.pi / 2 + 0.3 * b, 0.05), prec)
          for b in range(B)]
    Ps = [[_round(se2_gauss(L, 0.004 + 0.001 * t, 0.2 * t + 0.1 * b), prec) for t in range(k)] for b in range(B)]
    f = _dev(np.stack(Fs)[:, :, :, :], prec)
    Cs = [se2.grid_coeffs(plan, _dev(np.stack([Ps[b][t] for b in range(B)]), prec)) for t in range(k)]
    n0 = plan.launches()
    out = se2.grid_convolve_chain(plan, f, Cs)
    torch.cuda.synchronize()
    assert plan.launches() - n0 == 6
    got = out.double().cpu().numpy()
    Nx, Ny, Nr = N
    for b in range(B):
        want = U.series(Fs[b], Ps[b], (Nr, Ny, Nx)).real
        assert _rel(got[b], want) < TOL[prec], b


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_grid_coeffs(se2, prec):
    L = (9, 7, 11)
    plan = se2.GridPlan(L, batch=2, precision=prec)
    rng = np.random.default_rng(3)
    P = _round(rng.standard_normal((2, 11, 7, 9)), prec)
    C = se2.grid_coeffs(plan, _dev(P, prec)).cpu().numpy()
    want = np.fft.fftn(P, axes=(1, 2, 3))[..., :5] / (9 * 7 * 11)
    assert _rel(C, want) < {"f32": 1e-6, "f64": 1e-13}[prec]


def test_grid_shared_kernel_and_paper_e4(se2):
    """The paper's single-convolution experiment (L = (31, 33, 61), output
    36 x 38 x 76; f: H = diag(0.03, 0.01)^-1, s = 0.01, nu = pi/2; rho the
    radial deformed Gaussian U = (1/0.02) I with the same s, nu) on a batch
    of 4 sharing the kernel."""
    L, N = (31, 33, 61), (36, 38, 76)
    plan = se2.GridPlan(L, N, batch=4, precision="f32", flags=se2.SHARED_KERNEL)
    F = _round(deformed(L, [[1 / 0.03, 0], [0, 1 / 0.01]], math.pi / 2, 0.01), "f32")
    P = _round(deformed(L, [[1 / 0.02, 0], [0, 1 / 0.02]], math.pi / 2, 0.01), "f32")
    f = _dev(np.stack([F * (b + 1) for b in range(4)]), "f32")
    C = se2.grid_coeffs(plan, _dev(P[None], "f32"))
    out = se2.grid_convolve_chain(plan, f, [C]).double().cpu().numpy()
    want = U.series(F, [P], (76, 38, 36)).real
    for b in range(4):
        assert _rel(out[b], (b + 1) * want) < 1e-5


def test_grid_plan_errors(se2):
    with pytest.raises(se2.SE2Error) as e:
        se2.GridPlan((8, 9, 9))
    assert e.value.status == 2
    with pytest.raises(se2.SE2Error) as e:
        se2.GridPlan((9, 9, 9), (9, 8, 9))
    assert e.value.status == 1
    plan = se2.GridPlan((5, 5, 5), batch=1)
    f = torch.zeros((2, 5, 5, 5), device="cuda")
    with pytest.raises(se2.SE2Error):
        se2.grid_convolve_chain(plan, f, [])          # B above the plan's batch


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("L,N", [
    ((255, 3, 5), (1024, 3, 5)),     # largest sampling and output sizes along x
    ((3, 255, 5), (3, 1024, 5)),     # along y (FP64 column tile with the table in global memory)
    ((5, 3, 255), (5, 4, 1024)),     # along theta
])
def test_grid_largest_sizes(se2, prec, L, N):
    plan = se2.GridPlan(L, N, batch=1, precision=prec)
    rng = np.random.default_rng(sum(L))
    F = _round(rng.standard_normal(L[::-1]), prec)
    P = _round(rng.standard_normal(L[::-1]), prec)
    C = se2.grid_coeffs(plan, _dev(P[None], prec))
    out = se2.grid_convolve_chain(plan, _dev(F[None], prec), [C])[0].double().cpu().numpy()
    want = U.series(F, [P], N[::-1]).real
    assert _rel(out, want) < {"f32": 1e-5, "f64": 1e-10}[prec]


def test_grid_longest_chain(se2):
    """k = 32 kernels (the largest chain), batch 2 with per-problem kernels."""
    L, N = (5, 7, 9), (6, 8, 10)
    B, k = 2, 32
    plan = se2.GridPlan(L, N, batch=B, precision="f64")
    Fs = [deformed(L, [[30, 0], [0, 60]], 1.0 + b, 0.3) for b in range(B)]
    Ps = [[1.0 + 0.1 * se2_gauss(L, 0.01 + 0.0005 * t, 0.05 * t + b) for t in range(k)] for b in range(B)]
    Cs = [se2.grid_coeffs(plan, _dev(np.stack([Ps[b][t] for b in range(B)]), "f64")) for t in range(k)]
    out = se2.grid_convolve_chain(plan, _dev(np.stack(Fs), "f64"), Cs).cpu().numpy()
    for b in range(B):
        assert _rel(out[b], U.series(Fs[b], Ps[b], N[::-1]).real) < 1e-10


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_grid_samplers(se2, prec):
    """The samplers on a grid plan's odd, anisotropic Omega_L (one lattice
    image) against the oracle's pointwise functions."""
    L = (31, 33, 61)
    plan = se2.GridPlan(L, (36, 38, 76), batch=1, precision=prec)
    tol = {"f32": 1e-6, "f64": 1e-13}[prec]
    beta, Sig = (0.05, -0.1, math.pi / 4), np.array([[0.02, 0.004, 0.001], [0.004, 0.03, -0.002], [0.001, -0.002, 0.5]])
    got = se2.sample_se2_gaussian(plan, beta, Sigma=Sig, images=0)[0].double().cpu().numpy()
    x, y, t = _axes(L)
    T, Y, X = np.meshgrid(t, y, x, indexing="ij")
    assert _rel(got, G.se2_gaussian_at(X, Y, T, beta, Sig)) < tol
    H = [[1 / 0.03, 0.0], [0.0, 1 / 0.01]]
    got = se2.sample_deformed_gaussian(plan, H, math.pi / 2, 0.01, images=0)[0].double().cpu().numpy()
    assert _rel(got, deformed(L, H, math.pi / 2, 0.01)) < tol


def test_paper_e4_sampled_on_the_gpu(se2):
    """The paper's single-convolution experiment with both inputs sampled by
    the grid plan's samplers (f: H = diag(0.03, 0.01)^-1; rho: U = (1/0.02) I;
    s = 0.01, nu = pi/2), against the oracle's series."""
    L, N = (31, 33, 61), (36, 38, 76)
    plan = se2.GridPlan(L, N, batch=1, precision="f32")
    H, U_ = [[1 / 0.03, 0.0], [0.0, 1 / 0.01]], [[1 / 0.02, 0.0], [0.0, 1 / 0.02]]
    f = se2.sample_deformed_gaussian(plan, H, math.pi / 2, 0.01, images=0)
    rho = se2.sample_deformed_gaussian(plan, U_, math.pi / 2, 0.01, images=0)
    out = se2.grid_convolve_chain(plan, f, [se2.grid_coeffs(plan, rho)])[0].double().cpu().numpy()
    want = U.series(deformed(L, H, math.pi / 2, 0.01), [deformed(L, U_, math.pi / 2, 0.01)], N[::-1]).real
    assert _rel(out, want) < 1e-5


def _peak_theta(V, Nr):
    """Angle (in units of pi) of the theta slice holding the largest value."""
    l = np.unravel_index(np.argmax(V), V.shape)[0]
    return 2.0 * l / Nr


def test_paper_triple_convolution_e5(se2):
    """The paper's triple convolution: K = (20, 21, 50), L = (41, 43, 101),
    output 41 x 43 x 151; f = f_H^{pi/4, 0.0125}, H = diag(0.025, 0.0025)^-1,
    rho of Eq. gbS0 with sigma^2 = 0.005 shifted by pi/4.  Against the
    oracle's series, and the mass of f * rho^(3) sits at theta = pi, where
    the paper slices it (each factor adds pi/4)."""
    L, N = (41, 43, 101), (41, 43, 151)
    plan = se2.GridPlan(L, N, batch=1, precision="f32")
    H = [[1 / 0.025, 0.0], [0.0, 1 / 0.0025]]
    f = se2.sample_deformed_gaussian(plan, H, math.pi / 4, 0.0125, images=0)
    rho = se2.sample_se2_gaussian(plan, (0.0, 0.0, math.pi / 4), sigma2=0.005, images=0)
    C = se2.grid_coeffs(plan, rho)
    out = se2.grid_convolve_chain(plan, f, [C, C, C])[0].double().cpu().numpy()
    F = f[0].double().cpu().numpy()
    P = rho[0].double().cpu().numpy()
    want = U.series(F, [P, P, P], N[::-1]).real
    assert _rel(out, want) < 1e-5
    assert abs(_peak_theta(out, N[2]) - 1.0) <= 2.0 / N[2] + 1e-12


def test_paper_six_powers_e6(se2):
    """The paper's Algorithm 6 experiment: K = (15, 16, 30), grid 31 x 33 x 61;
    f = f_H^{pi/7, 0.0071}, H = diag(0.0143, 0.0014)^-1, rho of Eq. gbS0 with
    sigma^2 = 0.0029 shifted by pi/7.  V_p = f * rho^(p), p = 1..6, against the
    oracle's series; V_p peaks at theta = (p+1) pi/7, where the paper slices it."""
    L = (31, 33, 61)
    plan = se2.GridPlan(L, batch=1, precision="f32")
    H = [[1 / 0.0143, 0.0], [0.0, 1 / 0.0014]]
    f = se2.sample_deformed_gaussian(plan, H, math.pi / 7, 0.0071, images=0)
    rho = se2.sample_se2_gaussian(plan, (0.0, 0.0, math.pi / 7), sigma2=0.0029, images=0)
    C = se2.grid_coeffs(plan, rho)
    F = f[0].double().cpu().numpy()
    P = rho[0].double().cpu().numpy()
    for p in range(1, 7):
        out = se2.grid_convolve_chain(plan, f, [C] * p)[0].double().cpu().numpy()
        assert _rel(out, U.series(F, [P] * p, L[::-1]).real) < 1e-5, p
        assert abs(_peak_theta(out, L[2]) - (p + 1) / 7.0) <= 2.0 / L[2] + 1e-12, p


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_grid_chain_all_algorithm6(se2, prec):
    """se2_grid_convolve_chain_all: V_1..V_k from one forward transform
    (Algorithm 6) on an odd upsampled grid, per-problem kernels, against the
    oracle's series for every p; and the paper's six-power experiment."""
    L, N, B, k = (9, 11, 13), (12, 14, 20), 2, 4
    plan = se2.GridPlan(L, N, batch=B, precision=prec)
    Fs = [_round(deformed(L, [[30, 0], [0, 60]], 1.0 + b, 0.3), prec) for b in range(B)]
    Ps = [[_round(se2_gauss(L, 0.008 + 0.001 * t, 0.1 * t + 0.2 * b), prec) for t in range(k)] for b in range(B)]
    Cs = [se2.grid_coeffs(plan, _dev(np.stack([Ps[b][t] for b in range(B)]), prec)) for t in range(k)]
    n0 = plan.launches()
    V = se2.grid_convolve_chain_all(plan, _dev(np.stack(Fs), prec), Cs)
    torch.cuda.synchronize()
    assert plan.launches() - n0 == 3 + 3 * k
    V = V.double().cpu().numpy()
    for b in range(B):
        for p in range(1, k + 1):
            assert _rel(V[p - 1, b], U.series(Fs[b], Ps[b][:p], N[::-1]).real) < TOL[prec], (b, p)

    # the paper's six powers (K = (15, 16, 30), grid 31 x 33 x 61), all at once
    L6 = (31, 33, 61)
    plan6 = se2.GridPlan(L6, batch=1, precision="f32")
    f = se2.sample_deformed_gaussian(plan6, [[1 / 0.0143, 0.0], [0.0, 1 / 0.0014]], math.pi / 7, 0.0071, images=0)
    rho = se2.sample_se2_gaussian(plan6, (0.0, 0.0, math.pi / 7), sigma2=0.0029, images=0)
    C = se2.grid_coeffs(plan6, rho)
    V6 = se2.grid_convolve_chain_all(plan6, f, [C] * 6)[:, 0].double().cpu().numpy()
    F = f[0].double().cpu().numpy()
    P = rho[0].double().cpu().numpy()
    for p in range(1, 7):
        assert _rel(V6[p - 1], U.series(F, [P] * p, L6[::-1]).real) < 1e-5, p
