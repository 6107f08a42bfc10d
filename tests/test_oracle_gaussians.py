"""Pins of the oracle's analytic SE(2) input families (Eqs. gxyt, fbS, gbS0,
fHsnu) against library routines, closed forms and group identities that do
not reuse the oracle's own formulas."""
import math

import numpy as np
import pytest

import synth
from oracle import direct
from oracle import se2_gaussians as G
from oracle import se2_oracle as O

sl = pytest.importorskip("scipy.linalg")


def _hat(v1, v2, phi):
    return np.array([[0.0, -phi, v1], [phi, 0.0, v2], [0.0, 0.0, 0.0]])


def test_log_matches_scipy_logm():
    """The principal matrix logarithm of Eq. gxyt matrices, away from theta = pi."""
    rng = np.random.default_rng(11)
    for _ in range(60):
        x1, x2 = rng.uniform(-2, 2, 2)
        t = rng.uniform(-math.pi + 0.05, math.pi - 0.05)
        L = np.real(sl.logm(G.se2_matrix(x1, x2, t)))
        v1, v2, phi = G.se2_log(x1, x2, t)
        np.testing.assert_allclose([v1, v2, phi], [L[0, 2], L[1, 2], L[1, 0]], rtol=0, atol=1e-12)
        assert abs(L[0, 0]) < 1e-12 and abs(L[0, 1] + L[1, 0]) < 1e-12


@pytest.mark.parametrize("t", [0.0, 1e-9, -1e-7, 2.0, 3.0, math.pi - 1e-6, math.pi, 4.0, 2 * math.pi - 0.3, -5.0])
def test_exp_of_log_is_identity(t):
    """expm(log(g)^) = g, including the branch points near theta = pi and
    angles outside (-pi, pi] (reduced to the principal angle)."""
    x1, x2 = 0.37, -0.81
    v1, v2, phi = G.se2_log(x1, x2, t)
    assert -math.pi < float(phi) <= math.pi
    np.testing.assert_allclose(sl.expm(_hat(float(v1), float(v2), float(phi))), G.se2_matrix(x1, x2, t),
                               rtol=0, atol=1e-12)


def test_theta_zero_slice_is_euclidean_gaussian():
    """At R = I the logarithm is (x, 0), so f_{0,Sigma} is the Euclidean
    Gaussian with the translation block of Sigma^-1."""
    Sigma = np.array([[0.02, 0.004, 0.001], [0.004, 0.03, -0.002], [0.001, -0.002, 0.5]])
    Si = np.linalg.inv(Sigma)
    x = np.linspace(-0.5, 0.5, 17)
    X, Y = np.meshgrid(x, x, indexing="ij")
    want = np.exp(-0.5 * (Si[0, 0] * X * X + 2 * Si[0, 1] * X * Y + Si[1, 1] * Y * Y))
    got = G.se2_gaussian_at(X, Y, 0.0 * X, (0, 0, 0), Sigma)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)


def test_isotropic_kernel_is_radial_with_half_angle_norm():
    """For Sigma = sigma^2 I: |v| = |x| (phi/2) / sin(phi/2) (V(phi) is a
    scaled rotation by phi/2), so rho depends on |x| only."""
    rng = np.random.default_rng(5)
    s2 = 0.05
    for _ in range(40):
        r, a1, a2 = rng.uniform(0, 0.6), rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi)
        t = rng.uniform(-math.pi, math.pi)
        f1 = G.se2_gaussian_at(r * math.cos(a1), r * math.sin(a1), t, (0, 0, 0), s2 * np.eye(3))
        f2 = G.se2_gaussian_at(r * math.cos(a2), r * math.sin(a2), t, (0, 0, 0), s2 * np.eye(3))
        h = t / 2
        nv = r * (h / math.sin(h) if h != 0 else 1.0)
        want = math.exp(-(nv * nv + t * t) / (2 * s2))
        assert f1 == pytest.approx(want, rel=1e-12)
        assert f2 == pytest.approx(want, rel=1e-12)


def test_left_invariance_in_beta():
    """f_{beta,Sigma}(beta o g) = f_{0,Sigma}(g) (Eq. fbS evaluates at beta^-1 o g)."""
    rng = np.random.default_rng(8)
    Sigma = np.array([[0.05, 0.01, 0.0], [0.01, 0.02, 0.005], [0.0, 0.005, 0.3]])
    for _ in range(30):
        beta = tuple(rng.uniform(-0.5, 0.5, 2)) + (rng.uniform(0, 2 * math.pi),)
        g = tuple(rng.uniform(-0.4, 0.4, 2)) + (rng.uniform(-2.5, 2.5),)
        bg = G.se2_compose(beta, g)
        a = G.se2_gaussian_at(*bg, beta, Sigma)
        b = G.se2_gaussian_at(*g, (0, 0, 0), Sigma)
        assert abs(a - b) <= 1e-12 * b


def test_shifted_kernel_is_angle_translate():
    """beta = (0, R_nu) with isotropic Sigma shifts rho by nu in theta: on a
    grid where nu is a whole number of angle steps the samples roll."""
    N, M = 16, 32
    nu = 2 * math.pi * 5 / M
    a = G.se2_gaussian_kernel(N, M, 0.01, nu, images=1)
    b = G.se2_gaussian_kernel(N, M, 0.01, 0.0, images=1)
    assert np.max(np.abs(a - np.roll(b, 5, axis=0))) <= 1e-13 * np.max(b)


@pytest.mark.parametrize("s2,nu", [(0.01, 0.8), (0.005, math.pi / 4), (0.0029, math.pi / 7)])
def test_gbs0_kernel_spectral_scheme_equals_group_quadrature(s2, nu):
    """rho of Eq. gbS0 is radial in translations, so the spectral scheme with
    its samples equals the group-law rectangle rule (Theorem f*gP(1)), which
    evaluates the kernel at rotated arguments through a separately written
    half-angle formula (oracle/direct.c, kind 2)."""
    N, M = 16, 8
    prob = synth.make_problem(1, 3, N, M, n_bumps=3)
    F = synth.sample_bumps(N, M, prob.bumps)
    P = G.se2_gaussian_kernel(N, M, s2, nu, images=1)
    quad = direct.group_quadrature(F, 2, [s2, nu], images=1)
    got = O.convolve(F, P)
    assert np.max(np.abs(got - quad)) / np.max(np.abs(quad)) < 1e-12


def test_anisotropic_se2_gaussian_is_not_radial():
    """Negative check: with Sigma anisotropic in translations the scheme no
    longer equals the group-law quadrature of the isotropic kernel family."""
    N, M = 16, 8
    prob = synth.make_problem(1, 3, N, M, n_bumps=3)
    F = synth.sample_bumps(N, M, prob.bumps)
    P = G.se2_gaussian(N, M, (0, 0, 0.8), np.diag([0.004, 0.02, 0.01]), images=1)
    quad = direct.group_quadrature(F, 2, [0.01, 0.8], images=1)
    assert np.max(np.abs(O.convolve(F, P) - quad)) / np.max(np.abs(quad)) > 1e-2


def test_deformed_gaussian_integral_closed_form():
    """The rectangle rule of the lattice-periodised exp(-x^T H x) over the unit
    torus is the plane integral pi / sqrt(det H) (spectrally accurate); the
    angular factor integrates to sqrt(pi s) when it decays inside [0, 2 pi)."""
    N, M = 64, 128
    H = np.linalg.inv(np.array([[0.03, 0.008], [0.008, 0.01]]))
    nu, s = math.pi, 0.4
    F = G.deformed_gaussian(N, M, H, nu, s, images=3)
    integral = F.sum() * (1.0 / (N * N)) * (2 * math.pi / M)
    want = math.pi / math.sqrt(np.linalg.det(H)) * math.sqrt(math.pi * s)
    assert abs(integral - want) / want < 1e-9
    # H enters as x^T H x (no factor 1/2): the peak value and one off-axis point
    x = -0.5 + np.arange(N) / N
    assert F[M // 2, N // 2, N // 2] == pytest.approx(1.0, rel=1e-12)
    i, j = N // 2 + 5, N // 2 - 3
    q = H[0, 0] * x[i] ** 2 + 2 * H[0, 1] * x[i] * x[j] + H[1, 1] * x[j] ** 2
    g0 = G.deformed_gaussian(N, M, H, nu, s, images=0)
    assert g0[M // 2, j, i] == pytest.approx(math.exp(-q), rel=1e-12)


def test_chain_of_gbs0_kernels_keeps_mass_and_matches_group_quadrature():
    """The 2-fold chain f * rho * rho via the Hadamard square (Theorem f*gP(2))
    equals two successive group-law quadratures."""
    N, M = 16, 8
    s2, nu = 0.01, math.pi / 4
    prob = synth.make_problem(1, 4, N, M, n_bumps=2)
    F = synth.sample_bumps(N, M, prob.bumps)
    P = G.se2_gaussian_kernel(N, M, s2, nu, images=1)
    two = direct.group_quadrature(direct.group_quadrature(F, 2, [s2, nu], images=1), 2, [s2, nu], images=1)
    got = O.convolve_power(F, P, 2)
    assert np.max(np.abs(got - two)) / np.max(np.abs(two)) < 1e-12
    # mass: the mean of f * rho is mean(f) times mean(rho) (DC coefficients)
    assert got.mean() == pytest.approx(F.mean() * P.mean() ** 2, rel=1e-12)
