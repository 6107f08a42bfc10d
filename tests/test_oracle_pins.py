"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names the passage of arXiv 2504.05149 (or the mathematical fact) it
checks, and is chosen so that a plausible slip in the oracle -- a dropped W,
a wrong sign or index, a transposed operand, a wrong scale -- fails it.
"""
import math

import numpy as np
import pytest

import synth
from oracle import closed_forms as cf
from oracle import direct
from oracle import se2_oracle as O

RNG = np.random.default_rng(12345)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


# --- DFT conventions (Section 2.3, Eqs. 3DFT / 3iDFT) -----------------------

def test_dft_matrix_and_fft_routes_match_plain_loop():
    X = RNG.standard_normal((3, 2, 5)) + 1j * RNG.standard_normal((3, 2, 5))
    M, Ny, Nx = X.shape
    ref = np.zeros_like(X)
    for l in range(M):
        for m in range(Ny):
            for n in range(Nx):
                s = 0
                for i in range(M):
                    for j in range(Ny):
                        for k in range(Nx):
                            s += X[i, j, k] * np.exp(-2j * np.pi * (i * l / M + j * m / Ny + k * n / Nx))
                ref[l, m, n] = s
    assert _rel(O.dft3(X, "matrix"), ref) < 1e-13
    assert _rel(O.dft3(X, "fft"), ref) < 1e-13
    assert _rel(O.idft3(ref, "matrix"), X) < 1e-13
    assert _rel(O.idft3(ref, "fft"), X) < 1e-13


@pytest.mark.parametrize("shape", [(8, 16, 16), (5, 7, 9), (16, 32, 32)])
def test_dft_routes_agree(shape):
    X = RNG.standard_normal(shape)
    assert _rel(O.dft3(X, "matrix"), O.dft3(X, "fft")) < 1e-12


# --- Lemma TrigL: FFC exact for trigonometric polynomials -------------------

@pytest.mark.parametrize("K,even", [(3, False), (5, False), (4, True)])
def test_trig_lemma_ffc_exact(K, even):
    L = 2 * K + 2 if even else 2 * K + 1
    deg = K if not even else K  # even grid: |k| <= L/2 - 1
    ks = np.arange(-deg, deg + 1)
    a = RNG.standard_normal((ks.size,) * 3) + 1j * RNG.standard_normal((ks.size,) * 3)
    x = -0.5 + np.arange(L) / L
    th = 2 * np.pi * np.arange(L) / L
    ex = np.exp(2j * np.pi * np.outer(x, ks))          # [i, k1]
    et = np.exp(1j * np.outer(th, ks))                 # [l, k3]
    # P(x_i, y_j, theta_l) = sum a[k3, k2, k1] phi_k; array layout [l][j][i]
    P = np.einsum("cba,lc,jb,ia->lji", a, et, ex, ex)
    F = O.ffc(P)
    kb = O.signed_freq(L)
    for c, k3 in enumerate(ks):
        for b, k2 in enumerate(ks):
            for aa, k1 in enumerate(ks):
                got = F[np.where(kb == k3)[0][0], np.where(kb == k2)[0][0], np.where(kb == k1)[0][0]]
                assert abs(got - a[c, b, aa]) < 1e-12


# --- Aliased closed forms of the sampled inputs (Eq. FkLv + aliasing) --------

@pytest.mark.parametrize("N,M", [(16, 8), (32, 16), (64, 32)])
def test_kernel_coeffs_match_aliased_closed_form(N, M):
    kp = synth.KernelParams(0.05, 0.3, 0.7)
    P = synth.sample_kernel(N, M, kp)
    got = O.coeffs_full(P)
    want = cf.kernel_coeffs_dft(N, M, kp)
    assert _rel(got, want) < 1e-13
    # the half spectrum is the first N/2+1 x bins and rebuilds the rest
    assert _rel(O.half_to_full(O.coeffs_half(P), N), got) < 1e-14
    # separable shortcut of the oracle agrees
    gx, gy, gt = synth.kernel_factors(N, M, kp)
    assert _rel(O.coeffs_separable(gx, gy, gt), got) < 1e-13


@pytest.mark.parametrize("N,M", [(32, 16), (64, 16)])
def test_bump_ffc_matches_aliased_closed_form(N, M):
    prob = synth.make_problem(1, 0, N, M, n_bumps=3)
    F = synth.sample_bumps(N, M, prob.bumps)
    assert _rel(O.ffc(F), cf.bumps_ffc(N, M, prob.bumps)) < 1e-12


# --- The scheme itself -------------------------------------------------------

@pytest.mark.parametrize("N,M", [(16, 8), (32, 16)])
def test_scheme_equals_brute_force_direct_sum(N, M):
    """R1: the FFT closed form at N = L equals the discrete periodic
    convolution (rectangle rule of Eq. f*gRadialMain) on Omega_L."""
    prob = synth.make_problem(1, 0, N, M, n_bumps=3, kernel_fixed=synth.KernelParams(0.05, 0.3, 0.9))
    F = synth.sample_bumps(N, M, prob.bumps)
    P = synth.sample_kernel(N, M, prob.kernels[0])
    want = direct.direct_conv(F, P)
    assert _rel(O.convolve(F, P, "fft"), want) < 1e-13
    assert _rel(O.convolve(F, P, "matrix"), want) < 1e-13
    z = O.convolve_complex(F, P)
    assert np.max(np.abs(z.imag)) <= 1e-12 * np.max(np.abs(z.real))


def test_scheme_on_random_arrays_matches_direct_sum():
    """Same identity on unstructured inputs: catches a transposed axis."""
    F = RNG.standard_normal((4, 8, 8))
    P = RNG.standard_normal((4, 8, 8))
    assert _rel(O.convolve(F, P), direct.direct_conv(F, P)) < 1e-13


def test_group_law_quadrature_radial_equals_scheme():
    """Theorem f*gP(1): for a kernel radial in translations the SE(2)
    convolution with the rotated argument S^{-1}(x - y) reduces to the abelian
    convolution.  The kernel's angular centre nu != 0 makes theta - alpha vs
    alpha - theta distinguishable."""
    N, M = 16, 8
    kp = synth.KernelParams(0.06, 0.35, 0.8)
    prob = synth.make_problem(1, 1, N, M, n_bumps=3)
    F = synth.sample_bumps(N, M, prob.bumps)
    P = synth.sample_kernel(N, M, kp)
    quad = direct.group_quadrature(F, 0, [kp.sigma, kp.sigma_theta, kp.nu], images=1)
    assert _rel(O.convolve(F, P), quad) < 1e-12


def test_group_law_quadrature_nonradial_differs():
    """Negative check: an anisotropic (non-radial) kernel does not reduce."""
    N, M = 16, 8
    s1, s2, st, nu = 0.04, 0.12, 0.35, 0.8
    prob = synth.make_problem(1, 1, N, M, n_bumps=3)
    F = synth.sample_bumps(N, M, prob.bumps)
    x = -0.5 + np.arange(N) / N
    th = 2 * np.pi * np.arange(M) / M
    gx = sum(np.exp(-((x + n) ** 2) / (2 * s1 * s1)) for n in range(-2, 3)) / (math.sqrt(2 * math.pi) * s1)
    gy = sum(np.exp(-((x + n) ** 2) / (2 * s2 * s2)) for n in range(-2, 3)) / (math.sqrt(2 * math.pi) * s2)
    d = np.mod(th - nu + np.pi, 2 * np.pi) - np.pi
    gt = 2 * np.pi * sum(np.exp(-((d + 2 * np.pi * m) ** 2) / (2 * st * st)) for m in range(-4, 5)) / (st * math.sqrt(2 * math.pi))
    P = gt[:, None, None] * gy[None, :, None] * gx[None, None, :]
    quad = direct.group_quadrature(F, 1, [s1, s2, st, nu], images=1)
    assert _rel(O.convolve(F, P), quad) > 1e-2


@pytest.mark.parametrize("nk", [1, 3])
def test_scheme_matches_separable_closed_form(nk):
    N, M = 32, 16
    prob = synth.make_problem(1, 2, N, M, n_bumps=3, n_kernels=nk)
    prob.kernels = [synth.KernelParams(0.04 + 0.01 * i, 0.3 + 0.05 * i, 0.3 * i) for i in range(nk)]
    F = synth.sample_bumps(N, M, prob.bumps)
    Ps = [synth.sample_kernel(N, M, k) for k in prob.kernels]
    got = O.convolve_chain(F, Ps)
    want = cf.scheme_output(N, M, prob.bumps, prob.kernels)
    assert _rel(got, want.real) < 1e-12
    assert np.max(np.abs(want.imag)) < 1e-13 * np.max(np.abs(want.real))


def test_continuous_closed_form_variance_sum_chain():
    """The 8-fold chain against the continuous convolution (variances add,
    angular coefficients multiply).  They differ only by aliasing cross terms,
    tiny at this resolution for these widths (sigma >= 0.02, sigma_theta >= 0.3)."""
    N, M = 128, 64
    kernels = [synth.KernelParams(0.02 + 0.002 * i, 0.3 + 0.02 * i, 0.0) for i in range(8)]
    prob = synth.make_problem(2, 0, N, M, n_bumps=16)
    F = synth.sample_bumps(N, M, prob.bumps)
    gx, gy, gt = zip(*[synth.kernel_factors(N, M, k) for k in kernels])
    coeffs = [O.coeffs_separable(a, b, c) for a, b, c in zip(gx, gy, gt)]
    got = O.convolve_chain(F, None, coeffs=coeffs)
    want = cf.continuous_output(N, M, prob.bumps, kernels)
    assert _rel(got, want) < 1e-9


def test_continuous_closed_form_single_c1_within_aliasing():
    """At the 32x32x16 config the discrete scheme sits within ~1e-3 of the
    continuous convolution (aliasing of the von Mises / wrapped-normal
    harmonics at the angular Nyquist), as estimated from the closed forms."""
    N, M = 32, 16
    kp = synth.KernelParams(0.05, 0.3, 0.0)
    prob = synth.make_problem(1, 0, N, M, n_bumps=3)
    F = synth.sample_bumps(N, M, prob.bumps)
    P = synth.sample_kernel(N, M, kp)
    err = _rel(O.convolve(F, P), cf.continuous_output(N, M, prob.bumps, [kp]))
    assert 1e-8 < err < 5e-3


def test_mass_conservation():
    """DC bin: mean(out) = mean(F) * prod_i C_i[0]."""
    N, M = 32, 16
    F = RNG.random((M, N, N))
    Ps = [RNG.random((M, N, N)) for _ in range(3)]
    out = O.convolve_chain(F, Ps)
    want = F.mean() * np.prod([P.mean() for P in Ps])
    assert abs(out.mean() - want) < 1e-14 * abs(want)


def test_power_chain_fast_loop_and_naive_recursion_agree():
    """Algorithm 4 (power, W only for odd q) = chain of q equal kernels =
    Algorithm 6's V_q = q successive single convolutions (Algorithm 5,
    associativity Eq. Vq1q)."""
    N, M = 16, 8
    prob = synth.make_problem(1, 3, N, M, n_bumps=3)
    F = synth.sample_bumps(N, M, prob.bumps)
    P = synth.sample_kernel(N, M, synth.KernelParams(0.05, 0.4, 0.5))
    fast = O.convolve_all(F, [P] * 4)
    V = F
    for q in range(1, 5):
        V = O.convolve(V, P)
        a = O.convolve_power(F, P, q)
        b = O.convolve_chain(F, [P] * q)
        assert _rel(a, V) < 1e-12 and _rel(b, V) < 1e-12 and _rel(fast[q - 1], V) < 1e-12
    # the direct sum applied twice
    assert _rel(direct.direct_conv(direct.direct_conv(F, P), P), O.convolve_power(F, P, 2)) < 1e-12


# --- Adjoint and kernel-parameter gradients ----------------------------------

def test_adjoint_dot_product():
    N, M = 16, 8
    F = RNG.standard_normal((M, N, N))
    G = RNG.standard_normal((M, N, N))
    Ps = [RNG.random((M, N, N)) for _ in range(3)]
    for q in (1, 2, 3):
        lhs = np.vdot(O.convolve_chain(F, Ps[:q]), G)
        rhs = np.vdot(F, O.adjoint(G, Ps[:q]))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    P = Ps[0]
    lhs = np.vdot(O.convolve(F, P), G)
    rhs = np.vdot(P, O.grad_kernel_samples(F, G))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_adjoint_equals_direct_correlation():
    """grad_f of <G, conv(F, P)> is the correlation sum_n G[n] P[n - m + c]."""
    N, M = 8, 4
    G = RNG.standard_normal((M, N, N))
    P = RNG.standard_normal((M, N, N))
    L = N * N * M
    want = np.zeros((M, N, N))
    for l in range(M):
        for j in range(N):
            for i in range(N):
                Pi = P[(np.arange(M)[:, None, None] - l) % M,
                       (np.arange(N)[None, :, None] - j + N // 2) % N,
                       (np.arange(N)[None, None, :] - i + N // 2) % N]
                want[l, j, i] = np.sum(G * Pi) / L
    assert _rel(O.adjoint(G, [P]), want) < 1e-13


def test_kernel_parameter_gradient_finite_differences():
    """dL/dsigma and dL/dsigma_theta of L = 1/2 ||f * rho(sigma) - target||^2
    from the adjoint (grad_kernel_samples . dP/dparam) against central
    differences with h = 1e-4 in FP64 (samples from synth, independent of the
    oracle's derivative formulas)."""
    N, M = 32, 16
    prob = synth.make_problem(5, 0, N, M, n_bumps=4)
    tprob = synth.make_problem(5, 1, N, M, n_bumps=4)
    F = synth.sample_bumps(N, M, prob.bumps)
    target = O.convolve(synth.sample_bumps(N, M, tprob.bumps), synth.sample_kernel(N, M, synth.KernelParams(0.03, 0.3)))
    s, st = 0.045, 0.35

    def loss(s_, st_):
        r = O.convolve(F, synth.sample_kernel(N, M, synth.KernelParams(s_, st_))) - target
        return 0.5 * np.sum(r * r)

    P, dPs, dPt = O.kernel_samples_and_derivs(N, M, s, st)
    assert _rel(P, synth.sample_kernel(N, M, synth.KernelParams(s, st))) < 1e-14
    G = O.convolve(F, P) - target
    gP = O.grad_kernel_samples(F, G)
    gs, gt = np.sum(gP * dPs), np.sum(gP * dPt)
    h = 1e-4
    fs = (loss(s + h, st) - loss(s - h, st)) / (2 * h)
    ft = (loss(s, st + h) - loss(s, st - h)) / (2 * h)
    assert abs(gs - fs) < 1e-6 * abs(fs)
    assert abs(gt - ft) < 1e-6 * abs(ft)


# --- Theorem UkL / fkLmain bound on the paper's E2 function ------------------

def test_ffc_error_bound_deformed_gaussian_E2():
    """|f^[k] - f^[k; 2K+1]| <= 36 ||grad f|| / K (the constant of Theorem UkL
    with d = 3 and box side 2 pi) for f = exp(-x^T H x) exp(-(t-nu)^2/s),
    H = diag(0.04, 0.1)^-1, s = 0.4, nu = pi, k = (1, -2, 3) (Section 4.2)."""
    from scipy import integrate
    hx, hy, s, nu = 1 / 0.04, 1 / 0.1, 0.4, math.pi
    k1, k2, k3 = 1, -2, 3

    def c1d(fun, a, b, w):
        re = integrate.quad(lambda t: fun(t) * math.cos(w * t), a, b, limit=200, epsabs=1e-14)[0]
        im = integrate.quad(lambda t: -fun(t) * math.sin(w * t), a, b, limit=200, epsabs=1e-14)[0]
        return re + 1j * im
    true = (c1d(lambda x: math.exp(-hx * x * x), -0.5, 0.5, 2 * math.pi * k1)
            * c1d(lambda y: math.exp(-hy * y * y), -0.5, 0.5, 2 * math.pi * k2)
            * c1d(lambda t: math.exp(-(t - nu) ** 2 / s), 0, 2 * math.pi, k3) / (2 * math.pi))
    # sup of the Euclidean gradient norm, on a fine grid
    g = np.linspace(-0.5, 0.5, 201)
    t = np.linspace(0, 2 * math.pi, 401)
    X, Y, T = np.meshgrid(g, g, t, indexing="ij")
    f = np.exp(-hx * X * X - hy * Y * Y - (T - nu) ** 2 / s)
    grad = f * np.sqrt((2 * hx * X) ** 2 + (2 * hy * Y) ** 2 + (2 * (T - nu) / s) ** 2)
    gmax = grad.max()
    errs = []
    for K in range(3, 13):
        L = 2 * K + 1
        x = -0.5 + np.arange(L) / L
        th = 2 * math.pi * np.arange(L) / L
        F = np.exp(-(th[:, None, None] - nu) ** 2 / s) * np.exp(-hy * x[None, :, None] ** 2) * np.exp(-hx * x[None, None, :] ** 2)
        C = O.ffc(F)
        kb = O.signed_freq(L)
        got = C[np.where(kb == k3)[0][0], np.where(kb == k2)[0][0], np.where(kb == k1)[0][0]]
        err = abs(got - true)
        assert err <= 36 * gmax / K
        errs.append(err)
    # and the error actually decays with K
    assert errs[-1] < 0.1 * errs[0]


def test_origin_zero_is_the_plain_cyclic_convolution():
    """Grids sampled at x_i = i/N: the scheme without W equals the direct
    cyclic sum (1/|L|) sum_m F[m] P[n - m] (brute force, shift 0), on both
    DFT routes."""
    from oracle import direct
    N, M = 16, 8
    F = RNG.random((M, N, N))
    P = RNG.random((M, N, N))
    want = direct.direct_conv(F, P, origin_zero=True)
    for route in ("fft", "matrix"):
        got = O.convolve(F, P, route, origin_zero=True)
        assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))
    # and it is not the Omega_L result (W matters)
    assert np.max(np.abs(O.convolve(F, P) - want)) > 1e-3 * np.max(np.abs(want))


def test_origin_conventions_differ_by_a_half_period_shift():
    """The same periodic bumps and kernel sampled on Omega_L and at x_i = i/N:
    the Omega_L output (with W) is the origin-zero output (without W) shifted
    by N/2 in x and y, and a 3-kernel chain equals three successive singles."""
    N, M = 32, 16
    prob = synth.make_problem(1, 7, N, M, n_bumps=3, n_kernels=3)
    F1 = synth.sample_bumps(N, M, prob.bumps)
    F0 = synth.sample_bumps(N, M, prob.bumps, origin_zero=True)
    P1 = [synth.sample_kernel(N, M, k) for k in prob.kernels]
    P0 = [synth.sample_kernel(N, M, k, origin_zero=True) for k in prob.kernels]
    out1 = O.convolve(F1, P1[0])
    out0 = O.convolve(F0, P0[0], origin_zero=True)
    assert np.max(np.abs(out1 - np.roll(out0, (N // 2, N // 2), axis=(1, 2)))) < 1e-12 * np.max(np.abs(out1))
    chain = O.convolve_chain(F0, P0, origin_zero=True)
    seq = F0
    for P in P0:
        seq = O.convolve(seq, P, origin_zero=True)
    assert np.max(np.abs(chain - seq)) < 1e-12 * np.max(np.abs(seq))


def _rot90(F):
    """Left translation by the rotation R_{pi/2} on Omega_L: f'(x, y, theta) =
    f(y, -x, theta - pi/2).  The grid x_i = -1/2 + i/N is closed under
    x -> -x (index i -> -i mod N), so this is an index map; theta shifts by M/4."""
    M, N = F.shape[0], F.shape[-1]
    Y, X = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    Fr = np.roll(F, M // 4, axis=0)
    return Fr[:, (-X) % N, Y]


@pytest.mark.parametrize("N,M", [(8, 4), (16, 8)])
def test_convolution_commutes_with_rotation_and_translation(N, M):
    """Theorem f*gP: for a kernel radial in translations the SE(2) convolution
    commutes with left translations of f.  On the grid: a 90-degree rotation
    (with theta shifted by M/4) and cyclic grid shifts commute with the
    scheme; an anisotropic kernel breaks the rotation identity but not the
    shifts (checked against the direct sum as well)."""
    rng = np.random.default_rng(N + M)
    F = rng.standard_normal((M, N, N))
    P = synth.sample_kernel(N, M, synth.KernelParams(0.11, 0.5, 0.7))
    out = O.convolve(F, P)
    assert np.max(np.abs(O.convolve(_rot90(F), P) - _rot90(out))) < 1e-12 * np.max(np.abs(out))
    sh = (1, 3, N - 2)
    assert np.max(np.abs(O.convolve(np.roll(F, sh, axis=(0, 1, 2)), P) - np.roll(out, sh, axis=(0, 1, 2)))) < 1e-12
    assert np.max(np.abs(direct.direct_conv(F, P) - out)) < 1e-12 * np.max(np.abs(out))
    # an anisotropic kernel: x and y widths differ
    Pa = P * np.exp(-4.0 * ((np.arange(N) - N / 2) / N) ** 2)[None, None, :]
    outa = O.convolve(F, Pa)
    assert np.max(np.abs(O.convolve(_rot90(F), Pa) - _rot90(outa))) > 1e-3 * np.max(np.abs(outa))
    assert np.max(np.abs(O.convolve(np.roll(F, sh, axis=(0, 1, 2)), Pa) - np.roll(outa, sh, axis=(0, 1, 2)))) < 1e-12


def test_convolution_is_linear_in_f():
    N, M = 16, 8
    rng = np.random.default_rng(5)
    F1, F2 = rng.standard_normal((2, M, N, N))
    P = synth.sample_kernel(N, M, synth.KernelParams(0.05, 0.3))
    lhs = O.convolve(2.5 * F1 - 0.75 * F2, P)
    rhs = 2.5 * O.convolve(F1, P) - 0.75 * O.convolve(F2, P)
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(rhs))
