"""Pins of the odd-size / upsampled oracle (Eqs. Qf, W, MatSKfgonG,
Proposition LtoN1D, Lemma TrigL) against brute force, the N = L oracle and
closed forms."""
import math

import numpy as np
import pytest

from oracle import se2_gaussians as G
from oracle import se2_oracle as O
from oracle import se2_upsample as U


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("L,N,q", [
    ((5, 7, 3), (5, 7, 3), 1),
    ((5, 7, 3), (8, 9, 6), 1),
    ((7, 5, 9), (11, 12, 10), 2),
    ((3, 3, 5), (4, 6, 7), 3),
    ((9, 7, 5), (9, 16, 5), 0),
])
def test_series_equals_matrix_form(L, N, q):
    """The definition (sum over |k| <= K of FFC products times phi_k at the
    N-grid) equals the zero-padded matrix form Eq. MatSKfgonG."""
    F = _rand(L, 1)
    Ps = [_rand(L, 2 + i) for i in range(q)]
    a = U.series(F, Ps, N)
    b = U.matrix(F, Ps, N)
    assert _rel(a, b) < 1e-12


@pytest.mark.parametrize("L,q", [((5, 7, 3), 1), ((9, 5, 7), 2), ((3, 5, 5), 3)])
def test_n_equals_l_reduces_to_the_closed_form(L, q):
    """At N = L the series is the N = L oracle (W^q iDFT form, Eq. MatSqKfgG)."""
    F = _rand(L, 3)
    Ps = [_rand(L, 4 + i) for i in range(q)]
    a = U.series(F, Ps, L).real
    b = O.convolve_chain(F, Ps)
    assert _rel(a, b) < 1e-12


@pytest.mark.parametrize("r", [2, 3])
def test_restriction_to_coarse_grid(r):
    """For N = r L the N-grid contains Omega_L (x'_{r i} = x_i), where the
    upsampled series equals the N = L output."""
    L = (5, 7, 9)
    N = tuple(r * v for v in L)
    F = _rand(L, 5)
    P = _rand(L, 6)
    fine = U.series(F, [P], N)
    coarse = U.series(F, [P], L)
    assert _rel(fine[::r, ::r, ::r], coarse) < 1e-12


@pytest.mark.parametrize("L,N", [(5, 5), (7, 12), (9, 10), (3, 8)])
def test_proposition_ltoN_brute_force(L, N):
    """sum_{k=-K..K} c_k x(tau_L(k)) e^{2 pi i k l / N} = N iDFT(z)(l)
    (Proposition LtoN1D), and the (-1)^k case (Corollary LtoN1D-1)."""
    K = (L - 1) // 2
    rng = np.random.default_rng(L * 100 + N)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    c = rng.standard_normal(2 * K + 1) + 1j * rng.standard_normal(2 * K + 1)
    ks = np.arange(-K, K + 1)
    tau = np.where(ks >= 0, ks, L + ks)
    for cc in (c, (-1.0) ** ks, np.ones(2 * K + 1)):
        lhs = np.array([np.sum(cc * x[tau] * np.exp(2j * np.pi * ks * l / N)) for l in range(N)])
        rhs = N * np.fft.ifft(U.zero_pad(x, N, cc))
        assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))


def test_trig_polynomials_are_exact_off_grid():
    """For f = cos(2 pi a.x + a3 theta) and rho = cos(2 pi b.x + b3 theta) with
    |a|, |b| <= K the FFCs are exact (Lemma TrigL), so the series at any
    point is the product series in closed form; checked on an N-grid that
    is not a refinement of Omega_L."""
    L = (9, 7, 11)          # (L_r, L_y, L_x)
    N = (14, 10, 13)
    Lr, Ly, Lx = L
    x = -0.5 + np.arange(Lx) / Lx
    y = -0.5 + np.arange(Ly) / Ly
    t = 2 * np.pi * np.arange(Lr) / Lr
    T, Y, X = np.meshgrid(t, y, x, indexing="ij")
    a = (2, -3, 4)   # (k1, k2, k3)
    F = np.cos(2 * np.pi * (a[0] * X + a[1] * Y) + a[2] * T)
    P = np.cos(2 * np.pi * (a[0] * X + a[1] * Y) + a[2] * T) + 0.5
    got = U.series(F, [P], N)
    xs = -0.5 + np.arange(N[2]) / N[2]
    ys = -0.5 + np.arange(N[1]) / N[1]
    ts = 2 * np.pi * np.arange(N[0]) / N[0]
    T2, Y2, X2 = np.meshgrid(ts, ys, xs, indexing="ij")
    # f^ = (delta_a + delta_-a)/2, rho^ = (delta_a + delta_-a)/2 + 0.5 delta_0
    # product = (delta_a + delta_-a)/4  ->  S = cos(...)/2
    want = 0.5 * np.cos(2 * np.pi * (a[0] * X2 + a[1] * Y2) + a[2] * T2)
    assert np.max(np.abs(got - want)) < 1e-13
    assert _rel(U.matrix(F, [P], N).real, want) < 1e-12


def test_paper_e4_shape_smoke():
    """The paper's single-convolution experiment shape: K = (15, 16, 30),
    L = (31, 33, 61), output grid 36 x 38 x 76, with f_H^{nu,s} and the
    radial deformed Gaussian kernel f_U^{nu,s}; both routes agree and the
    output is real up to rounding."""
    Lx, Ly, Lr = 31, 33, 61
    Nx, Ny, Nr = 36, 38, 76

    def sample(Hm, nu, s):
        x = -0.5 + np.arange(Lx) / Lx
        y = -0.5 + np.arange(Ly) / Ly
        t = 2 * np.pi * np.arange(Lr) / Lr
        Y, X = np.meshgrid(y, x, indexing="ij")
        sp = np.exp(-(Hm[0][0] * X * X + Hm[1][1] * Y * Y))
        return np.exp(-((t - nu) ** 2) / s)[:, None, None] * sp[None]

    F = sample([[1 / 0.03, 0], [0, 1 / 0.01]], math.pi / 2, 0.01)
    P = sample([[1 / 0.02, 0], [0, 1 / 0.02]], math.pi / 2, 0.01)
    a = U.series(F, [P], (Nr, Ny, Nx))
    b = U.matrix(F, [P], (Nr, Ny, Nx))
    assert _rel(a, b) < 1e-12
    assert np.max(np.abs(a.imag)) < 1e-12 * np.max(np.abs(a.real))
