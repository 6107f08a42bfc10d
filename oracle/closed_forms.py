"""Closed forms that pin the FP64 oracle (TEST INFRASTRUCTURE ONLY).

None of these uses a DFT of samples: they are written from the continuous
Fourier coefficients of the test functions, so they are independent of
oracle/se2_oracle.py.

* Continuous coefficients (Section 3.1, Eq. fk, with dOmega = dx dy dtheta/2pi):
    periodised Gaussian e^{-(x-c)^2/2s^2}:   sqrt(2pi) s e^{-2 pi^2 s^2 k^2} e^{-2 pi i k c}
    normalised spatial kernel factor:         e^{-2 pi^2 sigma^2 k^2}
    von Mises e^{kappa (cos(t-mu) - 1)}:      I_k(kappa) e^{-kappa} e^{-i k mu}
    2 pi x wrapped normal (sigma_t, nu):      e^{-sigma_t^2 k^2 / 2} e^{-i k nu}
* Aliasing: sampling on Omega_L (Eq. OmL) gives the finite Fourier coefficient
  (Eq. fkLvMain) as the sum of the continuous coefficients over the aliases
  k + m L, times (-1)^{m L} on the two spatial axes (from the -1/2 offset).
  For band-limited inputs this is Lemma TrigL.
* The finite Fourier series at the grid points (Eq. SKvf / SKfg evaluated on
  Omega_L) is then a separable sum, which gives the output of the scheme in
  closed form for sums of separable bumps and separable radial kernels.
* The continuous convolution (Eq. f*gRadialMain) of these families has a
  closed form too: Gaussian variances add; angular coefficients multiply.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np
from scipy import special

from synth import Bump, KernelParams

_ALIASES = 6


def _bins_signed(n: int) -> np.ndarray:
    i = np.arange(n)
    return np.where(i <= (n - 1) // 2, i, i - n)


def gauss_coeff(k, c: float, s: float):
    k = np.asarray(k, dtype=np.float64)
    return math.sqrt(2 * math.pi) * s * np.exp(-2 * math.pi ** 2 * s * s * k * k) * np.exp(-2j * math.pi * k * c)


def kernel_space_coeff(k, sigma: float):
    k = np.asarray(k, dtype=np.float64)
    return np.exp(-2 * math.pi ** 2 * sigma * sigma * k * k) + 0j


def vonmises_coeff(k, kappa: float, mu: float):
    k = np.asarray(k)
    return special.ive(np.abs(k), kappa) * np.exp(-1j * k * mu)


def wn_coeff(k, sigma_t: float, nu: float):
    k = np.asarray(k, dtype=np.float64)
    return np.exp(-0.5 * sigma_t * sigma_t * k * k) * np.exp(-1j * k * nu)


def aliased(coeff_fn, n: int, spatial: bool) -> np.ndarray:
    """FFC at each DFT bin: sum_m coeff(k + m n) (-1)^{m n} (spatial axes) --
    the aliasing sum of Section 3.2's rectangle rule."""
    k = _bins_signed(n)
    acc = np.zeros(n, dtype=np.complex128)
    for m in range(-_ALIASES, _ALIASES + 1):
        sign = (-1.0) ** (m * n) if spatial else 1.0
        acc += sign * coeff_fn(k + m * n)
    return acc


def kernel_ffc_1d(N: int, M: int, kp: KernelParams):
    fx = aliased(lambda k: kernel_space_coeff(k, kp.sigma), N, True)
    ft = aliased(lambda k: wn_coeff(k, kp.sigma_theta, kp.nu), M, False)
    return fx, fx.copy(), ft


def bump_ffc_1d(N: int, M: int, b: Bump):
    fx = aliased(lambda k: gauss_coeff(k, b.cx, b.sx), N, True)
    fy = aliased(lambda k: gauss_coeff(k, b.cy, b.sy), N, True)
    ft = aliased(lambda k: vonmises_coeff(k, b.kappa, b.mu), M, False)
    return fx, fy, ft


def kernel_coeffs_dft(N: int, M: int, kp: KernelParams) -> np.ndarray:
    """Expected DFT(P)/|L| of the sampled kernel: W times its FFC (Eq. FkLv)."""
    fx, fy, ft = kernel_ffc_1d(N, M, kp)
    k = _bins_signed(N)
    wx = (-1.0) ** k
    return ft[:, None, None] * (wx * fy)[None, :, None] * (wx * fx)[None, None, :]


def bumps_ffc(N: int, M: int, bumps: Sequence[Bump]) -> np.ndarray:
    out = np.zeros((M, N, N), dtype=np.complex128)
    for b in bumps:
        fx, fy, ft = bump_ffc_1d(N, M, b)
        out += b.amp * ft[:, None, None] * fy[None, :, None] * fx[None, None, :]
    return out


def _series_at_grid(c: np.ndarray, pts: np.ndarray, period: float) -> np.ndarray:
    """sum over bins of c[k] exp(2 pi i k x / period) at the points x."""
    k = _bins_signed(c.size)
    return np.exp(2j * math.pi * np.outer(pts, k) / period) @ c


def scheme_output(N: int, M: int, bumps: Sequence[Bump], kernels: Sequence[KernelParams]) -> np.ndarray:
    """Closed form of the scheme's output on Omega_L (finite Fourier series of
    the product of FFCs, Eq. SKfg / SqKfg on the grid) for separable bumps and
    a chain of separable radial kernels.  Returns complex [M][N][N]."""
    x = -0.5 + np.arange(N) / N
    th = 2 * math.pi * np.arange(M) / M
    kx = np.ones(N, dtype=np.complex128)
    kt = np.ones(M, dtype=np.complex128)
    for kp in kernels:
        a, _, c = kernel_ffc_1d(N, M, kp)
        kx = kx * a
        kt = kt * c
    out = np.zeros((M, N, N), dtype=np.complex128)
    for b in bumps:
        fx, fy, ft = bump_ffc_1d(N, M, b)
        vx = _series_at_grid(fx * kx, x, 1.0)
        vy = _series_at_grid(fy * kx, x, 1.0)
        vt = _series_at_grid(ft * kt, th, 2 * math.pi)
        out += b.amp * vt[:, None, None] * vy[None, :, None] * vx[None, None, :]
    return out


def continuous_output(N: int, M: int, bumps: Sequence[Bump], kernels: Sequence[KernelParams],
                      kmax: int = 400) -> np.ndarray:
    """The continuous convolution f * rho_1 * ... * rho_q on the coset space,
    sampled on Omega_L: Gaussian variances add in x and y, angular Fourier
    coefficients multiply (Theorem f*gP(2) applied factor by factor)."""
    x = -0.5 + np.arange(N) / N
    th = 2 * math.pi * np.arange(M) / M
    S = sum(kp.sigma ** 2 for kp in kernels)
    k = np.arange(-kmax, kmax + 1)
    kt = np.ones(k.size, dtype=np.complex128)
    for kp in kernels:
        kt = kt * wn_coeff(k, kp.sigma_theta, kp.nu)
    out = np.zeros((M, N, N))
    for b in bumps:
        def gx(c, s):
            s2 = s * s + S
            d = np.mod(x - c + 0.5, 1.0) - 0.5
            acc = np.zeros(N)
            for n in range(-3, 4):
                acc += np.exp(-((d + n) ** 2) / (2 * s2))
            return acc * s / math.sqrt(s2)
        vt = (np.exp(1j * np.outer(th, k)) @ (vonmises_coeff(k, b.kappa, b.mu) * kt)).real
        out += b.amp * vt[:, None, None] * gx(b.cy, b.sy)[None, :, None] * gx(b.cx, b.sx)[None, None, :]
    return out


def continuous_output_points(bumps: Sequence[Bump], kernels: Sequence[KernelParams],
                             x: np.ndarray, y: np.ndarray, th: np.ndarray, kmax: int = 400) -> np.ndarray:
    """continuous_output at arbitrary points (x, y, theta) (1-D arrays)."""
    S = sum(kp.sigma ** 2 for kp in kernels)
    k = np.arange(-kmax, kmax + 1)
    kt = np.ones(k.size, dtype=np.complex128)
    for kp in kernels:
        kt = kt * wn_coeff(k, kp.sigma_theta, kp.nu)
    out = np.zeros(x.size)
    for b in bumps:
        def g(p, c, s):
            s2 = s * s + S
            d = np.mod(p - c + 0.5, 1.0) - 0.5
            acc = np.zeros(p.size)
            for n in range(-3, 4):
                acc += np.exp(-((d + n) ** 2) / (2 * s2))
            return acc * s / math.sqrt(s2)
        vt = (np.exp(1j * np.outer(th, k)) @ (vonmises_coeff(k, b.kappa, b.mu) * kt)).real
        out += b.amp * vt * g(y, b.cy, b.sy) * g(x, b.cx, b.sx)
    return out


def mass(F: np.ndarray) -> float:
    """Integral under the Haar measure on the coset space, rectangle rule:
    the mean of the samples (Eq. dg with Lemma intO)."""
    return float(np.mean(F, axis=(-3, -2, -1)).sum()) if F.ndim == 3 else np.mean(F, axis=(-3, -2, -1))
