"""Seeded synthetic inputs for the SE(2) convolution path.

This module is shared by the CUDA path's tests/bench and by the FP64 oracle's
tests.  It only *generates data*: it draws seeded parameters and samples the
test functions on the fundamental grid.  It contains none of the method's
arithmetic (no DFT, no coefficient product, no inverse transform).

Input recipe (the paper uses analytic inputs, not a dataset):

* Grid: the fundamental sampling grid Omega_L of Section 3.2 (Eq. OmL) with
  even N: x_i = -1/2 + i/N, y_j = -1/2 + j/N, theta_l = 2*pi*l/M (0-based).
  Arrays are laid out [theta_l][y_j][x_i], x contiguous.
* f1 ("bumps"): a sum of axis-aligned anisotropic Gaussians in (x, y), the
  diagonal-H deformed Gaussians of Section 4.2 (Eq. fHsnu), periodised over
  the lattice Z^2 (Eq. TH), times a von Mises angular profile
  exp(kappa*(cos(theta-mu)-1)) that is periodic in theta.  Centres ~ U[0,1)^2,
  sigma_x, sigma_y ~ U[0.03, 0.1], kappa ~ U[1, 8], mu ~ U[0, 2pi),
  amplitude 1 or log-uniform in [1e-6, 1].
* f2 (kernel, radial in translations, footnote of Section 5.1): a radial
  Gaussian of width sigma in x, normalised over R^2, periodised, times 2*pi
  times a wrapped normal of width sigma_theta centred at nu.  Its integral
  under the Haar measure dg = dx dy dtheta / (2 pi) (Eq. dg) is 1.

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), seeded per
problem as 1000 * config + problem index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

__all__ = [
    "SplitMix64", "Bump", "KernelParams", "Problem",
    "grid_axes", "draw_bumps", "draw_kernel", "sample_bumps", "sample_kernel",
    "make_problem", "config_seed",
]

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator: state += golden gamma, then a 3-step mix."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        # 53 random mantissa bits -> [0, 1)
        u = (self.next_u64() >> 11) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1))


def config_seed(config: int, problem: int) -> int:
    return 1000 * config + problem


@dataclass
class Bump:
    amp: float
    cx: float
    cy: float
    sx: float
    sy: float
    kappa: float
    mu: float


@dataclass
class KernelParams:
    sigma: float          # spatial width (radial Gaussian)
    sigma_theta: float    # angular width (wrapped normal)
    nu: float = 0.0       # angular centre


@dataclass
class Problem:
    N: int
    M: int
    bumps: List[Bump]
    kernels: List[KernelParams] = field(default_factory=list)


def grid_axes(N: int, M: int, origin_zero: bool = False):
    """The three axes of Omega_L for even N (0-based indices); with
    origin_zero the spatial axes are x_i = i/N instead of -1/2 + i/N."""
    x = (0.0 if origin_zero else -0.5) + np.arange(N, dtype=np.float64) / N
    th = 2.0 * math.pi * np.arange(M, dtype=np.float64) / M
    return x, x.copy(), th


def draw_bumps(rng: SplitMix64, n: int, log_amp: bool = False) -> List[Bump]:
    out = []
    for _ in range(n):
        cx = rng.uniform()
        cy = rng.uniform()
        sx = rng.uniform(0.03, 0.1)
        sy = rng.uniform(0.03, 0.1)
        kappa = rng.uniform(1.0, 8.0)
        mu = rng.uniform(0.0, 2.0 * math.pi)
        amp = 10.0 ** rng.uniform(-6.0, 0.0) if log_amp else 1.0
        out.append(Bump(amp, cx, cy, sx, sy, kappa, mu))
    return out


def draw_kernel(rng: SplitMix64, sig_lo=0.01, sig_hi=0.04, st_lo=0.1, st_hi=0.5) -> KernelParams:
    return KernelParams(rng.uniform(sig_lo, sig_hi), rng.uniform(st_lo, st_hi), 0.0)


def _periodic_gauss_1d(x: np.ndarray, c: float, s: float, images: int = 2) -> np.ndarray:
    """sum_n exp(-(d+n)^2 / (2 s^2)), d = x - c reduced to [-1/2, 1/2)."""
    d = np.mod(x - c + 0.5, 1.0) - 0.5
    acc = np.zeros_like(d)
    for n in range(-images, images + 1):
        acc += np.exp(-((d + n) ** 2) / (2.0 * s * s))
    return acc


def _wrapped_normal(th: np.ndarray, nu: float, s: float, terms: int = 4) -> np.ndarray:
    d = np.mod(th - nu + math.pi, 2.0 * math.pi) - math.pi
    acc = np.zeros_like(d)
    for m in range(-terms, terms + 1):
        acc += np.exp(-((d + 2.0 * math.pi * m) ** 2) / (2.0 * s * s))
    return acc / (s * math.sqrt(2.0 * math.pi))


def sample_bumps(N: int, M: int, bumps: Sequence[Bump], origin_zero: bool = False) -> np.ndarray:
    """f1 sampled on Omega_L (or at x_i = i/N) as float64 [M][N][N] (theta, y, x)."""
    x, y, th = grid_axes(N, M, origin_zero)
    nb = len(bumps)
    X = np.empty((N, nb))
    Y = np.empty((N, nb))
    T = np.empty((M, nb))
    for b, p in enumerate(bumps):
        X[:, b] = _periodic_gauss_1d(x, p.cx, p.sx)
        Y[:, b] = _periodic_gauss_1d(y, p.cy, p.sy)
        T[:, b] = p.amp * np.exp(p.kappa * (np.cos(th - p.mu) - 1.0))
    # F[l, j, i] = sum_b T[l, b] Y[j, b] X[i, b]
    G = (T[:, None, :] * Y[None, :, :]).reshape(M * N, nb)
    return (G @ X.T).reshape(M, N, N)


def kernel_factors(N: int, M: int, k: KernelParams, origin_zero: bool = False):
    """The three 1-D factors of the sampled kernel: rho = kx (x) ky (x) kt."""
    x, y, th = grid_axes(N, M, origin_zero)
    s = k.sigma
    gx = _periodic_gauss_1d(x, 0.0, s) / (math.sqrt(2.0 * math.pi) * s)
    gt = 2.0 * math.pi * _wrapped_normal(th, k.nu, k.sigma_theta)
    return gx, gx.copy(), gt


def sample_kernel(N: int, M: int, k: KernelParams, origin_zero: bool = False) -> np.ndarray:
    """Radial kernel f2 sampled on Omega_L (or at x_i = i/N) as float64 [M][N][N]."""
    gx, gy, gt = kernel_factors(N, M, k, origin_zero)
    return gt[:, None, None] * gy[None, :, None] * gx[None, None, :]


def make_problem(config: int, index: int, N: int, M: int, n_bumps: int,
                 n_kernels: int = 1, log_amp: bool = False,
                 kernel_fixed: KernelParams | None = None) -> Problem:
    rng = SplitMix64(config_seed(config, index))
    bumps = draw_bumps(rng, n_bumps, log_amp)
    if kernel_fixed is not None:
        kernels = [kernel_fixed] * n_kernels
    else:
        kernels = [draw_kernel(rng) for _ in range(n_kernels)]
    return Problem(N, M, bumps, kernels)


def sample_bumps_torch(N: int, M: int, bumps: Sequence[Bump], device, dtype=None):
    """sample_bumps evaluated with torch on `device` (same formulas), for
    batches too large to generate on the host.  Returns [M][N][N]."""
    import torch
    dtype = dtype or torch.float64
    x = torch.arange(N, dtype=torch.float64, device=device) / N - 0.5
    th = 2.0 * math.pi * torch.arange(M, dtype=torch.float64, device=device) / M
    cx = torch.tensor([b.cx for b in bumps], dtype=torch.float64, device=device)[:, None]
    cy = torch.tensor([b.cy for b in bumps], dtype=torch.float64, device=device)[:, None]
    sx = torch.tensor([b.sx for b in bumps], dtype=torch.float64, device=device)[:, None]
    sy = torch.tensor([b.sy for b in bumps], dtype=torch.float64, device=device)[:, None]
    ka = torch.tensor([b.kappa for b in bumps], dtype=torch.float64, device=device)[:, None]
    mu = torch.tensor([b.mu for b in bumps], dtype=torch.float64, device=device)[:, None]
    amp = torch.tensor([b.amp for b in bumps], dtype=torch.float64, device=device)[:, None]

    def per(c, s):
        d = torch.remainder(x[None, :] - c + 0.5, 1.0) - 0.5
        acc = torch.zeros_like(d)
        for n in range(-2, 3):
            acc = acc + torch.exp(-((d + n) ** 2) / (2.0 * s * s))
        return acc

    X = per(cx, sx)
    Y = per(cy, sy)
    T = amp * torch.exp(ka * (torch.cos(th[None, :] - mu) - 1.0))
    return torch.einsum("bl,bj,bi->lji", T, Y, X).to(dtype)
