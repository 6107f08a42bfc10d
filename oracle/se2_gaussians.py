"""FP64 CPU oracle for the paper's analytic input families on SE(2).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import, call or link anything
under oracle/.  The product path never does, and this module never imports
the product.

What it computes, with the passage of arXiv 2504.05149 each function follows:

* se2_matrix / se2_log: elements of SE(2) as 3x3 matrices (Eq. gxyt) and the
  principal matrix logarithm log: SE(2) -> se(2) followed by the
  identification ^v: se(2) -> R^3 (Section 5, text of Eq. fbS).  The
  translation part is obtained by solving V(theta) v = x with V(theta) the
  integral of exp(t theta J) over t in [0, 1], written out from that
  definition (no half-angle simplification).
* se2_gaussian: the multidimensional Gaussian f_{beta,Sigma} on SE(2)
  (Eq. fbS), sampled on Omega_L.
* se2_gaussian_kernel: the kernel rho of Eq. gbS0, shifted by nu in the
  rotation direction as in the paper's chain experiments (Section 6.3):
  f_{beta,Sigma} with beta = (0, R_nu) and Sigma = sigma^2 I_3.
* deformed_gaussian: the 3D deformed Gaussian f_H^{nu,s} (Eq. fHsnu).

Readings where the paper is silent (each also listed with the design notes):
* The principal logarithm takes the angle in (-pi, pi]; at theta = pi the
  logarithm is not unique and +pi is taken (for Sigma isotropic in the
  translations both choices give the same value).
* Functions on SE(2) become functions on Z^2\\SE(2) by summing the left
  translates by lattice vectors n in Z^2 with |n_1|, |n_2| <= images
  (images = 0 samples the function on Omega_L as it is).
* In Eq. fHsnu theta is the grid angle in [0, 2 pi) itself, without
  wrapping, as printed.

Pins (tests/test_oracle_gaussians.py): scipy.linalg.logm / expm, the
theta = 0 reduction to a Euclidean Gaussian, radiality and the closed norm
|v| = |x| (phi/2)/sin(phi/2) for isotropic Sigma, left invariance under
beta, the exact identity between the spectral scheme and the group-law
quadrature (oracle/direct.c) for the radial kernel, and the Gaussian
integral pi / sqrt(det H) * sqrt(pi s) for Eq. fHsnu.
"""
from __future__ import annotations

import numpy as np

__all__ = ["se2_matrix", "se2_log", "se2_compose", "se2_inverse", "se2_gaussian_at", "se2_gaussian",
           "se2_gaussian_kernel", "deformed_gaussian"]


def se2_matrix(x1, x2, theta) -> np.ndarray:
    """The 3x3 matrix of (x, R_theta) (Eq. gxyt); broadcasts, shape (..., 3, 3)."""
    x1, x2, theta = np.broadcast_arrays(np.asarray(x1, float), np.asarray(x2, float), np.asarray(theta, float))
    g = np.zeros(x1.shape + (3, 3))
    c, s = np.cos(theta), np.sin(theta)
    g[..., 0, 0], g[..., 0, 1], g[..., 0, 2] = c, -s, x1
    g[..., 1, 0], g[..., 1, 1], g[..., 1, 2] = s, c, x2
    g[..., 2, 2] = 1.0
    return g


def se2_compose(a, b):
    """(a1, a2, alpha) o (b1, b2, beta): the matrix product of Eq. gxyt."""
    a1, a2, al = a
    b1, b2, be = b
    c, s = np.cos(al), np.sin(al)
    return (a1 + c * b1 - s * b2, a2 + s * b1 + c * b2, al + be)


def se2_inverse(a):
    a1, a2, al = a
    c, s = np.cos(al), np.sin(al)
    return (-(c * a1 + s * a2), -(-s * a1 + c * a2), -al)


def _principal(theta):
    """Angle reduced to (-pi, pi]."""
    t = np.mod(np.asarray(theta, float) + np.pi, 2.0 * np.pi) - np.pi
    return np.where(t == -np.pi, np.pi, t)


def se2_log(x1, x2, theta):
    """log(g)^v = (v1, v2, phi) for g = (x, R_theta).

    phi is the principal angle; log R_phi = phi J with J = [[0, -1], [1, 0]],
    and v solves V(phi) v = x where V(phi) = int_0^1 exp(t phi J) dt =
    (sin phi / phi) I + ((1 - cos phi) / phi) J (V(0) = I)."""
    x1, x2, theta = np.broadcast_arrays(np.asarray(x1, float), np.asarray(x2, float), np.asarray(theta, float))
    phi = _principal(theta)
    small = phi == 0.0
    ps = np.where(small, 1.0, phi)
    a = np.where(small, 1.0, np.sin(ps) / ps)
    # 1 - cos(phi) written as 2 sin^2(phi/2): no cancellation for small phi
    b = np.where(small, 0.0, 2.0 * np.sin(0.5 * ps) ** 2 / ps)
    V = np.empty(phi.shape + (2, 2))
    V[..., 0, 0], V[..., 0, 1] = a, -b
    V[..., 1, 0], V[..., 1, 1] = b, a
    rhs = np.stack([x1, x2], axis=-1)[..., None]
    v = np.linalg.solve(V, rhs)[..., 0]
    return v[..., 0], v[..., 1], phi


def se2_gaussian_at(x1, x2, theta, beta, Sigma) -> np.ndarray:
    """f_{beta,Sigma}(g) of Eq. fbS at g = (x, R_theta), one lattice image."""
    Sinv = np.linalg.inv(np.asarray(Sigma, float))
    y1, y2, yt = se2_compose(se2_inverse(tuple(float(b) for b in beta)), (x1, x2, theta))
    v1, v2, phi = se2_log(y1, y2, yt)
    w = np.stack([v1, v2, phi], axis=-1)
    q = np.einsum("...i,ij,...j->...", w, Sinv, w)
    return np.exp(-0.5 * q)


def _grid(N: int, M: int, origin_zero: bool):
    x = (0.0 if origin_zero else -0.5) + np.arange(N) / N
    th = 2.0 * np.pi * np.arange(M) / M
    return x, th


def se2_gaussian(N: int, M: int, beta, Sigma, images: int = 1, origin_zero: bool = False) -> np.ndarray:
    """[M][N][N] samples of f_{beta,Sigma} (Eq. fbS) on Omega_L, summed over the
    lattice translates |n_1|, |n_2| <= images."""
    x, th = _grid(N, M, origin_zero)
    T, Y, X = np.meshgrid(th, x, x, indexing="ij")
    out = np.zeros((M, N, N))
    for n2 in range(-images, images + 1):
        for n1 in range(-images, images + 1):
            out += se2_gaussian_at(X + n1, Y + n2, T, beta, Sigma)
    return out


def se2_gaussian_kernel(N: int, M: int, sigma2: float, nu: float = 0.0, images: int = 1,
                        origin_zero: bool = False) -> np.ndarray:
    """rho of Eq. gbS0 with variance sigma2, shifted by nu in the rotations."""
    return se2_gaussian(N, M, (0.0, 0.0, nu), sigma2 * np.eye(3), images, origin_zero)


def deformed_gaussian(N: int, M: int, H, nu: float, s: float, images: int = 1,
                      origin_zero: bool = False) -> np.ndarray:
    """[M][N][N] samples of f_H^{nu,s}(x, R_theta) = exp(-x^T H x) exp(-(theta - nu)^2 / s)
    (Eq. fHsnu), summed over the lattice translates |n_1|, |n_2| <= images."""
    H = np.asarray(H, float)
    x, th = _grid(N, M, origin_zero)
    Y, X = np.meshgrid(x, x, indexing="ij")
    sp = np.zeros((N, N))
    for n2 in range(-images, images + 1):
        for n1 in range(-images, images + 1):
            u1, u2 = X + n1, Y + n2
            sp += np.exp(-(H[0, 0] * u1 * u1 + (H[0, 1] + H[1, 0]) * u1 * u2 + H[1, 1] * u2 * u2))
    ang = np.exp(-((th - nu) ** 2) / s)
    return ang[:, None, None] * sp[None, :, :]
