"""FP64 CPU oracle for the fast SE(2) convolution on Z^2\\SE(2).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import, call or link anything
under oracle/.  The product path (the CUDA library and its Python binding)
never does, and this module never imports the product.

What it computes, with the passage of arXiv 2504.05149 each function follows:

* Arrays are [theta_l][y_j][x_i] samples on the fundamental grid Omega_L
  (Section 3.2, Eq. OmL).  Frequencies are indexed by DFT bins; the signed
  frequency of bin i is tau_L^{-1}(i) (Section 2.1 item 3, Eq. tauKk).
* dft3 / idft3: the 3-D DFT and iDFT of Section 2.3 (Eqs. 3DFT, 3iDFT).
  Route "matrix" writes the DFT definition out with explicit DFT matrices;
  route "fft" calls numpy.fft (a library primitive used as one step).
* ffc: the finite Fourier coefficient via its matrix form (Section 4.1,
  Eq. FkLv).
* convolve: the convolutional finite Fourier series at N = L (Section 6.1,
  closed form below Eq. MatSKfgonG; Algorithm 3).
* convolve_power: the q-fold scheme with a Hadamard power and W only for odd
  q (Section 6.3, Eq. MatSqKfgG; Algorithm 4).
* convolve_chain: the same with q distinct radial kernels (the product of their
  coefficient arrays replaces the power; W^q).
* convolve_all: every intermediate V_p from one forward transform
  (Algorithm 6, the fast recursion).
* adjoint / grad_kernel_samples: transposes of the linear maps above (not in
  the paper; derived here: the transpose of iDFT(W.C.DFT(.)) is
  iDFT(W.conj(C).DFT(.)) for real arrays).

Readings where the paper is silent:
even grid sizes use the N = L closed form unchanged, W(k) = (-1)^(k1+k2) with
k the signed frequency of the bin; the output is the real part.

Every function here is pinned by tests/test_oracle_*.py against brute-force
sums (oracle/direct.c), closed forms of Gaussian/von Mises/wrapped-normal
inputs, Lemma TrigL, mass conservation and the error bound of Theorem UkL.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "signed_freq", "dft3", "idft3", "weight_W", "ffc", "coeffs_full", "coeffs_half",
    "coeffs_separable", "convolve", "convolve_complex", "convolve_power",
    "convolve_chain", "convolve_all", "adjoint", "grad_kernel_samples", "half_to_full",
]


def signed_freq(n: int) -> np.ndarray:
    """Signed frequency k of each DFT bin i = tau_n(k) (Eq. tauKk): i if
    i <= floor((n-1)/2) else i - n.  For even n the Nyquist bin gets -n/2;
    its parity, the only thing W uses, is the same as +n/2."""
    i = np.arange(n)
    return np.where(i <= (n - 1) // 2, i, i - n)


def _dft_matrix(n: int, sign: int) -> np.ndarray:
    # E[k, j] = exp(sign * 2 pi i k j / n); the exponent is reduced mod n first
    # so that large k*j keep full accuracy.
    kj = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(sign * 2j * np.pi * kj / n)


def dft3(X: np.ndarray, route: str = "fft") -> np.ndarray:
    """Unnormalised forward 3-D DFT over the last three axes (Eq. 3DFT)."""
    if route == "fft":
        return np.fft.fftn(X, axes=(-3, -2, -1))
    if route == "matrix":
        M, Ny, Nx = X.shape[-3:]
        Y = np.asarray(X, dtype=np.complex128)
        Y = np.einsum("...lji,ki->...ljk", Y, _dft_matrix(Nx, -1))
        Y = np.einsum("...lji,kj->...lki", Y, _dft_matrix(Ny, -1))
        Y = np.einsum("...lji,kl->...kji", Y, _dft_matrix(M, -1))
        return Y
    raise ValueError(route)


def idft3(X: np.ndarray, route: str = "fft") -> np.ndarray:
    """Inverse 3-D DFT with the 1/(L_x L_y L_r) factor (Eq. 3iDFT)."""
    if route == "fft":
        return np.fft.ifftn(X, axes=(-3, -2, -1))
    if route == "matrix":
        M, Ny, Nx = X.shape[-3:]
        Y = np.asarray(X, dtype=np.complex128)
        Y = np.einsum("...lji,ki->...ljk", Y, _dft_matrix(Nx, +1))
        Y = np.einsum("...lji,kj->...lki", Y, _dft_matrix(Ny, +1))
        Y = np.einsum("...lji,kl->...kji", Y, _dft_matrix(M, +1))
        return Y / (M * Ny * Nx)
    raise ValueError(route)


def weight_W(N: int, M: int, Ny: int | None = None) -> np.ndarray:
    """The weight array W of Eq. W at N = L: (-1)^(k1 + k2) at every bin,
    k1, k2 the signed x, y frequencies; constant along theta.
    Shape [M][Ny][N] (broadcastable)."""
    Ny = N if Ny is None else Ny
    kx = signed_freq(N)
    ky = signed_freq(Ny)
    w = ((-1.0) ** (ky[:, None] + kx[None, :]))
    return np.broadcast_to(w[None, :, :], (M, Ny, N)).copy()


def ffc(F: np.ndarray, route: str = "fft") -> np.ndarray:
    """Finite Fourier coefficients f^[k; L] at every DFT bin, through the
    matrix form Eq. FkLv: (-1)^(k1+k2) / (L_x L_y L_r) * DFT(F)(tau(k))."""
    M, Ny, Nx = F.shape[-3:]
    return weight_W(Nx, M, Ny) * dft3(F, route) / (M * Ny * Nx)


def coeffs_full(P: np.ndarray, route: str = "fft") -> np.ndarray:
    """Scaled kernel spectrum C = DFT(P) / |L| on all bins.  By Eq. FkLv this
    is W times the FFC of the kernel."""
    M, Ny, Nx = P.shape[-3:]
    return dft3(P, route) / (M * Ny * Nx)


def coeffs_half(P: np.ndarray, route: str = "fft") -> np.ndarray:
    """The bins 0..N/2 along x of coeffs_full: the layout [M][N][N/2+1] that
    the library exchanges (the rest follows from Hermitian symmetry)."""
    Nx = P.shape[-1]
    return coeffs_full(P, route)[..., : Nx // 2 + 1]


def half_to_full(Ch: np.ndarray, Nx: int) -> np.ndarray:
    """Rebuild all x bins from the half spectrum of a real array:
    C[l, j, i] = conj(C[-l, -j, -i])."""
    M, Ny, H = Ch.shape[-3:]
    full = np.empty(Ch.shape[:-1] + (Nx,), dtype=np.complex128)
    full[..., :H] = Ch
    for i in range(H, Nx):
        src = Ch[..., Nx - i]
        # conj at the negated (theta, y) bins
        src = np.roll(np.flip(src, axis=(-2, -1)), shift=(1, 1), axis=(-2, -1))
        full[..., i] = np.conj(src)
    return full


def coeffs_separable(gx: np.ndarray, gy: np.ndarray, gt: np.ndarray) -> np.ndarray:
    """DFT(P)/|L| for a separable kernel P[l, j, i] = gt[l] gy[j] gx[i]: the
    3-D DFT of an outer product is the outer product of the 1-D DFTs."""
    cx = np.fft.fft(gx) / gx.size
    cy = np.fft.fft(gy) / gy.size
    ct = np.fft.fft(gt) / gt.size
    return ct[:, None, None] * cy[None, :, None] * cx[None, None, :]


def _weight(Nx: int, M: int, Ny: int, origin_zero: bool):
    """W of Eq. W for grids on Omega_L (x_i = -1/2 + i/N); 1 for grids sampled
    at x_i = i/N, where the rectangle rule is the plain cyclic convolution
    (the -1/2 offset is what the half-period shift W undoes)."""
    return 1.0 if origin_zero else weight_W(Nx, M, Ny)


def convolve_complex(F: np.ndarray, P: np.ndarray, route: str = "fft", origin_zero: bool = False) -> np.ndarray:
    """Algorithm 3 at output grid N = L: (1/|L|) iDFT(W . DFT(F) . DFT(P))
    (closed form below Eq. MatSKfgonG), before taking the real part."""
    M, Ny, Nx = F.shape[-3:]
    L = M * Ny * Nx
    H = _weight(Nx, M, Ny, origin_zero) * dft3(F, route) * dft3(P, route)
    return idft3(H, route) / L


def convolve(F: np.ndarray, P: np.ndarray, route: str = "fft", origin_zero: bool = False) -> np.ndarray:
    """Re S_K[f, rho] on Omega_L (Algorithm 3; the paper plots the real part)."""
    return convolve_complex(F, P, route, origin_zero).real


def convolve_power(F: np.ndarray, P: np.ndarray, q: int, route: str = "fft") -> np.ndarray:
    """Algorithm 4 (Eq. MatSqKfgG at N = L): iDFT(W^q . F^ . P^^q) / |L|^q,
    with W applied only when q is odd."""
    M, Ny, Nx = F.shape[-3:]
    L = M * Ny * Nx
    Fh = dft3(F, route)
    Ph = dft3(P, route)
    H = Fh * Ph ** q
    if q % 2 == 1:
        H = weight_W(Nx, M, Ny) * H
    return (idft3(H, route) / float(L) ** q).real


def convolve_chain(F: np.ndarray, Ps, route: str = "fft", coeffs=None, origin_zero: bool = False) -> np.ndarray:
    """f * rho_1 * ... * rho_q for q radial kernels: iDFT(W^q . F^ . prod_i C_i)
    with C_i = DFT(P_i)/|L| (Eq. MatSqKfgG with the power replaced by the
    product of the coefficient arrays).  `coeffs` may pass the C_i directly."""
    M, Ny, Nx = F.shape[-3:]
    if coeffs is None:
        coeffs = [coeffs_full(P, route) for P in Ps]
    q = len(coeffs)
    H = dft3(F, route)
    for C in coeffs:
        H = H * C
    if q % 2 == 1:
        H = _weight(Nx, M, Ny, origin_zero) * H
    return idft3(H, route).real


def convolve_all(F: np.ndarray, Ps, route: str = "fft"):
    """Algorithm 6 (fast recursion): V = DFT(F); for p = 1..q:
    H = W . V . DFT(P_p); emit iDFT(H) / |L|^p; V = H.  Returns [V_1..V_q].
    A single kernel repeated q times is the paper's case; distinct kernels are
    allowed (same recursion)."""
    M, Ny, Nx = F.shape[-3:]
    L = M * Ny * Nx
    W = weight_W(Nx, M, Ny)
    V = dft3(F, route)
    outs = []
    for p, P in enumerate(Ps, start=1):
        H = W * V * dft3(P, route)
        outs.append((idft3(H, route) / float(L) ** p).real)
        V = H
    return outs


def adjoint(G: np.ndarray, Ps, route: str = "fft", coeffs=None, origin_zero: bool = False) -> np.ndarray:
    """Transpose of f -> convolve_chain(f, Ps) applied to G (the gradient of a
    loss with respect to f given its gradient G with respect to the output):
    iDFT(W^q . conj(prod_i C_i) . DFT(G)).  For q = 1 this is the discrete
    correlation with the kernel."""
    M, Ny, Nx = G.shape[-3:]
    if coeffs is None:
        coeffs = [coeffs_full(P, route) for P in Ps]
    H = dft3(G, route)
    for C in coeffs:
        H = H * np.conj(C)
    if len(coeffs) % 2 == 1:
        H = _weight(Nx, M, Ny, origin_zero) * H
    return idft3(H, route).real


def grad_kernel_samples(F: np.ndarray, G: np.ndarray, route: str = "fft") -> np.ndarray:
    """Gradient of <G, convolve(F, P)> with respect to the kernel samples P for
    a single convolution.  convolve is symmetric in (F, P), so this is the
    transpose of P -> convolve(F, P): iDFT(W . conj(DFT(F)) . DFT(G)) / |L|.
    Leading batch axes of F and G are summed."""
    M, Ny, Nx = G.shape[-3:]
    L = M * Ny * Nx
    H = weight_W(Nx, M, Ny) * np.conj(dft3(F, route)) * dft3(G, route)
    g = idft3(H, route).real / L
    while g.ndim > 3:
        g = g.sum(axis=0)
    return g


# ---------------------------------------------------------------------------
# The radial kernel family used for differentiation (Gaussian in x times 2 pi
# times a wrapped normal in theta; the paper's radial Gaussians of Section 6.2
# with unit mass under Eq. dg), and its derivatives in (sigma, sigma_theta).
# Independent of synth/ (which only samples the values).
# ---------------------------------------------------------------------------

def _kernel_1d(N: int, M: int, sigma: float, sigma_t: float, nu: float = 0.0, images: int = 2, terms: int = 4,
               origin_zero: bool = False):
    x = (0.0 if origin_zero else -0.5) + np.arange(N) / N
    d = np.mod(x + 0.5, 1.0) - 0.5
    g = np.zeros(N)
    dg = np.zeros(N)
    for n in range(-images, images + 1):
        u2 = (d + n) ** 2
        e = np.exp(-u2 / (2 * sigma * sigma))
        g += e
        dg += e * (-1.0 / sigma ** 2 + u2 / sigma ** 4)
    g /= np.sqrt(2 * np.pi) * sigma
    dg /= np.sqrt(2 * np.pi)
    th = 2 * np.pi * np.arange(M) / M
    v = np.mod(th - nu + np.pi, 2 * np.pi) - np.pi
    t = np.zeros(M)
    dt = np.zeros(M)
    for m in range(-terms, terms + 1):
        v2 = (v + 2 * np.pi * m) ** 2
        e = np.exp(-v2 / (2 * sigma_t * sigma_t))
        t += e
        dt += e * (-1.0 / sigma_t ** 2 + v2 / sigma_t ** 4)
    t *= np.sqrt(2 * np.pi) / sigma_t
    dt *= np.sqrt(2 * np.pi)
    return g, dg, t, dt


def kernel_samples_and_derivs(N: int, M: int, sigma: float, sigma_t: float, nu: float = 0.0,
                              origin_zero: bool = False):
    """P, dP/dsigma, dP/dsigma_theta sampled on Omega_L (or at x_i = i/N),
    each [M][N][N]."""
    g, dg, t, dt = _kernel_1d(N, M, sigma, sigma_t, nu, origin_zero=origin_zero)
    P = t[:, None, None] * g[None, :, None] * g[None, None, :]
    dPs = t[:, None, None] * (dg[None, :, None] * g[None, None, :] + g[None, :, None] * dg[None, None, :])
    dPt = dt[:, None, None] * g[None, :, None] * g[None, None, :]
    return P, dPs, dPt
