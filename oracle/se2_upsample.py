"""FP64 CPU oracle for the convolutional finite Fourier series on odd
sampling grids L = 2K + 1, evaluated on an output grid N >= L.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import, call or link anything
under oracle/.  The product path never does, and this module never imports
the product.

Arrays are [theta][y][x]: samples F = f on Omega_L (x_i = -1/2 + i/L_x,
theta_l = 2 pi l / L_r, 0-based) and outputs on the N-grid
x'_n = -1/2 + n/N_x, theta'_l = 2 pi l / N_r.  Sizes L_x, L_y, L_r are odd
(L = 2K + 1 per axis), N >= L per axis, any parity.

* series: the definition.  S_K[f, rho_1 .. rho_q](w) =
  sum_{|k| <= K} f^[k; L] rho_1^[k; L] ... rho_q^[k; L] phi_k(w) (Eq. SKfgq;
  Section 6.1), with the finite Fourier coefficients of Eq. FkLv and
  phi_k(x, y, theta) = exp(2 pi i (k1 x + k2 y)) exp(i k3 theta), summed
  with explicit exponential matrices on the N-grid.
* matrix: the paper's matrix form (Eq. MatSKfgonG, q = 1) with the
  zero-padded spectra Q of Eq. Qf and the sign array W of Eq. W on the N-grid,
  both written out case by case from their index sets I = 1:K+1 and
  J = N-K+1:N.  For q kernels the scale is N_x N_y N_r / |L|^(q+1) and the
  sign array is W^q (each extra coefficient array carries one more
  (-1)^(k1+k2), Eq. FkLv).
* zero_pad: the vector z of Proposition LtoN1D with c = 1 (Corollary LtoN1D+1).

Pinned by tests/test_oracle_upsample.py: series = matrix, N = L = the
N = L oracle (se2_oracle.convolve_chain), restriction of an N = rL output to
the coarse grid = the N = L output, Proposition LtoN1D and its corollaries by
brute force, and exactness for trigonometric polynomials of degree <= K
(Lemma TrigL) at off-grid output points.
"""
from __future__ import annotations

import numpy as np

__all__ = ["signed", "ffc_odd", "series", "matrix", "zero_pad", "q_array", "w_array"]


def signed(L: int) -> np.ndarray:
    """k = tau_L^{-1}(bin) for L = 2K+1 (Eq. tauKk): 0..K, then -K..-1."""
    K = (L - 1) // 2
    b = np.arange(L)
    return np.where(b <= K, b, b - L)


def _check_odd(shape):
    for L in shape:
        if L % 2 != 1:
            raise ValueError(f"sampling sizes must be odd (L = 2K+1), got {shape}")


def ffc_odd(F: np.ndarray) -> np.ndarray:
    """f^[k; L] at every bin (Eq. FkLv): (-1)^(k1+k2) / |L| * DFT(F)(tau(k))."""
    Lr, Ly, Lx = F.shape
    kx, ky = signed(Lx), signed(Ly)
    sgn = (-1.0) ** (ky[:, None] + kx[None, :])
    return sgn[None, :, :] * np.fft.fftn(F) / F.size


def series(F: np.ndarray, Ps, Nout) -> np.ndarray:
    """S_K[f, rho_1..rho_q] on the N-grid, from the definition (complex)."""
    _check_odd(F.shape)
    Lr, Ly, Lx = F.shape
    Nr, Ny, Nx = Nout
    c = ffc_odd(F)
    for P in Ps:
        c = c * ffc_odd(P)
    kx, ky, kr = signed(Lx), signed(Ly), signed(Lr)
    xs = -0.5 + np.arange(Nx) / Nx
    ys = -0.5 + np.arange(Ny) / Ny
    ts = 2.0 * np.pi * np.arange(Nr) / Nr
    Ex = np.exp(2j * np.pi * np.outer(xs, kx))   # [Nx][Lx bins]
    Ey = np.exp(2j * np.pi * np.outer(ys, ky))
    Er = np.exp(1j * np.outer(ts, kr))
    return np.einsum("ak,bj,ci,kji->abc", Er, Ey, Ex, c, optimize=True)


def zero_pad(x: np.ndarray, N: int, c=None) -> np.ndarray:
    """z of Proposition LtoN1D (1-based in the paper, 0-based here):
    z[n] = c_n x[n] for n <= K, z[n] = c_{n-N} x[L+n-N] for n >= N-K, else 0."""
    L = x.shape[-1]
    K = (L - 1) // 2
    cc = np.ones(2 * K + 1) if c is None else np.asarray(c)   # c indexed by k + K
    z = np.zeros(x.shape[:-1] + (N,), dtype=np.complex128)
    for n in range(K + 1):
        z[..., n] = cc[n + K] * x[..., n]
    for n in range(N - K, N):
        z[..., n] = cc[n - N + K] * x[..., L + n - N]
    return z


def q_array(Fh: np.ndarray, Nout) -> np.ndarray:
    """Q of Eq. Qf: the DFT Fh on L bins placed on N bins, the blocks of the
    index sets I = 0..K (0-based) and J = N-K..N-1 taken from bins 0..K and
    L-K..L-1, zero elsewhere."""
    Lr, Ly, Lx = Fh.shape
    Nr, Ny, Nx = Nout
    Q = np.zeros((Nr, Ny, Nx), dtype=np.complex128)

    def src(n, N, L):
        K = (L - 1) // 2
        if n <= K:
            return n
        if n >= N - K:
            return L + n - N
        return None

    for a in range(Nr):
        sa = src(a, Nr, Lr)
        if sa is None:
            continue
        for b in range(Ny):
            sb = src(b, Ny, Ly)
            if sb is None:
                continue
            for c in range(Nx):
                sc = src(c, Nx, Lx)
                if sc is not None:
                    Q[a, b, c] = Fh[sa, sb, sc]
    return Q


def w_array(Lshape, Nout) -> np.ndarray:
    """W of Eq. W on the N-grid: (-1)^(n_x + n_y) with n_x taken as n - N_x on
    J_x (and likewise for y), i.e. (-1)^(k1 + k2) of the signed frequency the
    bin holds; 0 outside the blocks."""
    Lr, Ly, Lx = Lshape
    Nr, Ny, Nx = Nout

    def sgn(n, N, L):
        K = (L - 1) // 2
        if n <= K:
            return (-1.0) ** n
        if n >= N - K:
            return (-1.0) ** (n - N)
        return 0.0

    sx = np.array([sgn(n, Nx, Lx) for n in range(Nx)])
    sy = np.array([sgn(n, Ny, Ly) for n in range(Ny)])
    sr = np.array([1.0 if (n <= (Lr - 1) // 2 or n >= Nr - (Lr - 1) // 2) else 0.0 for n in range(Nr)])
    return sr[:, None, None] * sy[None, :, None] * sx[None, None, :]


def matrix(F: np.ndarray, Ps, Nout) -> np.ndarray:
    """Eq. MatSKfgonG generalised to q kernels:
    N_x N_y N_r / |L|^(q+1) * iDFT(W^q . Q_f . Q_rho_1 ... Q_rho_q) (complex)."""
    _check_odd(F.shape)
    q = len(Ps)
    Lsz = F.size
    H = q_array(np.fft.fftn(F), Nout)
    for P in Ps:
        H = H * q_array(np.fft.fftn(P), Nout)
    W = w_array(F.shape, Nout)
    Nr, Ny, Nx = Nout
    return (Nr * Ny * Nx) / Lsz ** (q + 1) * np.fft.ifftn(W ** q * H)
