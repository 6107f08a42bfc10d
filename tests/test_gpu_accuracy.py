"""Algorithm 1 (accuracy-driven order K) and the FFC convergence report on
the GPU, for the paper's deformed Gaussian f = exp(-x^T H x) exp(-(t-nu)^2/s)
with H = diag(0.04, 0.1)^-1, s = 0.4, nu = pi (Section 4.2)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import se2_oracle as O  # noqa: E402

HX, HY, S, NU = 1 / 0.04, 1 / 0.1, 0.4, math.pi
KV = (1, -2, 3)


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    return m


def sample(L):
    Lx, Ly, Lr = L
    x = -0.5 + np.arange(Lx) / Lx
    y = -0.5 + np.arange(Ly) / Ly
    t = 2 * math.pi * np.arange(Lr) / Lr
    return (np.exp(-(t[:, None, None] - NU) ** 2 / S) * np.exp(-HY * y[None, :, None] ** 2)
            * np.exp(-HX * x[None, None, :] ** 2))


def exact_coeff(k):
    """f^[k] = (1/2pi) int over Omega of f conj(phi_k), by 1-D quadrature
    (the function is separable)."""
    from scipy import integrate
    k1, k2, k3 = k

    def c1d(fun, a, b, w):
        re = integrate.quad(lambda t: fun(t) * math.cos(w * t), a, b, limit=200, epsabs=1e-14)[0]
        im = integrate.quad(lambda t: -fun(t) * math.sin(w * t), a, b, limit=200, epsabs=1e-14)[0]
        return re + 1j * im
    return (c1d(lambda x: math.exp(-HX * x * x), -0.5, 0.5, 2 * math.pi * k1)
            * c1d(lambda y: math.exp(-HY * y * y), -0.5, 0.5, 2 * math.pi * k2)
            * c1d(lambda t: math.exp(-(t - NU) ** 2 / S), 0, 2 * math.pi, k3) / (2 * math.pi))


def grad_sup():
    g = np.linspace(-0.5, 0.5, 201)
    t = np.linspace(0, 2 * math.pi, 401)
    X, Y, T = np.meshgrid(g, g, t, indexing="ij")
    f = np.exp(-HX * X * X - HY * Y * Y - (T - NU) ** 2 / S)
    return float((f * np.sqrt((2 * HX * X) ** 2 + (2 * HY * Y) ** 2 + (2 * (T - NU) / S) ** 2)).max())


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ffc_report_matches_oracle_and_bound(se2, prec):
    Ks = list(range(3, 13))
    rep = se2.ffc_convergence(sample, KV, Ks, precision=prec)
    true = exact_coeff(KV)
    G = grad_sup()
    tol = {"f64": 1e-12, "f32": 2e-6}[prec]
    for (K, v, d), K0 in zip(rep, Ks):
        assert K == K0
        L = 2 * K + 1
        C = O.ffc(sample((L, L, L)))
        kb = O.signed_freq(L)
        want = C[np.where(kb == KV[2])[0][0], np.where(kb == KV[1])[0][0], np.where(kb == KV[0])[0][0]]
        assert abs(v - want) <= tol * np.max(np.abs(C))
        assert abs(v - true) <= 36 * G / K          # Theorem UkL's constant (the proof of fkLmain)
    assert abs(rep[-1][1] - true) < 0.1 * abs(rep[0][1] - true)


def test_algorithm1_end_to_end(se2):
    """Pick K by Algorithm 1 for eps = 1.5 (the bound is loose: K stays within
    the grid plans' sizes only for such eps), compute f^[k; 2K+1] on the GPU
    and check it against the exact coefficient."""
    G = grad_sup()
    eps = 1.5
    K = se2.accuracy_order(eps, G, KV, constant=36.0)
    assert K == max(math.ceil(36 * G / eps), 3)
    assert 2 * K + 1 <= 255
    (Kr, v, _), = se2.ffc_convergence(sample, KV, [K], precision="f32")
    assert abs(v - exact_coeff(KV)) <= eps
