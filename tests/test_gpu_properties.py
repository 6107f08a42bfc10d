"""Structural properties of the CUDA path (SURVEY-style property tests),
each exact in exact arithmetic, checked at the path's rounding level:

* linearity in f;
* cyclic grid shifts of f shift the output (the scheme is a cyclic
  convolution of the samples);
* a 90-degree rotation of f with theta shifted by M/4 rotates the output
  (the kernel is radial in translations, Theorem f*gP);
* a chain equals successive single convolutions (associativity).
The oracle pins the same identities in FP64 (test_oracle_pins.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402

TOL = {"f32": 2e-6, "f64": 1e-12}
NP = {"f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    return m


def _rot90(F):
    """f'(x, y, theta) = f(y, -x, theta - pi/2) on Omega_L (x_i = -1/2 + i/N)."""
    M, N = F.shape[-3], F.shape[-1]
    Y, X = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    Fr = np.roll(F, M // 4, axis=-3)
    return Fr[..., (-X) % N, Y]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _conv(se2, plan, F, C):
    return se2.convolve(plan, torch.from_numpy(np.ascontiguousarray(F)).cuda(), C).double().cpu().numpy()


@pytest.mark.parametrize("prec,N,M", [("f32", 256, 64), ("f32", 64, 16), ("f64", 32, 8)])
def test_linearity_shift_and_rotation(se2, prec, N, M):
    B = 2
    rng = np.random.default_rng(N * M)
    F = rng.standard_normal((B, M, N, N)).astype(NP[prec])
    G = rng.standard_normal((B, M, N, N)).astype(NP[prec])
    P = np.stack([synth.sample_kernel(N, M, synth.KernelParams(0.03 + 0.01 * b, 0.4, 0.3 * b)) for b in range(B)])
    plan = se2.Plan(N, M, batch=B, precision=prec)
    C, _ = se2.coeffs(plan, torch.from_numpy(P.astype(NP[prec])).cuda())
    out = _conv(se2, plan, F, C)
    tol = TOL[prec]
    # linearity: a f + b g (formed in FP64, rounded once)
    lin = (2.0 * F.astype(np.float64) - 0.5 * G.astype(np.float64)).astype(NP[prec])
    want = 2.0 * out - 0.5 * _conv(se2, plan, G, C)
    assert _rel(_conv(se2, plan, lin, C), want) < 4 * tol
    # cyclic shifts
    sh = (3, 5, N - 7)
    got = _conv(se2, plan, np.roll(F, sh, axis=(1, 2, 3)), C)
    assert _rel(got, np.roll(out, sh, axis=(1, 2, 3))) < tol
    # 90-degree rotation
    got = _conv(se2, plan, _rot90(F), C)
    assert _rel(got, _rot90(out)) < tol


def test_chain_equals_successive_convolutions(se2):
    N, M, B = 128, 32, 2
    rng = np.random.default_rng(11)
    F = rng.standard_normal((B, M, N, N)).astype(np.float32)
    kps = [synth.KernelParams(0.02, 0.3, 0.1), synth.KernelParams(0.035, 0.2, -0.4), synth.KernelParams(0.015, 0.45, 0.9)]
    plan = se2.Plan(N, M, batch=B)
    Cs = [se2.coeffs(plan, torch.from_numpy(np.stack([synth.sample_kernel(N, M, kp)] * B).astype(np.float32)).cuda())[0]
          for kp in kps]
    f = torch.from_numpy(F).cuda()
    chain = se2.convolve_chain(plan, f, Cs).double().cpu().numpy()
    step = f
    for C in Cs:
        step = se2.convolve(plan, step, C)
    assert _rel(step.double().cpu().numpy(), chain) < 5e-6
