"""Adjoint kernel and kernel-parameter gradients (through the C ABI) against
the FP64 oracle and central finite differences of the oracle loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import se2_oracle as O  # noqa: E402


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("prec,N,M", [("f64", 32, 16), ("f32", 64, 16), ("f32", 16, 8), ("f32", 512, 128)])
def test_sampled_kernel_family_matches_oracle(se2, prec, N, M):
    plan = se2.Plan(N, M, batch=1, precision=prec)
    P, dPs, dPt = se2.sample_radial_gaussian(plan, 0.03, 0.3, 0.4, derivs=True)
    wP, wdPs, wdPt = O.kernel_samples_and_derivs(N, M, 0.03, 0.3, 0.4)
    tol = 1e-13 if prec == "f64" else 1e-6
    assert _rel(P[0].double().cpu().numpy(), wP) < tol
    assert _rel(dPs[0].double().cpu().numpy(), wdPs) < tol
    assert _rel(dPt[0].double().cpu().numpy(), wdPt) < tol


@pytest.mark.parametrize("prec,N,M,B", [("f64", 32, 16, 3), ("f32", 64, 16, 4), ("f32", 256, 64, 2), ("f32", 16, 8, 2)])
def test_adjoint_and_parameter_gradients(se2, prec, N, M, B):
    """grad_f = W conj(C) G^ (correlation) and dL/d(sigma, sigma_theta)
    against the oracle's adjoint and grad_kernel_samples . dP/dparam."""
    npd = np.float64 if prec == "f64" else np.float32
    s, st = 0.035, 0.35
    plan = se2.Plan(N, M, batch=B, precision=prec, flags=se2.SHARED_KERNEL)
    rng = np.random.default_rng(N + M + B)
    F = np.stack([synth.sample_bumps(N, M, synth.make_problem(5, b, N, M, n_bumps=4).bumps) for b in range(B)]).astype(npd)
    G = rng.standard_normal((B, M, N, N)).astype(npd)
    P, dPs, dPt = se2.sample_radial_gaussian(plan, s, st, derivs=True)
    C, _ = se2.coeffs(plan, P)
    dCs, _ = se2.coeffs(plan, dPs)
    dCt, _ = se2.coeffs(plan, dPt)
    f = torch.from_numpy(F).cuda()
    g = torch.from_numpy(G).cuda()
    gf, gp = se2.backward(plan, g, C, f, [dCs, dCt])
    torch.cuda.synchronize()
    Pd = P[0].double().cpu().numpy()
    wP, wdPs, wdPt = O.kernel_samples_and_derivs(N, M, s, st)
    tol = 1e-10 if prec == "f64" else 1e-5
    Fd, Gd = F.astype(np.float64), G.astype(np.float64)
    for b in range(B):
        assert _rel(gf[b].double().cpu().numpy(), O.adjoint(Gd[b], [Pd])) < tol
    gP = O.grad_kernel_samples(Fd, Gd)
    want = np.array([np.sum(gP * wdPs), np.sum(gP * wdPt)])
    got = gp.cpu().numpy()
    assert np.max(np.abs(got - want) / np.abs(want)) < (1e-9 if prec == "f64" else 1e-4)


def test_parameters_only_and_shared_kernel_errors(se2):
    N, M = 32, 8
    plan = se2.Plan(N, M, batch=2, precision="f32", flags=se2.SHARED_KERNEL)
    P = se2.sample_radial_gaussian(plan, 0.05, 0.4)
    C, _ = se2.coeffs(plan, P)
    g = torch.randn((2, M, N, N), device="cuda")
    gf, gp = se2.backward(plan, g, C, want_grad_f=True)
    assert gf.shape == g.shape and gp.numel() == 0
    import ctypes
    lib = se2.load_library()
    # nothing requested -> INVALID_ARG
    assert lib.se2_backward(plan.handle, ctypes.c_void_p(g.data_ptr()), None, 2, ctypes.c_void_p(C.data_ptr()),
                            None, 0, None, None, None, None) == 1


def test_autograd_function_c5_shape_against_finite_differences(se2):
    """Differentiation config shape (N=256, M=64; batch 2 here to keep the
    oracle fast): loss = 1/2 ||f * rho(sigma, sigma_theta) - target||^2,
    autograd gradients vs the oracle gradient and central differences
    (h = 1e-4) of the FP64 oracle loss."""
    N, M, B = 256, 64, 2
    plan = se2.Plan(N, M, batch=B, precision="f32", flags=se2.SHARED_KERNEL)
    F = np.stack([synth.sample_bumps(N, M, synth.make_problem(5, b, N, M, n_bumps=16).bumps) for b in range(B)]).astype(np.float32)
    T = np.stack([O.convolve(synth.sample_bumps(N, M, synth.make_problem(5, 100 + b, N, M, n_bumps=16).bumps),
                             synth.sample_kernel(N, M, synth.KernelParams(0.03, 0.3))) for b in range(B)]).astype(np.float32)
    f = torch.from_numpy(F).cuda().requires_grad_(True)
    params = torch.tensor([0.025, 0.25], dtype=torch.float64, device="cuda", requires_grad=True)
    target = torch.from_numpy(T).cuda()
    out = se2.SE2Conv.apply(f, params, plan)
    loss = 0.5 * ((out - target) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    Fd, Td = F.astype(np.float64), T.astype(np.float64)

    def oloss(s, st):
        P = O.kernel_samples_and_derivs(N, M, s, st)[0]
        return 0.5 * sum(np.sum((O.convolve(Fd[b], P) - Td[b]) ** 2) for b in range(B))

    P, dPs, dPt = O.kernel_samples_and_derivs(N, M, 0.025, 0.25)
    R = np.stack([O.convolve(Fd[b], P) - Td[b] for b in range(B)])
    gP = O.grad_kernel_samples(Fd, R)
    want = np.array([np.sum(gP * dPs), np.sum(gP * dPt)])
    got = params.grad.cpu().numpy()
    # The gradient is an inner product of the residual R = out - target with
    # f * dP: an FP32 forward output (error ~3e-7 of max|out|) moves R, and
    # the sum cancels.  The oracle gradient taken on the GPU's own residual
    # (its FP32 output, exactly) separates that conditioning from the adjoint
    # kernel's own arithmetic, which must meet the FP32 bar.
    Rg = out.detach().double().cpu().numpy() - Td
    gPg = O.grad_kernel_samples(Fd, Rg)
    want_g = np.array([np.sum(gPg * dPs), np.sum(gPg * dPt)])
    err_adjoint = float(np.max(np.abs(got - want_g) / np.abs(want_g)))
    cond = float(np.max(np.abs(want_g - want) / np.abs(want)))
    err_total = float(np.max(np.abs(got - want) / np.abs(want)))
    print(f"c5 parameter gradients: vs oracle {err_total:.2e}; adjoint alone {err_adjoint:.2e}; "
          f"FP32 forward through the loss (oracle on the GPU residual) {cond:.2e}")
    assert err_adjoint < 1e-5
    assert err_total < max(1e-5, 2 * cond + 1e-5)
    h = 1e-4
    fd = np.array([(oloss(0.025 + h, 0.25) - oloss(0.025 - h, 0.25)) / (2 * h),
                   (oloss(0.025, 0.25 + h) - oloss(0.025, 0.25 - h)) / (2 * h)])
    assert np.max(np.abs(want - fd) / np.abs(fd)) < 1e-5         # oracle gradient vs FD
    assert np.max(np.abs(got - fd) / np.abs(fd)) < max(1e-5, 2 * cond + 2e-5)
    gf = f.grad.double().cpu().numpy()
    for b in range(B):
        assert _rel(gf[b], O.adjoint(Rg[b], [P])) < 1e-5           # the adjoint of the GPU residual
        assert _rel(gf[b], O.adjoint(R[b], [P])) < 1e-5


def test_autograd_spectra_cached_while_params_unchanged(se2):
    """SE2Conv reuses the kernel spectra while the params tensor is unchanged
    (no resampling: fewer launches) and recomputes them after an in-place
    update; the outputs follow the parameters."""
    N, M, B = 32, 8, 2
    plan = se2.Plan(N, M, batch=B, precision="f32", flags=se2.SHARED_KERNEL)
    f = torch.rand((B, M, N, N), device="cuda")
    params = torch.tensor([0.04, 0.3], dtype=torch.float64)      # on the host: never read from the device
    out1 = se2.SE2Conv.apply(f, params, plan)
    n1 = plan.launches()
    out2 = se2.SE2Conv.apply(f, params, plan)
    n2 = plan.launches()
    assert torch.equal(out1, out2)
    with torch.no_grad():
        params[0] = 0.05
    out3 = se2.SE2Conv.apply(f, params, plan)
    n3 = plan.launches()
    assert n3 - n2 > n2 - n1                                     # sampling and coefficients ran again
    P = O.kernel_samples_and_derivs(N, M, 0.05, 0.3)[0]
    want = O.convolve(f[0].double().cpu().numpy(), P)
    assert _rel(out3[0].double().cpu().numpy(), want) < 1e-5
