"""Mixed precision: the angular DFT on the tensor cores (tcgen05, bf16 or
fp16 hi+lo split, or one bf16 product, FP32 accumulation) against the FP64
oracle, beside the plain FP32 path.  Bars: 1e-3 relative for the split-bf16
mode (its error is reported, and in practice near 1e-5), 1e-5 (the FP32 bar)
for split fp16, 1e-2 for one bf16 product."""
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


@pytest.mark.parametrize("N,M,B", [(64, 64, 3), (128, 64, 2), (32, 128, 3), (256, 128, 1)])
def test_split_bf16_and_bf16_vs_oracle(se2, N, M, B):
    rng = np.random.default_rng(N + M)
    F = rng.standard_normal((B, M, N, N)).astype(np.float32)
    P = rng.random((B, M, N, N)).astype(np.float32)
    errs = {}
    for prec in ("f32", "split_bf16", "split_f16", "bf16"):
        plan = se2.Plan(N, M, batch=B, precision=prec)
        C, _ = se2.coeffs(plan, torch.from_numpy(P).cuda())
        out = se2.convolve(plan, torch.from_numpy(F).cuda(), C).double().cpu().numpy()
        plan.status()
        errs[prec] = max(_rel(out[b], O.convolve(F[b].astype(np.float64), P[b].astype(np.float64))) for b in range(B))
    assert errs["f32"] < 3e-6
    assert errs["split_bf16"] < 1e-3
    assert errs["split_f16"] < 1e-5          # the FP32 bar: about 22 bits kept
    assert errs["bf16"] < 2e-2
    assert errs["split_f16"] < errs["split_bf16"] < errs["bf16"]
    print("max-rel errors", errs)


def test_precision_config_chain_log_amplitudes(se2):
    """Precision-config shape at reduced size: 32-bump f1 with amplitudes
    log-uniform in [1e-6, 1] and a 32-fold separable kernel chain."""
    N, M = 128, 128
    prob = synth.make_problem(3, 0, N, M, n_bumps=32, n_kernels=32, log_amp=True)
    F = synth.sample_bumps(N, M, prob.bumps).astype(np.float32)
    params = torch.zeros((1, 32, 3), dtype=torch.float64)
    for j, kp in enumerate(prob.kernels):
        params[0, j] = torch.tensor([kp.sigma, kp.sigma_theta, kp.nu])
    coeffs = []
    for kp in prob.kernels:
        gx, gy, gt = synth.kernel_factors(N, M, kp)
        coeffs.append(O.coeffs_separable(gx, gy, gt))
    want = O.convolve_chain(F.astype(np.float64), None, coeffs=coeffs)
    for prec, tol in (("f32", 1e-5), ("split_bf16", 1e-3), ("split_f16", 1e-5)):
        plan = se2.Plan(N, M, batch=1, precision=prec)
        tab = se2.separable_tables(plan, params.cuda(), torch.tensor([32], dtype=torch.int32).cuda())
        out = se2.convolve_separable(plan, torch.from_numpy(F[None]).cuda(), tab)[0].double().cpu().numpy()
        plan.status()
        assert _rel(out, want) < tol, prec


def test_split_f16_scales_lines_into_range(se2):
    """Inputs far outside fp16's range (1e8 and 1e-8 amplitudes) keep FP32
    accuracy: each line is scaled by a power of two before the split."""
    N, M, B = 64, 64, 2
    rng = np.random.default_rng(7)
    F = rng.standard_normal((B, M, N, N)).astype(np.float32)
    F[0] *= np.float32(1e8)
    F[1] *= np.float32(1e-8)
    P = rng.random((B, M, N, N)).astype(np.float32)
    plan = se2.Plan(N, M, batch=B, precision="split_f16")
    C, _ = se2.coeffs(plan, torch.from_numpy(P).cuda())
    out = se2.convolve(plan, torch.from_numpy(F).cuda(), C).double().cpu().numpy()
    plan.status()
    for b in range(B):
        assert _rel(out[b], O.convolve(F[b].astype(np.float64), P[b].astype(np.float64))) < 1e-5


def test_tc_unsupported_angular_size(se2):
    with pytest.raises(se2.SE2Error) as ei:
        se2.Plan(64, 32, batch=1, precision="split_bf16")
    assert ei.value.status == 2


@pytest.mark.parametrize("prec,k,shared", [("split_bf16", 1, False), ("bf16", 1, True), ("f32", 8, False)])
def test_mass_renormalisation(se2, prec, k, shared):
    """SE2_MASS_RENORM: sum(out) equals sum(f) * prod C_i[0] * exp(sum ls) to
    FP64 rounding (the exact DC of the product), while the samples stay
    within the mode's error bar."""
    N, M, B = 64, 64, 2
    rng = np.random.default_rng(11 + k)
    F = (rng.random((B, M, N, N)) + 0.5).astype(np.float32)
    Ps = [(rng.random((1 if shared else B, M, N, N)) * (10.0 ** i)).astype(np.float32) for i in range(k)]
    flags = se2.MASS_RENORM | (se2.SHARED_KERNEL if shared else 0)
    outs = {}
    for fl in (0, flags):
        plan = se2.Plan(N, M, batch=B, precision=prec, flags=fl | (se2.SHARED_KERNEL if shared else 0))
        Cs, Ls = [], []
        for P in Ps:
            C, ls = se2.coeffs(plan, torch.from_numpy(P).cuda(), normalize=True)
            Cs.append(C)
            Ls.append(ls)
        outs[fl] = se2.convolve_chain(plan, torch.from_numpy(F).cuda(), Cs, Ls).double().cpu().numpy()
        plan.status()
        cdc = [C[:, 0, 0, 0].real.double().cpu().numpy() * np.exp(l.cpu().numpy()) for C, l in zip(Cs, Ls)]
    tol = {"split_bf16": 1e-3, "bf16": 2e-2, "f32": 1e-5}[prec]
    for b in range(B):
        bb = 0 if shared else b
        target = F[b].astype(np.float64).sum() * np.prod([c[bb] for c in cdc])
        got = outs[flags][b].sum()
        assert abs(got - target) <= 1e-9 * abs(target)   # FP32 rounding of the stored samples
        want = O.convolve_chain(F[b].astype(np.float64), [P[bb].astype(np.float64) for P in Ps])
        assert _rel(outs[flags][b], want) < tol
        # without the flag the mass carries the mode's rounding
        assert abs(outs[0][b].sum() - target) >= abs(got - target)


def _chain_coeffs_separable(N, M, kernels):
    """prod_i C_i of separable kernels, built from the product of their 1-D
    factors (the exact product of outer products)."""
    fx = np.ones(N, dtype=np.complex128)
    fy = np.ones(N, dtype=np.complex128)
    ft = np.ones(M, dtype=np.complex128)
    for kp in kernels:
        gx, gy, gt = synth.kernel_factors(N, M, kp)
        fx = fx * np.fft.fft(gx) / N
        fy = fy * np.fft.fft(gy) / N
        ft = ft * np.fft.fft(gt) / M
    return ft[:, None, None] * fy[None, :, None] * fx[None, None, :]


def test_separable_factor_product_matches_the_oracle_coefficients():
    """The factor-wise product used below equals the oracle's product of
    coeffs_separable arrays (checked at a small size)."""
    N, M = 16, 8
    rng = synth.SplitMix64(99)
    kernels = [synth.draw_kernel(rng) for _ in range(5)]
    want = np.ones((M, N, N), dtype=np.complex128)
    for kp in kernels:
        want = want * O.coeffs_separable(*synth.kernel_factors(N, M, kp))
    got = _chain_coeffs_separable(N, M, kernels)
    assert np.max(np.abs(got - want)) < 1e-14 * np.max(np.abs(want))


def test_c3_full_size_split_modes_vs_oracle(se2):
    """The precision config at its stated size: N = 512, M = 128, batch 8,
    32-bump f1 with amplitudes log-uniform in [1e-6, 1], a 32-fold separable
    kernel chain per problem; split-bf16, split-fp16 and FP32 against the FP64
    oracle on problems 0 and 7 (bars 1e-3, 1e-5, 1e-5)."""
    N, M, B, K = 512, 128, 8, 32
    dev = torch.device("cuda", 0)
    probs = [synth.make_problem(3, b, N, M, n_bumps=32, n_kernels=K, log_amp=True) for b in range(B)]
    f = torch.stack([synth.sample_bumps_torch(N, M, p.bumps, dev, torch.float32) for p in probs]).contiguous()
    params = torch.zeros((B, K, 3), dtype=torch.float64)
    for b, p in enumerate(probs):
        for j, kp in enumerate(p.kernels):
            params[b, j] = torch.tensor([kp.sigma, kp.sigma_theta, kp.nu])
    params = params.to(dev)
    kk = torch.full((B,), K, dtype=torch.int32, device=dev)
    outs = {}
    for prec in ("split_bf16", "split_f16", "f32"):
        plan = se2.Plan(N, M, batch=B, precision=prec)
        tab = se2.separable_tables(plan, params, kk)
        outs[prec] = se2.convolve_separable(plan, f, tab)
        plan.status()
        plan.close()
    errs = {p: 0.0 for p in outs}
    for b in (0, 7):
        F = f[b].double().cpu().numpy()
        C = _chain_coeffs_separable(N, M, probs[b].kernels)
        want = O.convolve_chain(F, None, coeffs=[C, 1.0])   # q = 2 coefficient factors: even, no W (32 kernels)
        for p, o in outs.items():
            errs[p] = max(errs[p], _rel(o[b].double().cpu().numpy(), want))
        del C, want
    print("c3 max-rel errors", errs)
    assert errs["f32"] < 1e-5
    assert errs["split_f16"] < 1e-5
    assert errs["split_bf16"] < 1e-3
