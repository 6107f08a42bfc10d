"""Full-size parity in the launch configuration bench.py times: batch 16 of
N = 256, M = 64 problems (16 bumps, one seeded kernel each, FP32), checked on
sampled outputs against the brute-force direct sum of the oracle (computed
one point at a time, independent of any FFT), and one whole problem against
the oracle's FFT route; plus the 8-fold chain shape."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import direct  # noqa: E402
from oracle import se2_oracle as O  # noqa: E402


@pytest.fixture(scope="module")
def se2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_05149_gb300 import build as b
    b.build()
    import paper_2504_05149_gb300 as m
    return m


def test_bench_workload_sampled_direct_sums(se2):
    N, M, B = 256, 64, 16
    Fs, Ps = [], []
    for b in range(B):
        prob = synth.make_problem(2, b, N, M, n_bumps=16, n_kernels=1)
        Fs.append(synth.sample_bumps(N, M, prob.bumps).astype(np.float32))
        Ps.append(synth.sample_kernel(N, M, prob.kernels[0]).astype(np.float32))
    F, P = np.stack(Fs), np.stack(Ps)
    plan = se2.Plan(N, M, batch=B, precision="f32")
    C, _ = se2.coeffs(plan, torch.from_numpy(P).cuda())
    out = se2.convolve(plan, torch.from_numpy(F).cuda(), C).double().cpu().numpy()
    rng = np.random.default_rng(99)
    for b in (0, 7, 15):
        pts = rng.choice(M * N * N, size=48, replace=False)
        want = direct.direct_conv_points(F[b].astype(np.float64), P[b].astype(np.float64), pts)
        got = out[b].reshape(-1)[pts]
        assert np.max(np.abs(got - want)) / np.max(np.abs(out[b])) < 1e-5
        # the peak of the output, where relative accuracy matters most
        peak = np.argmax(np.abs(out[b]).reshape(-1))
        w = direct.direct_conv_points(F[b].astype(np.float64), P[b].astype(np.float64), np.array([peak]))
        assert abs(out[b].reshape(-1)[peak] - w[0]) / abs(w[0]) < 1e-5
    full = O.convolve(F[3].astype(np.float64), P[3].astype(np.float64))
    assert np.max(np.abs(out[3] - full)) / np.max(np.abs(full)) < 1e-5


def test_edge_inputs_zero_constant_and_delta(se2):
    """Degenerate inputs: f = 0 gives 0; a constant f gives the constant times
    the kernel mass (DC bin only); a delta f reproduces the kernel shifted by
    the grid offset (the convolution's identity element check)."""
    N, M = 64, 16
    plan = se2.Plan(N, M, batch=3)
    rng = np.random.default_rng(5)
    P = rng.random((M, N, N)).astype(np.float32)
    F = np.zeros((3, M, N, N), dtype=np.float32)
    F[1] = 2.5
    F[2, 3, 10, 20] = float(N * N * M)          # delta of mass 1 under the rectangle rule
    C, _ = se2.coeffs(plan, torch.from_numpy(np.stack([P] * 3)).cuda())
    out = se2.convolve(plan, torch.from_numpy(F).cuda(), C).double().cpu().numpy()
    assert np.max(np.abs(out[0])) == 0.0
    assert np.allclose(out[1], 2.5 * P.astype(np.float64).mean(), rtol=2e-6, atol=0)
    want = direct.direct_conv_points(F[2].astype(np.float64), P.astype(np.float64), np.arange(M * N * N)).reshape(M, N, N)
    assert np.max(np.abs(out[2] - want)) / np.max(np.abs(want)) < 1e-5
