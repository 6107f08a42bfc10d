"""Separable chain tables, the separable convolution and the batched runner
(uneven sizes, chains of 1..16 kernels, CUDA graph) against the FP64 oracle."""
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


def _oracle_chain_coeffs(N, M, kernels):
    C = np.ones((M, N, N), dtype=np.complex128)
    for kp in kernels:
        gx, gy, gt = synth.kernel_factors(N, M, kp)
        C = C * O.coeffs_separable(gx, gy, gt)
    return C


@pytest.mark.parametrize("prec,N,M,k", [("f64", 32, 16, 1), ("f64", 32, 16, 4), ("f32", 64, 32, 7), ("f32", 256, 64, 16)])
def test_separable_tables_and_convolution(se2, prec, N, M, k):
    rng = synth.SplitMix64(777 + k)
    kernels = [synth.draw_kernel(rng) for _ in range(k)]
    kernels = [synth.KernelParams(kp.sigma, kp.sigma_theta, rng.uniform(0, 6.28)) for kp in kernels]
    plan = se2.Plan(N, M, batch=2, precision=prec)
    params = torch.zeros((2, 16, 3), dtype=torch.float64)
    for j, kp in enumerate(kernels):
        params[:, j] = torch.tensor([kp.sigma, kp.sigma_theta, kp.nu], dtype=torch.float64)
    kk = torch.tensor([k, k], dtype=torch.int32)
    tab = se2.separable_tables(plan, params.cuda(), kk.cuda())
    t = tab[0].cpu().numpy().astype(np.complex128)
    H = N // 2 + 1
    tx, ty, tt = t[:H], t[H:H + N], t[H + N:]
    C = tt[:, None, None] * ty[None, :, None] * tx[None, None, :]
    want = _oracle_chain_coeffs(N, M, kernels)[..., :H]
    if (k - 1) % 2:        # W^(k-1) folded in
        want = O.weight_W(N, M)[..., :H] * want
    tol = 1e-12 if prec == "f64" else 2e-6
    assert _rel(C, want) < tol
    npd = np.float64 if prec == "f64" else np.float32
    F = np.stack([synth.sample_bumps(N, M, synth.make_problem(4, b, N, M, n_bumps=5).bumps) for b in range(2)]).astype(npd)
    out = se2.convolve_separable(plan, torch.from_numpy(F).cuda(), tab).double().cpu().numpy()
    Ps = [synth.sample_kernel(N, M, kp) for kp in kernels]
    for b in range(2):
        assert _rel(out[b], O.convolve_chain(F[b].astype(np.float64), Ps)) < (1e-10 if prec == "f64" else 1e-5)


def test_batch_runner_uneven_sizes_graph(se2, tmp_path):
    """A small batch shaped like the batching config (sizes N in {32,64,128},
    M in {16,32}, chains of 1..16 kernels, 3..16 bumps), autotuned, captured
    in a CUDA graph and replayed twice; every problem against the oracle."""
    from paper_2504_05149_gb300.batch import BatchRunner
    rng = synth.SplitMix64(4000)
    shapes, probs = [], []
    for i in range(14):
        N = [32, 64, 128][rng.randint(0, 2)]
        M = [16, 32][rng.randint(0, 1)]
        k = rng.randint(1, 16)
        prob = synth.make_problem(4, i, N, M, n_bumps=rng.randint(3, 16), n_kernels=k)
        shapes.append((N, M))
        probs.append(prob)
    runner = BatchRunner(shapes, cache_path=str(tmp_path / "tune.json"))
    for i, prob in enumerate(probs):
        runner.f_of(i).copy_(torch.from_numpy(synth.sample_bumps(prob.N, prob.M, prob.bumps).astype(np.float32)))
        runner.set_chain(i, [(kp.sigma, kp.sigma_theta, kp.nu) for kp in prob.kernels])
    runner.build_tables()
    runner.tune(reps=1)
    runner.capture()
    for rep in range(2):
        for c in runner.order:
            runner.out[c].zero_()
        runner.replay()
        torch.cuda.synchronize()
        for i, prob in enumerate(probs):
            F = synth.sample_bumps(prob.N, prob.M, prob.bumps).astype(np.float32).astype(np.float64)
            Ps = [synth.sample_kernel(prob.N, prob.M, kp) for kp in prob.kernels]
            want = O.convolve_chain(F, Ps)
            assert _rel(runner.out_of(i).double().cpu().numpy(), want) < 1e-5, (i, prob.N, prob.M, len(prob.kernels))
    assert runner.launches_per_run() > 0
    assert (tmp_path / "tune.json").exists()


def test_batch_runner_c4_classes_with_256x64(se2, tmp_path):
    """The batching config's size classes including N = 256 and M = 64, chains
    of 1..16 kernels: 64 seeded problems drawn as the config draws them, run
    through the batched runner (autotuned, graph-captured), each against the
    FP64 oracle."""
    from paper_2504_05149_gb300.batch import BatchRunner
    rng = synth.SplitMix64(synth.config_seed(4, 0))
    shapes, bumps, chains = [], [], []
    for i in range(64):
        N = [32, 64, 128, 256][rng.randint(0, 3)]
        M = [16, 32, 64][rng.randint(0, 2)]
        k = rng.randint(1, 16)
        nb = rng.randint(3, 16)
        shapes.append((N, M))
        bumps.append(synth.draw_bumps(rng, nb))
        chains.append([synth.draw_kernel(rng) for _ in range(k)])
    assert (256, 64) in shapes and max(len(c) for c in chains) >= 12
    runner = BatchRunner(shapes, cache_path=str(tmp_path / "tune.json"))
    for i in range(64):
        N, M = shapes[i]
        runner.f_of(i).copy_(torch.from_numpy(synth.sample_bumps(N, M, bumps[i]).astype(np.float32)))
        runner.set_chain(i, [(kp.sigma, kp.sigma_theta, kp.nu) for kp in chains[i]])
    runner.build_tables()
    runner.tune(reps=1)
    runner.capture()
    runner.replay()
    torch.cuda.synchronize()
    for i in range(64):
        N, M = shapes[i]
        F = synth.sample_bumps(N, M, bumps[i]).astype(np.float32).astype(np.float64)
        C = _oracle_chain_coeffs(N, M, chains[i])
        want = O.convolve_chain(F, None, coeffs=[C] if len(chains[i]) % 2 else [C, 1.0])
        assert _rel(runner.out_of(i).double().cpu().numpy(), want) < 1e-5, (i, N, M, len(chains[i]))


def test_batch_lanes_give_identical_results_and_tuner_keeps_the_fastest(se2, tmp_path):
    """The classes on 1, 2 and all stream lanes compute the same outputs bit
    for bit (each class runs the same kernels; only their concurrency
    changes); the tuner times the lane counts and keeps the fastest."""
    from paper_2504_05149_gb300.batch import BatchRunner
    rng = synth.SplitMix64(4100)
    shapes = [([32, 64, 128][rng.randint(0, 2)], [16, 32][rng.randint(0, 1)]) for _ in range(24)]
    runner = BatchRunner(shapes, cache_path=str(tmp_path / "tune.json"))
    for i, (N, M) in enumerate(shapes):
        b = synth.draw_bumps(rng, 6)
        runner.f_of(i).copy_(torch.from_numpy(synth.sample_bumps(N, M, b).astype(np.float32)))
        runner.set_chain(i, [(0.03, 0.4, 0.2)] * (1 + i % 3))
    runner.build_tables()
    nc = len(runner.order)
    assert runner.lanes()[0] == 1                      # a new plan runs the classes one after another
    outs = []
    for L in (1, 2, nc):
        cur, lane_of, _ = runner.lanes(L)
        assert cur == min(L, nc) and max(lane_of) == cur - 1 and min(lane_of) == 0
        runner.out_packed.zero_()
        _run_untuned(runner)
        torch.cuda.synchronize()
        outs.append(runner.out_packed.cpu().clone())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    runner.tune(reps=1)
    cur, _, lane_ms = runner.lanes()
    assert 1 in lane_ms and nc in lane_ms
    assert lane_ms[cur] == min(lane_ms.values())
    runner.out_packed.zero_()
    runner.run()
    torch.cuda.synchronize()
    assert torch.equal(runner.out_packed.cpu(), outs[0])


def _run_untuned(runner):
    from paper_2504_05149_gb300 import _check, _ptr, _stream
    _check(runner.lib.se2_batch_convolve_separable(runner._h, _ptr(runner.f_packed), _ptr(runner.tab_packed),
                                                   _ptr(runner.out_packed), _stream(runner.dev)))


def _c4_sample(se2, n, tmp_path, seed_offset=0):
    from paper_2504_05149_gb300.batch import BatchRunner
    rng = synth.SplitMix64(synth.config_seed(4, seed_offset))
    shapes, bumps, chains = [], [], []
    for i in range(n):
        N = [32, 64, 128, 256][rng.randint(0, 3)]
        M = [16, 32, 64][rng.randint(0, 2)]
        k = rng.randint(1, 16)
        nb = rng.randint(3, 16)
        shapes.append((N, M))
        bumps.append(synth.draw_bumps(rng, nb))
        chains.append([synth.draw_kernel(rng) for _ in range(k)])
    runner = BatchRunner(shapes, cache_path=str(tmp_path / "tune.json"), autotune=False)
    for i in range(n):
        N, M = shapes[i]
        runner.f_of(i).copy_(torch.from_numpy(synth.sample_bumps(N, M, bumps[i]).astype(np.float32)))
        runner.set_chain(i, [(kp.sigma, kp.sigma_theta, kp.nu) for kp in chains[i]])
    runner.build_tables()
    return runner, shapes, bumps, chains


def test_one_launch_matches_lanes_bit_for_bit_and_is_one_kernel(se2, tmp_path):
    """The whole batch as one persistent kernel (work list over every class,
    per-problem counters, scratch rings) gives the lane schedule's outputs
    bit for bit, eagerly and from a CUDA graph, as one launch per run; two
    problems are also checked against the FP64 oracle."""
    runner, shapes, bumps, chains = _c4_sample(se2, 96, tmp_path)
    assert len(runner.order) >= 10
    runner.run()
    runner.status()
    torch.cuda.synchronize()
    ref = runner.out_packed.cpu().clone()
    assert runner.one_launch(True)[0]
    for rep in range(2):
        runner.out_packed.zero_()
        n0 = runner.launches()
        runner.run()
        runner.status()
        torch.cuda.synchronize()
        assert runner.launches() - n0 == 1
        assert torch.equal(runner.out_packed.cpu(), ref)
    runner.capture()
    runner.out_packed.zero_()
    runner.replay()
    torch.cuda.synchronize()
    assert runner.launches_per_run() == 1
    assert torch.equal(runner.out_packed.cpu(), ref)
    for i in (0, len(shapes) - 1):
        N, M = shapes[i]
        F = synth.sample_bumps(N, M, bumps[i]).astype(np.float32).astype(np.float64)
        C = _oracle_chain_coeffs(N, M, chains[i])
        want = O.convolve_chain(F, None, coeffs=[C] if len(chains[i]) % 2 else [C, 1.0])
        assert _rel(runner.out_of(i).double().cpu().numpy(), want) < 1e-5
    assert not runner.one_launch(False)[0]


def test_one_launch_bounded_wait_reports_timeout(se2, tmp_path):
    """A wait of the one-launch kernel that can never be met gives up after a
    bounded number of polls; se2_batch_plan_status returns SE2_ERR_TIMEOUT,
    and the plan then runs normally."""
    from paper_2504_05149_gb300 import _ptr, _stream, SE2Error
    runner, _, _, _ = _c4_sample(se2, 12, tmp_path, seed_offset=7)
    runner.run()
    torch.cuda.synchronize()
    ref = runner.out_packed.cpu().clone()
    st = runner.lib.se2_debug_batch_wait_timeout(runner._h, _ptr(runner.f_packed), _ptr(runner.tab_packed),
                                                 _ptr(runner.out_packed), _stream(runner.dev))
    assert st == 0
    with pytest.raises(SE2Error) as ei:
        runner.status()
    assert ei.value.status == 5          # SE2_ERR_TIMEOUT
    runner.status()                      # cleared
    runner.one_launch(True)
    runner.out_packed.zero_()
    runner.run()
    runner.status()
    torch.cuda.synchronize()
    assert torch.equal(runner.out_packed.cpu(), ref)
