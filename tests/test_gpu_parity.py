"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs are the seeded synth arrays rounded to the path's real type; the
oracle gets those exact values upcast to FP64.  Errors are normwise:
max-rel = max|gpu - oracle| / max|oracle|.  Bars: 1e-10 (FP64), 1e-5 (FP32).
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import closed_forms as cf  # noqa: E402
from oracle import direct  # noqa: E402
from oracle import se2_oracle as O  # noqa: E402

TOL = {"f32": 1e-5, "f64": 1e-10}
NP = {"f32": np.float32, "f64": np.float64}


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


def _problem(cfg, idx, N, M, nb, kernels):
    prob = synth.make_problem(cfg, idx, N, M, n_bumps=nb)
    F = synth.sample_bumps(N, M, prob.bumps)
    Ps = [synth.sample_kernel(N, M, k) for k in kernels]
    return prob, F, Ps


def _dev(x, prec):
    return torch.from_numpy(np.ascontiguousarray(x.astype(NP[prec]))).cuda()


def _run(se2, prec, F_list, P_lists, normalize=False, flags=0):
    """F_list: B grids; P_lists: B lists of k kernels (or one list if shared)."""
    N, M = F_list[0].shape[1], F_list[0].shape[0]
    B = len(F_list)
    plan = se2.Plan(N, M, batch=B, precision=prec, flags=flags)
    f = _dev(np.stack(F_list), prec)
    k = len(P_lists[0])
    Cs, Ls = [], []
    for i in range(k):
        P = np.stack([pl[i] for pl in P_lists])
        C, ls = se2.coeffs(plan, _dev(P, prec), normalize=normalize)
        Cs.append(C)
        Ls.append(ls)
    out = se2.convolve_chain(plan, f, Cs, Ls if normalize else None)
    torch.cuda.synchronize()
    return out.double().cpu().numpy(), [C.cpu().numpy() for C in Cs], [None if l is None else l.cpu().numpy() for l in Ls]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c1_single_convolution(se2, prec):
    """N=32, M=16, 3 bumps, kernel sigma=0.05, sigma_theta=0.3."""
    N, M = 32, 16
    kp = synth.KernelParams(0.05, 0.3)
    prob, F, (P,) = _problem(1, 0, N, M, 3, [kp])
    F = F.astype(NP[prec]).astype(np.float64)
    P = P.astype(NP[prec]).astype(np.float64)
    out, (C,), _ = _run(se2, prec, [F], [[P]])
    assert _rel(C[0], O.coeffs_half(P)) < TOL[prec]
    want = O.convolve(F, P)
    assert _rel(out[0], want) < TOL[prec]
    # and the brute-force direct sum
    assert _rel(out[0], direct.direct_conv(F, P)) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c1_brute_force_16x16x8(se2, prec):
    N, M = 16, 8
    kp = synth.KernelParams(0.05, 0.3)
    prob, F, (P,) = _problem(1, 0, N, M, 3, [kp])
    F = F.astype(NP[prec]).astype(np.float64)
    P = P.astype(NP[prec]).astype(np.float64)
    out, _, _ = _run(se2, prec, [F], [[P]])
    assert _rel(out[0], direct.direct_conv(F, P)) < TOL[prec]


def test_c2_single_and_8_chain_fp32(se2):
    """N=256, M=64, 16 bumps: single convolution and an 8-fold chain with
    sigma ~ U[.01,.04], sigma_theta ~ U[.1,.5], against the oracle; the chain
    also against the continuous closed form (variances add)."""
    N, M = 256, 64
    prob = synth.make_problem(2, 0, N, M, n_bumps=16, n_kernels=8)
    F = synth.sample_bumps(N, M, prob.bumps).astype(np.float32).astype(np.float64)
    Ps = [synth.sample_kernel(N, M, k).astype(np.float32).astype(np.float64) for k in prob.kernels]
    out1, _, _ = _run(se2, "f32", [F], [[Ps[0]]])
    assert _rel(out1[0], O.convolve(F, Ps[0])) < 1e-5
    out8, _, _ = _run(se2, "f32", [F], [Ps])
    want8 = O.convolve_chain(F, Ps)
    assert _rel(out8[0], want8) < 1e-5
    cont = cf.continuous_output(N, M, prob.bumps, prob.kernels)
    assert _rel(out8[0], cont) < 1e-4     # FP32 rounding of inputs + aliasing


@pytest.mark.parametrize("N,M", [(8, 2), (8, 4), (16, 16), (32, 8), (64, 32), (128, 16), (256, 8),
                                 (512, 8), (32, 128), (128, 128)])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_sizes_random_inputs(se2, N, M, prec):
    """Unstructured inputs over the supported size range (both fused and
    split passes), B = 3 with distinct kernels."""
    rng = np.random.default_rng(N * 1000 + M)
    Fs = [rng.standard_normal((M, N, N)) for _ in range(3)]
    Ps = [[rng.random((M, N, N))] for _ in range(3)]
    Fs = [x.astype(NP[prec]).astype(np.float64) for x in Fs]
    Ps = [[x[0].astype(NP[prec]).astype(np.float64)] for x in Ps]
    out, _, _ = _run(se2, prec, Fs, Ps)
    for b in range(3):
        want = O.convolve(Fs[b], Ps[b][0])
        assert _rel(out[b], want) < TOL[prec] * (3 if prec == "f32" else 1)


def test_largest_size_split_path_fp32(se2):
    N, M = 512, 128
    prob, F, (P,) = _problem(3, 0, N, M, 8, [synth.KernelParams(0.02, 0.3)])
    F = F.astype(np.float32).astype(np.float64)
    P = P.astype(np.float32).astype(np.float64)
    out, _, _ = _run(se2, "f32", [F], [[P]])
    assert _rel(out[0], O.convolve(F, P)) < 1e-5


def test_normalised_coeffs_and_log_scale(se2):
    """se2_coeffs with log_scale: C / mean|P| and ln(mean|P|); the chain
    multiplies back exp(sum ln s) in FP64."""
    N, M = 64, 16
    rng = np.random.default_rng(7)
    F = rng.random((M, N, N))
    Ps = [rng.random((M, N, N)) * s for s in (1e-3, 50.0, 2.0)]
    Fq = F.astype(np.float32).astype(np.float64)
    Pq = [P.astype(np.float32).astype(np.float64) for P in Ps]
    out, Cs, Ls = _run(se2, "f32", [Fq], [Pq], normalize=True)
    for P, C, ls in zip(Pq, Cs, Ls):
        s = np.mean(np.abs(P))
        assert abs(ls[0] - math.log(s)) < 1e-6
        assert _rel(C[0], O.coeffs_half(P) / s) < 1e-5
    assert _rel(out[0], O.convolve_chain(Fq, Pq)) < 1e-5


def test_shared_kernel_flag(se2):
    N, M, B = 64, 32, 4
    rng = np.random.default_rng(11)
    Fs = [rng.standard_normal((M, N, N)).astype(np.float32).astype(np.float64) for _ in range(B)]
    P = rng.random((M, N, N)).astype(np.float32).astype(np.float64)
    plan = se2.Plan(N, M, batch=B, precision="f32", flags=se2.SHARED_KERNEL)
    C, _ = se2.coeffs(plan, _dev(P[None], "f32"))
    out = se2.convolve(plan, _dev(np.stack(Fs), "f32"), C).double().cpu().numpy()
    for b in range(B):
        assert _rel(out[b], O.convolve(Fs[b], P)) < 1e-5


def test_equal_kernels_chain_is_hadamard_power(se2):
    """Algorithm 4 (Hadamard power, W only for odd q) from k equal kernels."""
    N, M = 32, 16
    kp = synth.KernelParams(0.04, 0.4, 0.3)
    prob, F, (P,) = _problem(1, 4, N, M, 3, [kp])
    F = F.astype(np.float32).astype(np.float64)
    P = P.astype(np.float32).astype(np.float64)
    for q in (2, 3, 5):
        out, _, _ = _run(se2, "f32", [F], [[P] * q])
        assert _rel(out[0], O.convolve_power(F, P, q)) < 1e-5


def _sub(env, code):
    r = subprocess.run([sys.executable, "-c", code], env={**os.environ, **env}, capture_output=True, text=True,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


_RAGGED = r"""
import numpy as np, torch, sys
sys.path.insert(0, '.')
import paper_2504_05149_gb300 as se2
from oracle import se2_oracle as O
N, M, B = 64, 16, 5
rng = np.random.default_rng(3)
F = rng.standard_normal((B, M, N, N)).astype(np.float32)
P = rng.random((B, M, N, N)).astype(np.float32)
plan = se2.Plan(N, M, batch=B)
C, _ = se2.coeffs(plan, torch.from_numpy(P).cuda())
out = se2.convolve(plan, torch.from_numpy(F).cuda(), C).double().cpu().numpy()
err = max(np.abs(out[b] - O.convolve(F[b].astype(float), P[b].astype(float))).max()
          / np.abs(O.convolve(F[b].astype(float), P[b].astype(float))).max() for b in range(B))
assert err < 1e-5, err
print("ok", err)
"""


def test_ragged_chunks_and_forced_split_path(se2):
    """B = 5 through a scratch of 2 problems (chunks 2, 2, 1), on the fused
    and on the split pass structure."""
    _sub({"SE2_MAX_CHUNK": "2"}, _RAGGED)
    _sub({"SE2_MAX_CHUNK": "2", "SE2_FORCE_SPLIT": "1"}, _RAGGED)


def test_paired_and_generic_fp32_kernels_agree(se2):
    """The FP32 paired-FFT kernels (default where they exist) and the generic
    kernels (SE2_FAST=0) both give the oracle's result at 256^2 x 64, and at
    128^2 x 128 through ragged scratch chunks."""
    code = _RAGGED.replace("N, M, B = 64, 16, 5", "N, M, B = 256, 64, 3")
    _sub({"SE2_FAST": "0"}, code)
    _sub({}, code)
    code = _RAGGED.replace("N, M, B = 64, 16, 5", "N, M, B = 128, 128, 3")
    _sub({"SE2_MAX_CHUNK": "2"}, code)


@pytest.mark.parametrize("k", [2, 3])
def test_pipelined_chains_with_log_scale(se2, k):
    """Fast path at 256^2 x 64 with B = 5 (pipeline groups 2, 2, 1): chains of
    k distinct kernels (W^k for odd and even k) with normalised spectra and
    FP64 log scales, against the oracle's chain."""
    N, M, B = 256, 64, 5
    Fs, Ps = [], []
    for b in range(B):
        prob = synth.make_problem(2, 700 + 10 * k + b, N, M, n_bumps=16, n_kernels=k)
        Fs.append(synth.sample_bumps(N, M, prob.bumps).astype(np.float32).astype(np.float64))
        # kernel i scaled by 10^(i-1): the log scales carry the magnitudes
        Ps.append([(synth.sample_kernel(N, M, kp) * 10.0 ** (i - 1)).astype(np.float32).astype(np.float64)
                   for i, kp in enumerate(prob.kernels)])
    out, _, Ls = _run(se2, "f32", Fs, Ps, normalize=True)
    for b in range(B):
        assert _rel(out[b], O.convolve_chain(Fs[b], Ps[b])) < 1e-5


def test_pipelined_groups_on_several_streams(se2):
    """FP32 fast path with the batch in groups on 3 streams (ragged last
    group), and the same call captured in a CUDA graph and replayed."""
    code = _RAGGED.replace("N, M, B = 64, 16, 5", "N, M, B = 64, 16, 7")
    _sub({"SE2_PIPE_DEPTH": "3", "SE2_PIPE_GROUP": "2"}, code)
    graph = r"""
import numpy as np, torch, sys
sys.path.insert(0, '.')
import paper_2504_05149_gb300 as se2
from oracle import se2_oracle as O
N, M, B = 32, 8, 6
rng = np.random.default_rng(5)
F = rng.standard_normal((B, M, N, N)).astype(np.float32)
P = rng.random((B, M, N, N)).astype(np.float32)
plan = se2.Plan(N, M, batch=B)
C, _ = se2.coeffs(plan, torch.from_numpy(P).cuda())
f = torch.from_numpy(F).cuda()
out = torch.empty_like(f)
s = torch.cuda.Stream()
s.wait_stream(torch.cuda.current_stream())
with torch.cuda.stream(s):
    se2.convolve(plan, f, C, out=out)
torch.cuda.current_stream().wait_stream(s)
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g):
    se2.convolve(plan, f, C, out=out)
out.zero_()
g.replay()
torch.cuda.synchronize()
got = out.double().cpu().numpy()
err = max(np.abs(got[b] - O.convolve(F[b].astype(float), P[b].astype(float))).max()
          / np.abs(O.convolve(F[b].astype(float), P[b].astype(float))).max() for b in range(B))
assert err < 1e-5, err
print("ok", err)
"""
    _sub({"SE2_PIPE_DEPTH": "2", "SE2_PIPE_GROUP": "2"}, graph)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_convolution(se2, pinned):
    """se2_convolve_host: f and out on the host, groups of 4 through three
    staging slots (B = 9: five groups of at most 2, slots reused)."""
    N, M, B = 64, 16, 9
    rng = np.random.default_rng(13)
    F = rng.standard_normal((B, M, N, N)).astype(np.float32)
    P = rng.random((B, M, N, N)).astype(np.float32)
    plan = se2.Plan(N, M, batch=B, flags=se2.HOST_STAGING)
    C, _ = se2.coeffs(plan, torch.from_numpy(P).cuda())
    hf = torch.from_numpy(F)
    if pinned:
        hf = hf.pin_memory()
    for _ in range(2):   # the second call reuses the staging buffers; no call allocates
        before = se2.alloc_stats()
        out = se2.convolve_host(plan, hf, C).double().numpy()
        assert se2.alloc_stats() == before
        for b in range(B):
            want = O.convolve(F[b].astype(float), P[b].astype(float))
            assert _rel(out[b], want) < 1e-5
    with pytest.raises(se2.SE2Error):   # a plan without the staging flag
        se2.convolve_host(se2.Plan(N, M, batch=B), hf, C)
    import ctypes
    lib = se2.load_library()
    st = lib.se2_convolve_host(plan.handle, ctypes.c_void_p(hf.data_ptr()), 2, ctypes.c_void_p(C.data_ptr()), None,
                               ctypes.c_void_p(hf.data_ptr() + 4), None)
    assert st == 1      # out overlaps f


def test_input_offset_by_one_float(se2):
    """f starting 4 bytes past a 16-byte boundary (a view one float into a
    buffer) still matches the oracle."""
    N, M, B = 64, 16, 3
    rng = np.random.default_rng(17)
    F = rng.standard_normal((B, M, N, N)).astype(np.float32)
    P = rng.random((B, M, N, N)).astype(np.float32)
    plan = se2.Plan(N, M, batch=B)
    C, _ = se2.coeffs(plan, torch.from_numpy(P).cuda())
    big = torch.zeros(F.size + 1, dtype=torch.float32, device="cuda")
    f = big[1:].view(B, M, N, N)
    f.copy_(torch.from_numpy(F))
    assert f.data_ptr() % 16 == 4
    out = se2.convolve(plan, f, C).double().cpu().numpy()
    for b in range(B):
        assert _rel(out[b], O.convolve(F[b].astype(float), P[b].astype(float))) < 1e-5


_ORIGIN = r"""
import numpy as np, torch, sys
sys.path.insert(0, '.')
import paper_2504_05149_gb300 as se2
import synth
from oracle import se2_oracle as O
def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
for N, M, B, k in ((64, 16, 3, 1), (256, 64, 3, 2), (256, 64, 3, 3), (32, 8, 2, 1)):
    plan = se2.Plan(N, M, batch=B, flags=se2.GRID_ORIGIN_ZERO)
    Fs, Ps = [], []
    for b in range(B):
        prob = synth.make_problem(6, 10 * N + b, N, M, n_bumps=6, n_kernels=k)
        Fs.append(synth.sample_bumps(N, M, prob.bumps, origin_zero=True).astype(np.float32))
        Ps.append([synth.sample_kernel(N, M, kp, origin_zero=True).astype(np.float32) for kp in prob.kernels])
    f = torch.from_numpy(np.stack(Fs)).cuda()
    Cs = [se2.coeffs(plan, torch.from_numpy(np.stack([p[i] for p in Ps])).cuda())[0] for i in range(k)]
    out = se2.convolve_chain(plan, f, Cs).double().cpu().numpy()
    for b in range(B):
        want = O.convolve_chain(Fs[b].astype(np.float64), [P.astype(np.float64) for P in Ps[b]], origin_zero=True)
        assert rel(out[b], want) < 1e-5, (N, M, k, rel(out[b], want))
# the adjoint without W
N, M, B = 64, 16, 2
plan = se2.Plan(N, M, batch=B, flags=se2.GRID_ORIGIN_ZERO | se2.SHARED_KERNEL)
P, dPs, dPt = se2.sample_radial_gaussian(plan, 0.04, 0.3, derivs=True)
wP, _, _ = O.kernel_samples_and_derivs(N, M, 0.04, 0.3, origin_zero=True)
assert rel(P[0].double().cpu().numpy(), wP) < 1e-6
C, _ = se2.coeffs(plan, P)
G = np.random.default_rng(3).standard_normal((B, M, N, N)).astype(np.float32)
gf, _ = se2.backward(plan, torch.from_numpy(G).cuda(), C)
for b in range(B):
    want = O.adjoint(G[b].astype(np.float64), [P[0].double().cpu().numpy()], origin_zero=True)
    assert rel(gf[b].double().cpu().numpy(), want) < 1e-5
# separable chain tables sampled at x_i = i/N, no W folded in
N, M, B, k = 64, 32, 2, 3
plan = se2.Plan(N, M, batch=B, flags=se2.GRID_ORIGIN_ZERO)
rng = synth.SplitMix64(91)
kernels = [synth.draw_kernel(rng) for _ in range(k)]
params = torch.zeros((B, 16, 3), dtype=torch.float64)
for j, kp in enumerate(kernels):
    params[:, j] = torch.tensor([kp.sigma, kp.sigma_theta, kp.nu], dtype=torch.float64)
tab = se2.separable_tables(plan, params.cuda(), torch.tensor([k] * B, dtype=torch.int32).cuda())
F = np.stack([synth.sample_bumps(N, M, synth.make_problem(7, b, N, M, n_bumps=4).bumps, origin_zero=True)
              for b in range(B)]).astype(np.float32)
out = se2.convolve_separable(plan, torch.from_numpy(F).cuda(), tab).double().cpu().numpy()
Ps = [synth.sample_kernel(N, M, kp, origin_zero=True) for kp in kernels]
for b in range(B):
    assert rel(out[b], O.convolve_chain(F[b].astype(np.float64), Ps, origin_zero=True)) < 1e-5
print("ok")
"""


def test_grid_origin_zero_flag(se2):
    """SE2_GRID_ORIGIN_ZERO: grids sampled at x_i = i/N, single convolutions
    and chains without W, the sampler on that grid and the adjoint, on the fast
    kernels and (SE2_FAST=0) on the generic ones."""
    _sub({}, _ORIGIN)
    _sub({"SE2_FAST": "0"}, _ORIGIN)


@pytest.mark.parametrize("N,M,B,k,normalize", [(64, 16, 3, 4, False), (256, 64, 2, 3, True), (32, 8, 5, 2, False)])
def test_chain_emit_all_intermediates(se2, N, M, B, k, normalize):
    """se2_convolve_chain_all: V_1..V_k of Algorithm 6 from one forward
    transform, against the oracle's fast recursion (with FP64 log scales in
    one case); B = 5 at 32^2 x 8 runs through scratch groups."""
    Fs, Ps = [], []
    for b in range(B):
        prob = synth.make_problem(8, 100 * N + b, N, M, n_bumps=6, n_kernels=k)
        Fs.append(synth.sample_bumps(N, M, prob.bumps).astype(np.float32).astype(np.float64))
        Ps.append([(synth.sample_kernel(N, M, kp) * (10.0 ** i if normalize else 1.0)).astype(np.float32).astype(np.float64)
                   for i, kp in enumerate(prob.kernels)])
    plan = se2.Plan(N, M, batch=B)
    Cs, Ls = [], []
    for i in range(k):
        C, ls = se2.coeffs(plan, _dev(np.stack([p[i] for p in Ps]), "f32"), normalize=normalize)
        Cs.append(C)
        Ls.append(ls)
    out = se2.convolve_chain_all(plan, _dev(np.stack(Fs), "f32"), Cs, Ls if normalize else None)
    out = out.double().cpu().numpy()
    for b in range(B):
        want = O.convolve_all(Fs[b], Ps[b])
        for p in range(k):
            assert _rel(out[p, b], want[p]) < 1e-5, (b, p)


def test_invalid_arguments_on_gpu_plan(se2):
    plan = se2.Plan(32, 16, batch=2)
    f = torch.zeros((3, 16, 32, 32), device="cuda")
    C = torch.zeros((3, 16, 32, 17), dtype=torch.complex64, device="cuda")
    import ctypes
    lib = se2.load_library()
    # B larger than the plan batch
    st = lib.se2_convolve(plan.handle, ctypes.c_void_p(f.data_ptr()), 3, ctypes.c_void_p(C.data_ptr()), None,
                          ctypes.c_void_p(f.data_ptr() + 4), None)
    assert st == 1
    # misaligned coefficient pointer
    st = lib.se2_convolve(plan.handle, ctypes.c_void_p(f.data_ptr()), 1, ctypes.c_void_p(C.data_ptr() + 4), None,
                          ctypes.c_void_p(f.data_ptr() + 4 * 16 * 32 * 32), None)
    assert st == 1
    # out aliases f
    st = lib.se2_convolve(plan.handle, ctypes.c_void_p(f.data_ptr()), 1, ctypes.c_void_p(C.data_ptr()), None,
                          ctypes.c_void_p(f.data_ptr()), None)
    assert st == 1
    with pytest.raises(ValueError):
        se2.convolve(plan, f[:1].double(), C[:1])


def test_persistent_and_three_kernel_paths_agree(se2):
    """The persistent dataflow kernel (default for FP32 fused sizes) and the
    three-kernel sequence give the oracle's result on B = 7 problems (more
    than the 3 scratch slots, so slots are reused)."""
    code = _RAGGED.replace("N, M, B = 64, 16, 5", "N, M, B = 256, 64, 7")
    _sub({"SE2_PERSIST": "1"}, code)
    _sub({}, code)


def test_bounded_wait_times_out_and_plan_recovers(se2):
    """A dependency nothing satisfies: the kernel's wait gives up, the host
    reads SE2_ERR_TIMEOUT, and the plan then computes correctly again."""
    os.environ["SE2_PERSIST"] = "1"    # read at plan creation
    N, M = 64, 16
    rng = np.random.default_rng(5)
    F = rng.standard_normal((1, M, N, N)).astype(np.float32)
    P = rng.random((1, M, N, N)).astype(np.float32)
    try:
        plan = se2.Plan(N, M, batch=2)
    finally:
        del os.environ["SE2_PERSIST"]
    f = torch.from_numpy(F).cuda()
    C, _ = se2.coeffs(plan, torch.from_numpy(P).cuda())
    out = torch.empty_like(f)
    import ctypes
    lib = se2.load_library()
    st = lib.se2_debug_wait_timeout(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    with pytest.raises(se2.SE2Error) as ei:
        plan.status()
    assert ei.value.status == 5
    plan.status()   # cleared
    out = se2.convolve(plan, f, C)
    plan.status()
    want = O.convolve(F[0].astype(np.float64), P[0].astype(np.float64))
    assert _rel(out[0].double().cpu().numpy(), want) < 1e-5


def test_unit_timing_counts_launches(se2):
    """se2_plan_timing: every unit launch of the FP32 fast path is timed on
    its own stream; counts match the launches and durations are positive."""
    N, M, B = 64, 32, 6
    plan = se2.Plan(N, M, batch=B)
    f = torch.rand((B, M, N, N), device="cuda")
    C, _ = se2.coeffs(plan, torch.rand((B, M, N, N), device="cuda"))
    out = torch.empty_like(f)
    plan.timing(True)
    n0 = plan.launches()
    for _ in range(3):
        se2.convolve(plan, f, C, out=out)
    torch.cuda.synchronize()
    stats = plan.timing_read()
    plan.timing(False)
    launched = plan.launches() - n0
    assert sum(c for _, c in stats) == launched
    assert stats[0][1] == stats[1][1] == stats[2][1] > 0
    assert stats[3][1] == 0     # no whole-batch dataflow launch on this plan
    assert all(ms > 0 for ms, _ in stats[:3])
    plan.timing(True)           # switching on again clears the records
    assert plan.timing_read() == [(0.0, 0)] * 4
    plan.timing(False)


@pytest.mark.parametrize("N,M,k", [(256, 64, 1), (64, 32, 3), (32, 16, 2)])
def test_kernel_ysym_flag_reads_half_the_rows(se2, N, M, k):
    """SE2_KERNEL_YSYM with radial kernels (mirror-symmetric in y on Omega_L):
    the same result as the full read, against the oracle; the rows ky > N/2
    are not read (they are overwritten with NaN here)."""
    B = 2
    kps = [synth.KernelParams(0.02 + 0.01 * i, 0.2 + 0.1 * i, 0.3 * i) for i in range(k)]
    Fs = [synth.sample_bumps(N, M, synth.make_problem(9, b, N, M, n_bumps=4).bumps).astype(np.float32)
          for b in range(B)]
    Ps = [synth.sample_kernel(N, M, kp).astype(np.float32) for kp in kps]
    plan = se2.Plan(N, M, batch=B, flags=se2.KERNEL_YSYM)
    Cs = []
    for P in Ps:
        C, _ = se2.coeffs(plan, _dev(np.stack([P] * B), "f32"))
        C[:, :, N // 2 + 1:, :] = float("nan")
        Cs.append(C)
    out = se2.convolve_chain(plan, _dev(np.stack(Fs), "f32"), Cs).double().cpu().numpy()
    for b in range(B):
        want = O.convolve_chain(Fs[b].astype(np.float64), [P.astype(np.float64) for P in Ps])
        assert _rel(out[b], want) < 1e-5
    # every intermediate of the chain (Algorithm 6) reads the same folded rows
    allv = se2.convolve_chain_all(plan, _dev(np.stack(Fs), "f32"), Cs).double().cpu().numpy()
    for b in range(B):
        wants = O.convolve_all(Fs[b].astype(np.float64), [P.astype(np.float64) for P in Ps])
        for p in range(k):
            assert _rel(allv[p, b], wants[p]) < 1e-5
