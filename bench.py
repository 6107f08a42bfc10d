#!/usr/bin/env python3
"""Throughput of the fast SE(2) convolution (arXiv 2504.05149, Algorithm 3 at
N = L) on GB300: SE(2) convolutions per second at N = 256, M = 64, FP32.

Default arm: a batch of independent problems per GPU (seeded synthetic f1 =
16 bumps; its own radial kernel per problem, whose coefficient spectrum is
computed once by se2_coeffs before timing), one step = one se2_convolve call
over the batch.  Inputs (f, coefficients, out: 808 MB per step) are larger
than L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(numpy FFT route) on the host instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_DEF, M_DEF = 256, 64
B_SINGLE, B_CHAIN = 64, 16   # default batches: single convolutions, 8-fold chains
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=None,
                    help=f"problems per step (default {B_SINGLE} for c2, {B_CHAIN} for c2chain/c2all)")
    ap.add_argument("--N", type=int, default=N_DEF)
    ap.add_argument("--M", type=int, default=M_DEF)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", default="c2", choices=["c2", "c2sep", "c2chain", "c2all", "c3", "c4", "c5", "e4"],
                    help="c2: single convolutions at 256^2x64 (the headline); c2chain: 8-fold chains; "
                         "c2all: 8-fold chains emitting every intermediate (Algorithm 6); "
                         "c4: 4096 uneven problems with separable chains (CUDA graph); c5: forward+adjoint; "
                         "e4: the paper's single-convolution experiment, L = (31, 33, 61) sampled, "
                         "output on 36 x 38 x 76 (grid plan, odd sizes, upsampled)")
    ap.add_argument("--grid-batch", type=int, default=1024, help="e4 batch size")
    ap.add_argument("--ysym", action="store_true",
                    help="c2: declare the (radial) kernel spectra mirror-symmetric in y (SE2_KERNEL_YSYM)")
    ap.add_argument("--problems", type=int, default=4096, help="c4 batch size")
    ap.add_argument("--schedule", default="tuned", choices=["tuned", "lanes", "one"],
                    help="c4: the tuner's choice, or force the lane schedule or the one-launch kernel")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "split_bf16", "split_f16", "bf16"],
                    help="c2: arithmetic of the angular DFT (tensor cores for split_bf16 / split_f16 / bf16)")
    return ap.parse_args()


def rank_problem_ids(rank, B):
    """Seeds of the B problems rank `rank` works on (disjoint across ranks for
    B <= 100): each replica gets its own independent problems (weak scaling)."""
    return [100 * rank + b for b in range(B)]


def aggregate(ms_local, units_per_rank, world, reduce_max=None):
    """Whole-job throughput: units processed by all ranks / the slowest rank's
    time.  reduce_max(float) -> float takes the maximum over ranks (identity
    for one rank)."""
    ms = ms_local if reduce_max is None else reduce_max(ms_local)
    return ms, units_per_rank * world / (ms / 1e3)


def workload_inputs(N, M, B, rank):
    """Seeded synthetic batch: f1 (16 bumps) and one kernel per problem."""
    import synth
    Fs, Ps = [], []
    for b in rank_problem_ids(rank, B):
        prob = synth.make_problem(2, b, N, M, n_bumps=16, n_kernels=1)
        Fs.append(synth.sample_bumps(N, M, prob.bumps).astype(np.float32))
        Ps.append(synth.sample_kernel(N, M, prob.kernels[0]).astype(np.float32))
    return np.stack(Fs), np.stack(Ps)


def peaks():
    try:
        with open(MEASURED) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             + ",".join("clocks_event_reasons." + r for r in REASONS))
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 6 + len(REASONS):
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [p for (t, p) in self.rows if t0 <= t <= t1] or [p for (_, p) in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(p[2]) for p in rows if p[2].replace(".", "").isdigit()]
        mx = [float(p[3]) for p in rows if p[3].replace(".", "").isdigit()]
        reasons = set()
        for p in rows:
            for i, r in enumerate(REASONS):
                if p[6 + i].lower().startswith("active"):
                    reasons.add(r)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def _oracle_worker(args):
    """Convolutions (k = 1) or k-fold chains of the oracle for `seconds` (one
    process; at least one)."""
    N, M, seconds = args[:3]
    k = args[3] if len(args) > 3 else 1
    from oracle import se2_oracle as O
    import synth
    prob = synth.make_problem(2, 0, N, M, n_bumps=16, n_kernels=k)
    F = synth.sample_bumps(N, M, prob.bumps)
    Cs = [O.coeffs_full(synth.sample_kernel(N, M, kp)) for kp in prob.kernels]
    n = 0
    t0 = time.perf_counter()
    while True:
        O.convolve_chain(F, None, coeffs=Cs)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= 64:
            return n, el


def _oracle_adjoint_worker(args):
    """Forward + adjoint steps of the oracle for `seconds` (one process; at
    least one): the convolution with the sampled kernel, the residual, the
    input gradient and the two parameter partials through the kernel
    samples' derivatives.  Returns (steps, seconds)."""
    N, M, seconds = args
    import numpy as np
    from oracle import se2_oracle as O
    import synth
    F = synth.sample_bumps(N, M, synth.make_problem(5, 0, N, M, n_bumps=16).bumps)
    target = np.random.default_rng(5).standard_normal((M, N, N))
    n = 0
    t0 = time.perf_counter()
    while True:
        P, dPs, dPt = O.kernel_samples_and_derivs(N, M, 0.025, 0.25)
        C = O.coeffs_full(P)
        G = O.convolve_chain(F, None, coeffs=[C]) - target
        O.adjoint(G, None, coeffs=[C])
        gk = O.grad_kernel_samples(F, G)
        float((gk * dPs).sum()), float((gk * dPt).sum())
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= 64:
            return n, el


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(N, M, seconds=10.0, k=1, unit="conv/s", procs=None):
    """The FP64 oracle (numpy FFT route, as it stands) on host cores: single
    convolutions (k = 1) or k-fold chains of the same workload with
    precomputed kernel spectra, on one core, then one process per core
    (spawned; `procs` caps the count where one problem needs much memory) for
    the same time."""
    import multiprocessing as mp
    n1, el1 = _oracle_worker((N, M, seconds, k))
    ncores = os.cpu_count() or 1
    np_ = min(ncores, procs) if procs else ncores
    with mp.get_context("spawn").Pool(np_) as pool:
        res = pool.map(_oracle_worker, [(N, M, seconds, k)] * np_)
    total = sum(n / el for n, el in res)
    what = "single convolutions" if k == 1 else f"{k}-fold chains"
    return {"value": total, "unit": unit, "cores": np_, "kind": "oracle", "nproc": ncores,
            "cpu_model": cpu_model(),
            "single_core": {"value": n1 / el1, "unit": unit, "cores": 1},
            "sample": f"numpy FFT route, FP64, precomputed kernel spectra: {n1} {what} N={N} M={M} "
                      f"on one core in {el1:.1f} s; then {np_} spawned processes, one per core, "
                      f"{sum(n for n, _ in res)} in about {seconds:.0f} s"}


METRIC_C2 = "SE(2) convolutions/s at N=256, M=64 (FP32) and fraction of HBM roofline"


def c2_config(N, M, B, world):
    return {"workload": f"se2_convolve, batch of {B} independent problems per GPU, N={N}, M={M}, "
                        f"one radial kernel per problem (precomputed spectra), 16-bump f1",
            "global_batch": B * world, "grid": [M, N, N], "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import se2_oracle as O
    import synth
    N, M = args.N, args.M
    prob = synth.make_problem(2, 0, N, M, n_bumps=16, n_kernels=1)
    F = synth.sample_bumps(N, M, prob.bumps)
    C = O.coeffs_full(synth.sample_kernel(N, M, prob.kernels[0]))
    for _ in range(args.warmup):
        O.convolve_chain(F, None, coeffs=[C])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.convolve_chain(F, None, coeffs=[C])
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {"metric": METRIC_C2, "value": v, "unit": "conv/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**c2_config(N, M, args.batch, 1),
                       "sample": f"one of the {args.batch} problems per step (bounded sample on the host)"},
            "cpu_baseline": {"value": v, "unit": "conv/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} single convolutions, numpy FFT route, FP64"},
            "e2e": {"value": v, "unit": "conv/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.batch is None:
        args.batch = B_CHAIN if args.config in ("c2chain", "c2all") else B_SINGLE
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config != "c2":
        from functools import partial
        {"c2sep": run_separable, "c2chain": run_chain8, "c2all": partial(run_chain8, emit_all=True), "c3": run_precision,
         "c4": run_batch, "c5": run_adjoint, "e4": run_grid_e4}[args.config](args)
        return
    import torch
    import torch.distributed as dist
    import paper_2504_05149_gb300 as se2

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, M, B = args.N, args.M, args.batch
    L = N * N * M

    F, P = workload_inputs(N, M, B, rank)
    if args.precision == "f64":   # the paper's arithmetic, for context
        F, P = F.astype(np.float64), P.astype(np.float64)
    plan = se2.Plan(N, M, batch=B, precision=args.precision, device=local,
                    flags=se2.HOST_STAGING | (se2.KERNEL_YSYM if args.ysym else 0))
    f = torch.from_numpy(F).to(dev)
    C, _ = se2.coeffs(plan, torch.from_numpy(P).to(dev))
    out = torch.empty_like(f)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up, then ~0.5 s more untimed work so the clock sampler sees load
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    sampler = ClockSampler(vis.split(",")[local].strip() if vis else local)
    sampler.start()
    for _ in range(args.warmup):
        se2.convolve(plan, f, C, out=out)
    barrier()
    t_settle = time.time()
    while time.time() - t_settle < 0.6:
        se2.convolve(plan, f, C, out=out)
        torch.cuda.synchronize(dev)

    barrier()
    t_wall0 = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = plan.launches()
    e0.record(stream)
    for _ in range(args.steps):
        se2.convolve(plan, f, C, out=out)
    e1.record(stream)
    launches_timed = plan.launches() - launches0
    barrier()
    t_wall1 = time.time()
    ms = e0.elapsed_time(e1)
    sampler.stop()
    clocks = sampler.summary(t_settle, t_wall1)

    def reduce_max(v):
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms, value = aggregate(ms, B * args.steps, world, reduce_max)
    ms_step = ms / args.steps

    # per-kernel launch durations, live: a second pass of the same steps with
    # CUDA events around every unit launch, recorded by the library on the
    # stream each launch runs on (FP32 fast path only).  In the pipeline two
    # streams overlap, so these durations include the neighbour's contention.
    plan.timing(True)
    for _ in range(args.steps):
        se2.convolve(plan, f, C, out=out)
    torch.cuda.synchronize(dev)
    unit_stats = plan.timing_read()
    plan.timing(False)
    # the same launches serialised (one stream, groups of 2 problems as in the
    # pipeline): each kernel's own duration, the per-kernel roofline
    splan = plan_with_env(se2, {"SE2_PIPE_DEPTH": "1", "SE2_MAX_CHUNK": "2"}, N, M, B, args.precision, local,
                          se2.KERNEL_YSYM if args.ysym else 0)
    for _ in range(2):
        se2.convolve(splan, f, C, out=out)
    ns = max(3, min(args.steps, 10))
    splan.timing(True)
    for _ in range(ns):
        se2.convolve(splan, f, C, out=out)
    torch.cuda.synchronize(dev)
    unit_stats_serial = splan.timing_read()
    splan.timing(False)
    splan.close()
    se2.convolve(plan, f, C, out=out)
    out0 = out[0].double().cpu().numpy()

    # end to end through the public API with host buffers (se2_convolve_host):
    # pinned host f -> device, convolve, device -> host out, overlapped by groups
    hf = torch.from_numpy(F).pin_memory()
    hout = torch.empty(F.shape, dtype=torch.float64 if args.precision == "f64" else torch.float32).pin_memory()
    for _ in range(2):
        se2.convolve_host(plan, hf, C, out=hout)
    barrier()
    # the host link's throughput varies from run to run: the median
    # of three timed repetitions of ke steps
    ke = max(3, min(args.steps, 10))
    reps = []
    for _ in range(3):
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(ke):
            se2.convolve_host(plan, hf, C, out=hout)
        e3.record(stream)
        barrier()
        reps.append(e2.elapsed_time(e3))
    _, e2e_val = aggregate(sorted(reps)[1], B * ke, world, reduce_max)
    assert np.isfinite(hout.numpy()).all()
    link = host_link_rate(torch, stream, hf, f, out, hout)

    # comparator (context only, not the product): the same convolution written
    # with torch.fft (cuFFT) on the same batch: irfftn(W . rfftn(f) . C)
    comp = None
    if args.precision == "f32":
        ky = torch.arange(N, device=dev)
        kx = torch.arange(N // 2 + 1, device=dev)
        W = torch.where(((ky[:, None] + kx[None, :]) % 2) == 1, -1.0, 1.0).to(torch.complex64)

        def torch_fft_step():
            H = torch.fft.rfftn(f, dim=(-3, -2, -1)) * C * W
            return torch.fft.irfftn(H, s=(M, N, N), dim=(-3, -2, -1))

        ref_out = torch_fft_step()
        se2.convolve(plan, f, C, out=out)
        torch.cuda.synchronize(dev)
        agree = float((ref_out - out).abs().max() / ref_out.abs().max())
        for _ in range(3):
            torch_fft_step()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        for _ in range(args.steps):
            torch_fft_step()
        e5.record(stream)
        torch.cuda.synchronize(dev)
        comp = {"torch_fft": {"value": B * args.steps / (e4.elapsed_time(e5) / 1e3), "unit": "conv/s",
                              "what": "torch.fft.rfftn/irfftn (cuFFT) pipeline on the same batch, "
                                      "a comparator for context, not the product",
                              "max_rel_diff_vs_se2": agree}}

    # mixed precision against plain FP32 on the same batch: conv/s and max-rel
    # error against the FP64 oracle on problem 0
    mixed = None
    if args.precision == "f32" and rank == 0 and world == 1:
        mixed = mixed_vs_fp32(se2, torch, dev, stream, N, M, B, F, P, f, value, out0, args)

    hbm, src = peaks()
    c_rows = N // 2 + 1 if args.ysym else N                        # kernel-spectrum rows read per problem
    re = 8 if args.precision == "f64" else 4                          # bytes per real value
    alg_bytes = B * (2 * re * L + 2 * re * M * c_rows * (N // 2 + 1))  # read f, write out, read the spectrum
    achieved = alg_bytes / (ms_step / 1e3) / 1e9

    line = None
    if rank == 0:
        base = None if args.no_cpu_baseline or world > 1 else cpu_baseline(N, M)
        line = {
            "metric": METRIC_C2,
            "value": value, "unit": "conv/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision if args.precision in ("f32", "f64") else
                     f"f32 storage, {args.precision} tensor-core angular DFT",
            "data": "synthetic",
            "config": {**c2_config(N, M, B, world),
                       "l2": f"inputs larger than L2 ({alg_bytes / 1e6:.0f} MB moved per step)"},
            "roofline": kernel_roofline(unit_stats_serial, N, M, B, ns, hbm, src, achieved, alg_bytes,
                                        args.precision, c_rows, overlapped=(unit_stats, args.steps)),
            "mixed_vs_fp32": mixed,
            "cpu_baseline": base,
            "e2e": {"value": e2e_val, "unit": "conv/s", "h2d_bytes_per_step": int(F.nbytes),
                    "d2h_bytes_per_step": int(F.nbytes),
                    "host_link": {"achieved_GBps": e2e_val / B * 2 * F.nbytes / 1e9,
                                  "copy_GBps": link, "frac": e2e_val / B * 2 * F.nbytes / 1e9 / link,
                                  "what": "host<->device bytes of the e2e run per second, against plain "
                                          "cudaMemcpyAsync of the same buffers, both directions at once"}},
            "gpu_launches": launches_timed,
            "comparators": comp,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def plan_with_env(se2, env, N, M, B, precision, device, flags):
    """A plan created with the given environment settings (read at creation)."""
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return se2.Plan(N, M, batch=B, precision=precision, device=device, flags=flags)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


MIXED_BAR = 1e-5   # the accuracy at which mixed precision is compared with FP32


def mixed_vs_fp32(se2, torch, dev, stream, N, M, B, F, P, f, f32_value, f32_out0, args):
    """The tensor-core angular DFT modes (split fp16, split bf16: FP32 storage,
    hi + lo operands, FP32 accumulation) against the plain FP32 path on the
    same batch: conv/s, and max-rel error of problem 0 against the FP64
    oracle; the fastest mode within MIXED_BAR is compared with FP32."""
    from oracle import se2_oracle as O
    want = O.convolve_chain(F[0].astype(np.float64), None, coeffs=[O.coeffs_full(P[0].astype(np.float64))])

    def err(o):
        return float(np.max(np.abs(o - want)) / np.max(np.abs(want)))

    modes = {"f32": {"value": f32_value, "unit": "conv/s", "max_rel_err": err(f32_out0)}}
    km = max(3, min(args.steps, 5))
    for prec in ("split_f16", "split_bf16"):
        try:
            plan = se2.Plan(N, M, batch=B, precision=prec, device=dev.index or 0)
        except se2.SE2Error as ex:   # the tensor-core angular DFT exists for M = 64 and 128
            modes[prec] = {"unsupported": str(ex)}
            continue
        Cm, _ = se2.coeffs(plan, torch.from_numpy(P).to(dev))
        outm = torch.empty_like(f)
        for _ in range(2):
            se2.convolve(plan, f, Cm, out=outm)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(km):
            se2.convolve(plan, f, Cm, out=outm)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        plan.status()
        modes[prec] = {"value": B * km / (e0.elapsed_time(e1) / 1e3), "unit": "conv/s",
                       "max_rel_err": err(outm[0].double().cpu().numpy())}
        plan.close()
    within = [m for m in modes if m != "f32" and modes[m].get("max_rel_err", np.inf) <= MIXED_BAR]
    best = max(within, key=lambda m: modes[m]["value"]) if within else None
    return {**modes, "accuracy_bar": MIXED_BAR, "fastest_mixed_within_bar": best,
            "mixed_beats_fp32": bool(best is not None and modes[best]["value"] > f32_value),
            "what": f"split_f16 / split_bf16: tensor-core (tcgen05) angular DFT with hi + lo operands; "
                    f"{km} timed steps of the same batch; errors of problem 0 against the FP64 oracle"}


# DRAM bytes of the FP32 paired kernels at 256^2 x 64 per launch (2 problems):
# dram__bytes_read.sum + dram__bytes_write.sum of kf_fwd_xt, kf_lines and
# kf_inv_tx, means over 8 launches of one one-pass ncu capture of the current
# kernels (profiles/kf_units_f32_256x256x64_b16_dram_cold_warm.md).  ncu
# flushes the caches before each kernel, so the scratch that the live run
# keeps in L2 is counted as DRAM traffic: an upper bound.  None where the
# kernel has changed since the capture.
NCU_TRAFFIC_PER_LAUNCH = {(256, 64, "f32"): ((33.603232 + 0.051648) * 1e6, (71.606432 + 0.042944) * 1e6,
                                             (37.783840 + 0.013664) * 1e6)}
NCU_TRAFFIC_PER_CONV = {k: (None if any(x is None for x in v) else sum(v) / 2) for k, v in NCU_TRAFFIC_PER_LAUNCH.items()}
# The same counters with the cache left warm (`ncu --cache-control none`, same
# capture): the scratch stays in L2 as in the live run, so this is the
# live-like figure.
NCU_TRAFFIC_WARM_PER_LAUNCH = {(256, 64, "f32"): ((33.772224 + 27.140896) * 1e6, (36.260768 + 6.264480) * 1e6,
                                                  (0.023904 + 30.791264) * 1e6)}
UNIT_NAMES = ("kf_fwd_xt", "kf_lines", "kf_inv_tx")


def host_link_rate(torch, stream, hf, f, out, hout, reps=3):
    """GB/s of the host link for the e2e traffic: pinned hf -> device f and
    device out -> pinned hout as plain copies on two streams at once (median
    of `reps`).  Both copies rewrite data that is already there."""
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    times = []
    for _ in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        with torch.cuda.stream(s_in):
            f.copy_(hf, non_blocking=True)
        with torch.cuda.stream(s_out):
            hout.copy_(out, non_blocking=True)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sorted(times[1:])[len(times[1:]) // 2]
    return (hf.numel() * hf.element_size() + out.numel() * out.element_size()) / (ms / 1e3) / 1e9


def kernel_roofline(unit_stats, N, M, B, steps, hbm, src, step_achieved, step_bytes, precision, c_rows=None,
                    overlapped=None):
    """Roofline of the dominant kernel from per-launch durations of a
    serialised pass (each kernel alone on the GPU); `overlapped` = (stats,
    steps) of the pipelined pass, reported beside them.  Algorithmic bytes
    per problem: kf_fwd_xt reads f (4|L|), kf_lines reads the kernel spectrum
    (8 M N (N/2+1)), kf_inv_tx writes out (4|L|); the scratch between them is
    not algorithmic."""
    L = N * N * M
    step = {"scope": "whole se2_convolve step (all kernels)", "achieved": step_achieved,
            "frac": step_achieved / hbm, "alg_bytes_per_conv": step_bytes / B, **traffic_fields(N, M, precision)}
    per_problem = (4 * L, 8 * M * (N if c_rows is None else c_rows) * (N // 2 + 1), 4 * L)
    kern = []
    for name, bpp, (tms, cnt) in zip(UNIT_NAMES, per_problem, unit_stats):
        if cnt == 0:
            continue
        ppl = B * steps / cnt
        avg = tms / cnt
        ach = bpp * ppl / (avg / 1e3) / 1e9
        kern.append({"kernel": name, "launches": cnt, "avg_launch_ms": avg, "total_ms": tms,
                     "problems_per_launch": ppl, "alg_bytes_per_launch": bpp * ppl, "achieved": ach,
                     "frac": ach / hbm})
    over = []
    if overlapped is not None:
        ostats, osteps = overlapped
        for name, bpp, (tms, cnt) in zip(UNIT_NAMES, per_problem, ostats):
            if cnt:
                ppl = B * osteps / cnt
                over.append({"kernel": name, "launches": cnt, "avg_launch_ms": tms / cnt,
                             "frac": bpp * ppl / (tms / cnt / 1e3) / 1e9 / hbm})
    if not kern:   # not the FP32 fast path: the whole step only
        return {"bound": "hbm", "achieved": step_achieved, "peak": hbm, "unit": "GB/s",
                "frac": step_achieved / hbm, "peak_source": src, **step}
    dom = max(kern, key=lambda d: d["total_ms"])
    tr = NCU_TRAFFIC_PER_LAUNCH.get((N, M, precision))
    ti = UNIT_NAMES.index(dom["kernel"])
    same = abs(dom["problems_per_launch"] - 2) < 1e-9 and c_rows in (None, N)
    traffic = tr[ti] if (tr is not None and same) else None
    tw = NCU_TRAFFIC_WARM_PER_LAUNCH.get((N, M, precision))
    warm = tw[ti] if (tw is not None and same) else None
    return {"bound": "hbm", "achieved": dom["achieved"], "peak": hbm, "unit": "GB/s", "frac": dom["frac"],
            "peak_source": src, "kernel": dom["kernel"], "avg_launch_ms": dom["avg_launch_ms"],
            "alg_bytes_per_launch": dom["alg_bytes_per_launch"], "traffic": traffic,
            "traffic_source": "ncu one-pass dram counters, caches flushed (upper bound), per launch of 2 problems; "
                              "profiles/kf_units_f32_256x256x64_b16_dram_cold_warm.md",
            "traffic_warm_cache": warm,
            "traffic_warm_cache_source": "ncu --cache-control none (L2 as the previous launch left it), per launch of "
                                         "2 problems; profiles/kf_units_f32_256x256x64_b16_dram_cold_warm.md",
            "timing": "CUDA events around each launch, serialised pass (one stream, 2 problems per launch, "
                      "no other kernel running); the pipelined step is roofline.step",
            "kernels": kern, "kernels_overlapped": over, "step": step}


def traffic_fields(N, M, precision):
    t = NCU_TRAFFIC_PER_CONV.get((N, M, precision))
    if t is None:
        return {"traffic": None}
    tw = NCU_TRAFFIC_WARM_PER_LAUNCH.get((N, M, precision))
    return {"traffic": t, "traffic_unit": "bytes per convolution",
            "traffic_source": "ncu one-pass dram counters, caches flushed per kernel (upper bound); "
                              "profiles/kf_units_f32_256x256x64_b16_dram_cold_warm.md",
            "traffic_warm_cache": None if tw is None else sum(tw) / 2,
            "traffic_warm_cache_source": "ncu --cache-control none; "
                                         "profiles/kf_units_f32_256x256x64_b16_dram_cold_warm.md"}


def _clock_and_time(fn, steps, warmup, dev, settle=0.6, plans=()):
    """Warm up, settle ~0.6 s under load (clock sampling), then time `steps`
    calls of fn with CUDA events on the current stream.  Returns (ms, clocks,
    kernels the given plans launched in the timed region)."""
    import torch
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    sampler = ClockSampler(vis.split(",")[dev.index or 0].strip() if vis else (dev.index or 0))
    sampler.start()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    t0 = time.time()
    while time.time() - t0 < settle:
        fn()
        torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sum(p.launches() for p in plans)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    launched = sum(p.launches() for p in plans) - l0
    torch.cuda.synchronize(dev)
    t1 = time.time()
    sampler.stop()
    return e0.elapsed_time(e1), sampler.summary(t0, t1), launched


def _line(metric, value, unit, args, ms, cfg, extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
         "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
         "dtype": "f32", "data": "synthetic", "config": cfg}
    d.update(extra)
    print(json.dumps(d), flush=True)


def run_chain8(args, emit_all=False):
    """8-fold chains f * rho_1 * ... * rho_8 at 256^2 x 64 (the chain's second
    config), one chain of distinct kernels per problem; with emit_all every
    intermediate V_1..V_8 (Algorithm 6) is written."""
    import torch
    import paper_2504_05149_gb300 as se2
    import synth
    N, M, B, k = args.N, args.M, args.batch, 8
    dev = torch.device("cuda", 0)
    plan = se2.Plan(N, M, batch=B)
    Fs, Cs = [], [[] for _ in range(k)]
    for b in range(B):
        prob = synth.make_problem(2, 500 + b, N, M, n_bumps=16, n_kernels=k)
        Fs.append(torch.from_numpy(synth.sample_bumps(N, M, prob.bumps).astype(np.float32)))
        for i, kp in enumerate(prob.kernels):
            Cs[i].append(torch.from_numpy(synth.sample_kernel(N, M, kp).astype(np.float32)))
    f = torch.stack(Fs).to(dev)
    C = [se2.coeffs(plan, torch.stack(c).to(dev))[0] for c in Cs]
    L = N * N * M
    if emit_all:
        out = torch.empty((k,) + tuple(f.shape), dtype=f.dtype, device=dev)
        fn = lambda: se2.convolve_chain_all(plan, f, C, out=out)                  # noqa: E731
        alg = B * (4 * L + k * (4 * L + 8 * M * N * (N // 2 + 1)))                # read f; per step read C_p, write V_p
        metric, what = "8-fold SE(2) convolution chains/s with all 8 intermediates at N=256, M=64 (FP32)", \
            f"se2_convolve_chain_all k=8 distinct kernels, V_1..V_8 written, batch {B}"
    else:
        out = torch.empty_like(f)
        fn = lambda: se2.convolve_chain(plan, f, C, out=out)                      # noqa: E731
        alg = B * (8 * L + k * 8 * M * N * (N // 2 + 1))
        metric, what = "8-fold SE(2) convolution chains/s at N=256, M=64 (FP32)", \
            f"se2_convolve_chain k=8 distinct kernels, batch {B}"
    ms, clocks, launched = _clock_and_time(fn, args.steps, args.warmup, dev, plans=(plan,))
    hbm, src = peaks()
    ach = alg / (ms / args.steps / 1e3) / 1e9
    # the oracle computes the final chain; emit-all adds only writes of V_p
    cpu = None if args.no_cpu_baseline else cpu_baseline(N, M, k=k, unit="chain/s")
    _line(metric, B * args.steps / (ms / 1e3), "chain/s", args, ms,
          {"workload": what, "grid": [M, N, N]},
          {"roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                        "traffic": None, "peak_source": src, "alg_bytes_per_chain": alg / B},
           "cpu_baseline": cpu, "gpu_launches": launched, "clocks": clocks})


def run_separable(args):
    """The separable-kernel path at 256^2 x 64: each problem's chain of 8
    radial kernels (Gaussian x wrapped normal) kept as three 1-D tables, so
    the step moves only f in and out back (8 B per point)."""
    import torch
    import paper_2504_05149_gb300 as se2
    import synth
    N, M, B, k = args.N, args.M, args.batch, 8
    dev = torch.device("cuda", 0)
    plan = se2.Plan(N, M, batch=B)
    params = torch.zeros((B, 16, 3), dtype=torch.float64)
    Fs = []
    for b in range(B):
        prob = synth.make_problem(2, 700 + b, N, M, n_bumps=16, n_kernels=k)
        Fs.append(torch.from_numpy(synth.sample_bumps(N, M, prob.bumps).astype(np.float32)))
        for j, kp in enumerate(prob.kernels):
            params[b, j] = torch.tensor([kp.sigma, kp.sigma_theta, kp.nu], dtype=torch.float64)
    f = torch.stack(Fs).to(dev)
    tab = se2.separable_tables(plan, params.to(dev), torch.full((B,), k, dtype=torch.int32, device=dev))
    out = torch.empty_like(f)
    fn = lambda: se2.convolve_separable(plan, f, tab, out)                        # noqa: E731
    ms, clocks, launched = _clock_and_time(fn, args.steps, args.warmup, dev, plans=(plan,))
    plan.status()
    hbm, src = peaks()
    L = N * N * M
    alg = B * 8 * L
    ach = alg / (ms / args.steps / 1e3) / 1e9
    cpu = None if args.no_cpu_baseline else cpu_baseline(N, M, k=k, unit="conv/s")
    _line("SE(2) convolutions/s at N=256, M=64 with an 8-fold separable kernel chain (FP32)",
          B * args.steps / (ms / 1e3), "conv/s", args, ms,
          {"workload": f"se2_convolve_separable, batch {B}, 8-kernel chain per problem as three 1-D tables",
           "grid": [M, N, N], "l2": f"inputs larger than L2 ({alg / 1e6:.0f} MB moved per step)"},
          {"roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                        "traffic": None, "peak_source": src, "alg_bytes_per_conv": 8 * L},
           "cpu_baseline": cpu, "gpu_launches": launched, "clocks": clocks})


def grid_flops(L, N, k=1):
    """Real flops of the six direct-DFT passes of one grid-plan convolution
    (a complex multiply-add counts 8, a real-by-complex or real-part one 4)."""
    (Lx, Ly, Lr), (Nx, Ny, Nr) = L, N
    Hx = (Lx - 1) // 2 + 1
    return (4 * Lr * Ly * Hx * Lx + 8 * Lr * Hx * Ly * Ly + 8 * Ly * Hx * Lr * Lr
            + 8 * Ly * Hx * Nr * Lr + 6 * k * Lr * Ly * Hx + 8 * Nr * Hx * Ny * Ly + 4 * Nr * Ny * Hx * Nx)


def alu_peak_f32(sm_mhz):
    """FP32 FMA peak: 152 SMs x 128 lanes x 2 flops per cycle at the given clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def run_grid_e4(args):
    """The paper's single-convolution experiment (Section 6.2): f = f_H^{nu,s}
    with H = diag(0.03, 0.01)^-1, rho = f_U^{nu,s} with U = (1/0.02) I,
    s = 0.01, nu = pi/2, sampled on L = (31, 33, 61) and evaluated on a
    36 x 38 x 76 grid; a batch of such problems (amplitudes vary) through one
    grid plan, FP32."""
    import math
    import torch
    import paper_2504_05149_gb300 as se2
    L, N, B = (31, 33, 61), (36, 38, 76), args.grid_batch
    dev = torch.device("cuda", 0)
    plan = se2.GridPlan(L, N, batch=B, precision="f32", flags=se2.SHARED_KERNEL)

    def deformed(Hd, nu, s):
        x = -0.5 + np.arange(L[0]) / L[0]
        y = -0.5 + np.arange(L[1]) / L[1]
        t = 2 * np.pi * np.arange(L[2]) / L[2]
        Y, X = np.meshgrid(y, x, indexing="ij")
        sp = np.exp(-(Hd[0] * X * X + Hd[1] * Y * Y))
        return (np.exp(-((t - nu) ** 2) / s)[:, None, None] * sp[None]).astype(np.float32)

    F = torch.from_numpy(deformed((1 / 0.03, 1 / 0.01), math.pi / 2, 0.01))
    P = torch.from_numpy(deformed((1 / 0.02, 1 / 0.02), math.pi / 2, 0.01))
    amp = torch.linspace(0.5, 1.5, B).view(B, 1, 1, 1)
    f = (F[None] * amp).contiguous().to(dev)
    C = se2.grid_coeffs(plan, P[None].contiguous().to(dev))
    out = torch.empty(plan.out_shape(B), dtype=torch.float32, device=dev)
    fn = lambda: se2.grid_convolve_chain(plan, f, [C], out=out)                 # noqa: E731
    ms, clocks, launched = _clock_and_time(fn, args.steps, args.warmup, dev, plans=(plan,))
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import se2_upsample as U
        Fd, Pd = F.double().numpy(), P.double().numpy()
        n, t0 = 0, time.time()
        while time.time() - t0 < 3.0:
            U.series(Fd, [Pd], (N[2], N[1], N[0]))
            n += 1
        el = time.time() - t0
        cpu = {"value": n / el, "unit": "conv/s", "cores": torch.get_num_threads(), "kind": "oracle",
               "sample": f"{n} single convolutions over {el:.1f} s, series definition (numpy einsum), FP64"}
    fl = grid_flops(L, N) * B
    ach = fl / (ms / args.steps / 1e3) / 1e12
    mhz = clocks.get("sm_mhz") or 2070
    peak = alu_peak_f32(mhz)
    in_bytes = 4 * B * L[0] * L[1] * L[2]
    out_bytes = 4 * B * N[0] * N[1] * N[2]
    _line("SE(2) convolutions/s, the paper's single-convolution experiment (L=(31,33,61) -> 36x38x76, FP32)",
          B * args.steps / (ms / 1e3), "conv/s", args, ms,
          {"workload": f"grid plan, f_H and radial f_U deformed Gaussians, batch {B}, shared kernel",
           "L": list(L), "N": list(N), "l2": f"inputs {in_bytes / 1e6:.0f} MB + outputs {out_bytes / 1e6:.0f} MB "
                                            "per step, larger than L2"},
          {"roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                        "traffic": None, "peak_source": f"152 SMs x 128 FP32 lanes x 2 flops at {mhz:.0f} MHz",
                        "flops_per_conv": grid_flops(L, N)},
           "paper_context": "0.0849 s per convolution for the FFT scheme with upsampling (MATLAB, the paper's "
                            "hardware, not stated); brute-force quadrature 6.8638e3 s",
           "cpu_baseline": cpu, "gpu_launches": launched, "clocks": clocks})


def run_batch(args):
    """4096 independent problems of uneven size (N in {32,64,128,256}, M in
    {16,32,64}), each with a chain of k ~ U{1..16} separable radial kernels,
    as one CUDA graph of per-class launches."""
    import torch
    import synth
    from paper_2504_05149_gb300.batch import BatchRunner
    dev = torch.device("cuda", 0)
    rng = synth.SplitMix64(synth.config_seed(4, 0))
    shapes, chains, bumps = [], [], []
    for i in range(args.problems):
        N = [32, 64, 128, 256][rng.randint(0, 3)]
        M = [16, 32, 64][rng.randint(0, 2)]
        k = rng.randint(1, 16)
        nb = rng.randint(3, 16)
        shapes.append((N, M))
        bumps.append(synth.draw_bumps(rng, nb))
        chains.append([synth.draw_kernel(rng) for _ in range(k)])
    runner = BatchRunner(shapes, device=0)
    for i in range(args.problems):
        N, M = shapes[i]
        runner.f_of(i).copy_(synth.sample_bumps_torch(N, M, bumps[i], dev, torch.float32))
        runner.set_chain(i, [(kp.sigma, kp.sigma_theta, kp.nu) for kp in chains[i]])
    runner.build_tables()
    runner.tune()
    if args.schedule != "tuned":
        runner.one_launch(args.schedule == "one")
    lanes, lane_of, lane_ms = runner.lanes()
    one_on, one_ms = runner.one_launch()
    runner.capture()
    ms, clocks, _ = _clock_and_time(runner.replay, args.steps, args.warmup, dev)
    pts = runner.points()
    hbm, src = peaks()
    alg = 8 * pts                                     # read f, write out (factored coefficients)
    ach = alg / (ms / args.steps / 1e3) / 1e9
    _line(f"SE(2) convolutions/s, {args.problems} uneven problems with separable kernel chains (FP32)",
          args.problems * args.steps / (ms / 1e3), "conv/s", args, ms,
          {"workload": f"{args.problems} problems, N~U{{32,64,128,256}}, M~U{{16,32,64}}, chains k~U{{1..16}}, 3..16 bumps; "
                       "per-size-class plans on tuned stream lanes or one persistent launch, in one CUDA graph",
                       "points_per_step": pts,
           "classes": {f"{N}x{M}": [len(v), runner.config[(N, M)][0], runner.config[(N, M)][1]]
                       for (N, M), v in runner.classes.items()},
           "lanes": lanes, "tuned_ms_by_lanes": {str(L): round(v, 4) for L, v in lane_ms.items()},
           "schedule": "one persistent launch" if one_on else f"{lanes} stream lane(s)",
           "one_launch_tuned_ms": round(one_ms, 4)},
          {"points_per_s": pts * args.steps / (ms / 1e3),
           "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                        "traffic": None, "peak_source": src, "alg_bytes_per_step": alg},
           "gpu_launches": runner.launches_per_run() * args.steps, "clocks": clocks})


def run_precision(args):
    """Precision config: N=512, M=128, batch 8, 32-bump f1 with amplitudes
    log-uniform in [1e-6, 1], a 32-fold separable kernel chain per problem;
    split-bf16 tensor-core angular DFT vs the plain FP32 path, both timed,
    max-rel error of each against the FP64 oracle on problem 0."""
    import torch
    import paper_2504_05149_gb300 as se2
    import synth
    from oracle import se2_oracle as O
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
    res = {}
    for prec in ("split_bf16", "split_f16", "f32"):
        plan = se2.Plan(N, M, batch=B, precision=prec)
        tab = se2.separable_tables(plan, params, kk)
        out = torch.empty_like(f)
        ms, clocks, launched = _clock_and_time(lambda: se2.convolve_separable(plan, f, tab, out), args.steps,
                                               args.warmup, dev, plans=(plan,))
        plan.status()
        res[prec] = (B * args.steps / (ms / 1e3), ms, out[0].double().cpu().numpy(), clocks, launched)
        plan.close()
    F0 = f[0].double().cpu().numpy()
    coeffs = []
    for kp in probs[0].kernels:
        gx, gy, gt = synth.kernel_factors(N, M, kp)
        coeffs.append(O.coeffs_separable(gx, gy, gt))
    t0 = time.perf_counter()
    want = O.convolve_chain(F0, None, coeffs=coeffs)
    el = time.perf_counter() - t0
    # one core only: the 32 full FP64 spectra of one problem take 17 GB, too
    # many for a process per core
    cpu = {"value": 1.0 / el, "unit": "conv/s", "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"one 32-fold chain of problem 0 (N={N}, M={M}, precomputed separable spectra), numpy FFT "
                     f"route, FP64, {el:.1f} s on one core"}
    err = {p: float(np.max(np.abs(res[p][2] - want)) / np.max(np.abs(want))) for p in res}
    v, ms, _, clocks, launched = res["split_bf16"]
    _line("SE(2) convolutions/s at N=512, M=128, 32-fold chain: split-bf16 tensor-core angular DFT",
          v, "conv/s", args, ms,
          {"workload": "batch 8, 32-bump f1 with amplitudes log-uniform in [1e-6, 1], 32-fold separable chain",
           "grid": [M, N, N]},
          {"fp32_value": res["f32"][0], "split_f16_value": res["split_f16"][0], "max_rel_err_vs_fp64_oracle": err,
           "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": launched})


def run_adjoint(args):
    """Differentiation config: forward + adjoint (grad f, grad sigma, grad
    sigma_theta) at 256^2 x 64, batch 64, shared kernel, FP32."""
    import torch
    import paper_2504_05149_gb300 as se2
    import synth
    N, M, B = args.N, args.M, 64
    dev = torch.device("cuda", 0)
    plan = se2.Plan(N, M, batch=B, flags=se2.SHARED_KERNEL)
    f = torch.stack([synth.sample_bumps_torch(N, M, synth.make_problem(5, b, N, M, n_bumps=16).bumps, dev, torch.float32)
                     for b in range(B)]).contiguous().requires_grad_(True)
    target = torch.randn_like(f)
    params = torch.tensor([0.025, 0.25], dtype=torch.float64, device=dev, requires_grad=True)

    def step():
        out = se2.SE2Conv.apply(f, params, plan)
        loss = 0.5 * ((out - target) ** 2).sum()
        loss.backward()
    ms, clocks, launched = _clock_and_time(step, args.steps, args.warmup, dev, plans=(plan,))
    cpu = None
    if not args.no_cpu_baseline:
        import multiprocessing as mp
        n1, el1 = _oracle_adjoint_worker((N, M, 10.0))
        ncores = os.cpu_count() or 1
        with mp.get_context("spawn").Pool(ncores) as pool:
            res = pool.map(_oracle_adjoint_worker, [(N, M, 10.0)] * ncores)
        cpu = {"value": sum(n / el for n, el in res), "unit": "conv/s", "cores": ncores, "kind": "oracle",
               "nproc": ncores, "cpu_model": cpu_model(),
               "single_core": {"value": n1 / el1, "unit": "conv/s", "cores": 1},
               "sample": f"forward + adjoint steps of one problem (kernel samples and derivatives, coefficients, "
                         f"convolution, input gradient, two parameter partials), numpy FFT route, FP64: {n1} on "
                         f"one core in {el1:.1f} s; then {ncores} spawned processes, "
                         f"{sum(n for n, _ in res)} in about 10 s"}
    _line("SE(2) forward+adjoint convolutions/s at N=256, M=64, batch 64 (FP32)", B * args.steps / (ms / 1e3),
          "conv/s", args, ms, {"workload": "loss = 1/2||f * rho(sigma, sigma_theta) - target||^2, grads wrt f and "
                               "(sigma, sigma_theta); includes kernel sampling, 3 coefficient transforms, forward, adjoint",
                               "grid": [M, N, N], "global_batch": B},
          {"cpu_baseline": cpu, "clocks": clocks, "gpu_launches": launched})


if __name__ == "__main__":
    main()
