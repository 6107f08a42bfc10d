"""The N>1 path of bench.py on CPU: two gloo ranks (127.0.0.1) each take their
own problems (replicas, no data-path collective), run them through the FP64
oracle, and reduce their times with a max over ranks, as bench.py does on
GPUs with NCCL."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    from oracle import se2_oracle as O
    N, M, B = 16, 8, 3
    ids = bench.rank_problem_ids(rank, B)
    # every rank's problems are distinct from every other rank's
    gathered = [None] * world
    dist.all_gather_object(gathered, ids)
    flat = [i for g in gathered for i in g]
    assert len(flat) == len(set(flat)) == world * B
    F, P = bench.workload_inputs(N, M, B, rank)
    F, P = F.astype(np.float64), P.astype(np.float64)
    outs = [O.convolve(F[b], P[b]) for b in range(B)]
    # mass conservation of each replica's result (its own independent problems)
    for b in range(B):
        want = F[b].mean() * P[b].mean()
        assert abs(outs[b].mean() - want) < 1e-12 * abs(want)

    def reduce_max(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local_ms = 10.0 * (rank + 1)          # the slower rank sets the job's time
    ms, value = bench.aggregate(local_ms, B, world, reduce_max)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([ms, value]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_problems_and_take_the_max_time(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms, value = np.load(tmp_path / f"r{r}.npy")
        assert ms == 20.0                  # max over ranks, seen by every rank
        assert abs(value - 3 * 2 / 0.020) < 1e-9   # all ranks' units / the max time


def test_single_rank_aggregate_is_identity():
    import bench
    ms, value = bench.aggregate(4.0, 8, 1)
    assert ms == 4.0 and abs(value - 2000.0) < 1e-9
