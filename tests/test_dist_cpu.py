"""The multi-rank host logic of bench.py, on CPU with the gloo backend.

With N GPUs every rank solves its own replica of a single-tensor workload, and the tensors of
the batched workload are split over the ranks (longest processing time first, by estimated
slice-SVD cost) with no collective on the data path; the only collective is the maximum of the
ranks' timings.  Two spawned gloo ranks check that they compute the same split, that the split
covers every tensor once with balanced loads, and that the maximum reaches every rank.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1407_1785_gb300 import synth  # noqa: E402


def _costs():
    return [bench.tensor_cost((s["n1"], s["n2"], s["n3"])) for s in synth.workload_batch_shapes(seed=1)]


def test_lpt_shard_covers_every_tensor_once_with_balanced_loads():
    costs = _costs()
    for world in (1, 2, 3, 4, 8):
        parts = bench.lpt_shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT is within 4/3 of the optimum, itself >= the mean load and >= the largest tensor
        assert max(loads) <= 4.0 / 3.0 * max(sum(costs) / world, max(costs)) + 1e-9


def test_max_over_ranks_without_a_process_group_is_the_value():
    assert bench.max_over_ranks(3.5) == 3.5


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, queue):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        mine = bench.lpt_shard(_costs(), world)[rank]
        tmax = bench.max_over_ranks(10.0 + rank)
        seen = [None] * world
        dist.all_gather_object(seen, mine)
        queue.put((rank, mine, tmax, seen))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_the_batch_and_agree_on_the_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    results = [queue.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    expect = bench.lpt_shard(_costs(), 2)
    for rank, mine, tmax, seen in results:
        assert tmax == 11.0                     # the slower rank's time reaches both
        assert mine == expect[rank]             # every rank computes the same split
        assert seen == expect
    assert sorted(results[0][1] + results[1][1]) == list(range(64))
